"""Split runs on the CUDA path (through the C ABI): the event-based launch followed by the
history-style tail launch with per-warp stacks of secondaries must give exactly the results of the
one-launch run, since every random number is keyed by the particle and fixed-point tallies do not
depend on the order of their adds.

- The lattice (production, so secondaries in every generation of the tail) and the 1D slab: a
  default run (split), a run whose bank is too small for stacks (one launch), history-based runs
  (the whole run in the tail launch), and tails that start early (16x the default drain threshold,
  and a threshold above the whole run) give equal tallies and counters.
- A run that ends inside the event-based launch (no history-style iteration left) adds nothing in
  the tail launch: the leakage of a purely absorbing slab is the E3 closed form, and the counters
  match a one-launch run.
- mc_run_launches counts each kind of run's kernels.
"""
import numpy as np
import pytest

from oracle import closed_forms as CF
from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _t


@pytest.mark.parametrize("name,n", [("config3", 300_000), ("config1", 1_000_000)])
def test_split_run_equals_one_launch(torch, name, n):
    p = mc.Problem(getattr(P, name)())
    # 2^16 particles leave fewer than 32 per warp for stacks: the run stays one launch
    p.run(n, 41, bank_capacity=1 << 16)
    ref_t, ref_c = p.tally_batches(0), {k: v for k, v in p.counters().items() if k != "iterations"}
    ref_l = p.leakage()
    for opts in ({}, {"algorithm": "history"}, {"drain_threshold": 16 * 2 * 152 * 3 * 256},
                 {"drain_threshold": 1 << 40}):
        p.run(n, 41, **opts)
        c = {k: v for k, v in p.counters().items() if k != "iterations"}
        assert np.array_equal(p.tally_batches(0), ref_t), opts
        assert c == ref_c, (opts, c, ref_c)
        lm, ls = p.leakage()
        assert np.array_equal(lm, ref_l[0]) and np.array_equal(ls, ref_l[1]), opts
    p.close()


def test_run_ending_in_the_event_launch(torch):
    """Sigma_s = 0: every particle ends at its first event, so the last event-based iteration
    leaves no work; the tail launch must then add nothing."""
    prob = P.config1(sigma_s=0.0)
    pl, pr = CF.slab_leakage(1.0, 5.0, 1.0)
    p = mc.Problem(prob)
    p.run(2_000_000, 43)
    lm, ls = (a.ravel() for a in p.leakage())
    assert abs(lm[0] - pl) < 4 * ls[0] and abs(lm[1] - pr) < 4 * ls[1]
    c_split = {k: v for k, v in p.counters().items() if k != "iterations"}
    t_split = p.tally_batches(0)
    p.run(2_000_000, 43, bank_capacity=1 << 16)
    assert {k: v for k, v in p.counters().items() if k != "iterations"} == c_split
    assert np.array_equal(p.tally_batches(0), t_split)
    assert c_split["source"] == 2_000_000
    p.close()


def test_launch_count_of_each_kind_of_run(torch):
    """mc_run_launches: a split run is two transport launches, a one-launch run one; the range
    walk adds its reconstruction and every run its batch statistics."""
    p = mc.Problem(P.config3())
    p.run(100_000, 44)
    assert p.launches() == 3  # event-based part, tail, statistics
    p.run(100_000, 44, bank_capacity=1 << 16)
    assert p.launches() == 2  # too small a bank for stacks: one transport launch
    p.run(100_000, 44, precision="fp64")
    assert p.launches() == 2  # FP64 tracking is not split
    p.close()
    q = mc.Problem(P.config2())
    q.run(1_000_000, 45)
    assert q.launches() == 4  # event-based part, tail, range-walk reconstruction, statistics
    q.close()
