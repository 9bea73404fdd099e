"""Batched persistent launch (mc_run_batch) and its autotuner, through the C ABI.

- Identity: random numbers are keyed by (seed, particle lineage, event), tallies are integers, and
  problem i of a batch uses seed + i, so every problem's fixed-point batch tallies and event
  counters equal those of a separate mc_run with that seed, in FP32 and FP64 tracking, whatever
  the block size, register budget or work-unit size.
- Statistics: a batched problem agrees with the CPU oracle within 4 sigma.
- Scheduling: per-problem completion times are reported, short problems finish first, a failing
  problem stops alone.
"""
import numpy as np
import pytest

import oracle
from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _t


def conserved(c):
    started = c["source"] + c["secondary"] + c["ww_split"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"]
    return started == ended


def mixed_batch(n=10, n_lo=2_000, n_hi=40_000):
    """A few problems of every kind of the uneven workload (1D slab, 2D slab, small lattice with
    secondary production), the slab of the first workload, and the supercritical AZURV1 medium
    (deep secondary stacks, census)."""
    probs, nh = P.config5(seed=11, n_problems=n, n_lo=n_lo, n_hi=n_hi)
    probs += [P.config1(), P.azurv1()]
    nh += [30_000, 3_000]
    return probs, nh


def results(p, n_tallies):
    out = [p.tally_batches(t) for t in range(n_tallies + 1)]  # mesh tallies and the leakage tally
    c = p.counters()
    c.pop("iterations")
    return out, c


def assert_same(a, b, what):
    (ta, ca), (tb, cb) = a, b
    for i, (x, y) in enumerate(zip(ta, tb)):
        assert np.array_equal(x, y), f"{what}: tally {i} differs"
    assert ca == cb, f"{what}: counters differ"


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_separate_runs(torch, precision):
    probs, nh = mixed_batch()
    ps = [mc.Problem(q) for q in probs]
    seed = 77
    ref = []
    for i, (p, q) in enumerate(zip(ps, probs)):
        p.run(nh[i], seed + i, precision=precision, bank_capacity=1 << 20)
        ref.append(results(p, len(q["tallies"])))
    o = mc.run_opts(precision=precision, batch_unit=64)
    mc.run_batch([p.h for p in ps], nh, seed, o)
    for i, (p, q) in enumerate(zip(ps, probs)):
        got = results(p, len(q["tallies"]))
        assert conserved(got[1]), q["name"]
        assert_same(got, ref[i], q["name"])
    for p in ps:
        p.close()


def test_batch_configurations_and_replays_identical(torch):
    """Block size, register budget and work-unit size change the schedule only; graph replays of
    one plan and a second plan with the same shape give the same numbers."""
    probs, nh = mixed_batch(n=6)
    ps = [mc.Problem(q) for q in probs]
    hs = [p.h for p in ps]
    ref = None
    for block, bps, unit in ((256, 0, 128), (128, 0, 32), (256, 2, 512), (128, 2, 1), (256, 0, 128)):
        mc.run_batch(hs, nh, 5, mc.run_opts(block_size=block, blocks_per_sm=bps, batch_unit=unit))
        got = [results(p, len(q["tallies"])) for p, q in zip(ps, probs)]
        if ref is None:
            ref = got
        else:
            for i in range(len(ps)):
                assert_same(got[i], ref[i], f"{probs[i]['name']} block={block} bps={bps} unit={unit}")
    for p in ps:
        p.close()


def test_batched_problems_match_oracle(torch):
    """Two batched problems (the 1D slab with leakage, a lattice with secondary production)
    against the FP64 oracle: 4 sigma of the combined error on every well-sampled bin."""
    lat = P.config5(seed=3, n_problems=8)[0]
    lat = [q for q in lat if q["name"].endswith("lattice")][0]
    probs = [P.config1(), lat]
    nh = [2_000_000, 400_000]
    ps = [mc.Problem(q) for q in probs]
    mc.run_batch([p.h for p in ps], nh, 9)
    for p, q, n in zip(ps, probs, nh):
        o = oracle.run(q, n // 10, seed=4, threads=16)
        for t in range(len(q["tallies"])):
            mg, sg = p.tally(t)
            mo, so = o.tallies[t]
            mg, sg, mo, so = (np.ravel(a) for a in (mg, sg, mo, so))
            ok = (sg > 0) & (so > 0) & (sg < 0.1 * np.abs(mg)) & (so < 0.1 * np.abs(mo))
            z = (mg[ok] - mo[ok]) / np.sqrt(sg[ok] ** 2 + so[ok] ** 2)
            assert z.size >= 10 and np.all(np.abs(z) < 4.0), (q["name"], z.size, np.abs(z).max())
        assert conserved(p.counters())
    for p in ps:
        p.close()


def test_batch_wall_times(torch):
    probs, nh = P.config5(seed=5, n_problems=48, n_lo=1e3, n_hi=1e5)
    ps = [mc.Problem(q) for q in probs]
    wall = mc.run_batch([p.h for p in ps], nh, 1, wall=True)
    assert np.all(np.isfinite(wall)) and np.all(wall > 0)
    # within a geometry kind problems are scheduled in ascending size: the smallest finishes
    # before the largest
    for lattice in (False, True):
        idx = [i for i, q in enumerate(probs) if q["name"].endswith("lattice") == lattice]
        order = sorted(idx, key=lambda i: nh[i])
        assert wall[order[0]] <= wall[order[-1]]
    for p in ps:
        assert p.timing()[0] > 0.0
        assert conserved(p.counters())
    for p in ps:
        p.close()


def test_failing_problem_stops_alone(torch):
    """A source box that pokes out of the slab loses particles: that problem reports
    MC_ERR_LOST, the others finish and equal their separate runs."""
    bad = P.slab_problem(L=5.0, src_hi=6.0, name="leaky_source")
    good = [P.config1(), P.config5(seed=2, n_problems=1)[0][0]]
    ps = [mc.Problem(q) for q in [good[0], bad, good[1]]]
    nh = [20_000, 20_000, 20_000]
    mc.run_batch([p.h for p in ps], nh, 40)
    with pytest.raises(mc.McError) as e:
        ps[1].wait()
    assert e.value.code == mc.MC_ERR_LOST
    for k in (0, 2):
        q = good[0 if k == 0 else 1]
        got = results(ps[k], len(q["tallies"]))
        ps[k].run(nh[k], 40 + k)
        assert_same(got, results(ps[k], len(q["tallies"])), q["name"])
    for p in ps:
        p.close()


def test_autotuner_picks_a_candidate_and_reuses_it(torch):
    probs, nh = P.config5(seed=8, n_problems=16, n_lo=1e3, n_hi=3e4)
    ps = [mc.Problem(q) for q in probs]
    hs = [p.h for p in ps]
    tuned, ms = mc.batch_tune(hs, nh, 3)
    assert tuned.block_size in (128, 256) and tuned.blocks_per_sm in (0, 2)
    assert tuned.batch_unit in (32, 64, 128, 256, 512) and ms > 0.0
    ref = [results(p, len(q["tallies"])) for p, q in zip(ps, probs)]
    mc.run_batch(hs, nh, 3)  # default options: the stored configuration for this shape
    for i, (p, q) in enumerate(zip(ps, probs)):
        assert_same(results(p, len(q["tallies"])), ref[i], q["name"])
    for p in ps:
        p.close()


def test_batch_argument_errors(torch):
    ps = [mc.Problem(P.config1()) for _ in range(2)]
    with pytest.raises(mc.McError) as e:
        mc.run_batch([ps[0].h, ps[0].h], [100, 100], 1)  # the same problem twice
    assert e.value.code == mc.MC_ERR_INVALID
    with pytest.raises(mc.McError) as e:
        mc.run_batch([p.h for p in ps], [100, 1], 1)  # fewer histories than batches
    assert e.value.code == mc.MC_ERR_INVALID
    with pytest.raises(mc.McError) as e:
        mc.run_batch([p.h for p in ps], [100, 100], 1, mc.run_opts(ww_enable=1))
    assert e.value.code == mc.MC_ERR_STATE
    for p in ps:
        p.close()


@pytest.mark.parametrize("algorithm", ["event", "history"])
def test_corner_crossing_terminates(torch, algorithm):
    """FP32 regression: history 218025 of the 2D slab that is problem 32 of the uneven workload
    (seed 538) flies exactly onto the point where the four cells meet, heading into the cell it
    is not in.  The corner is resolved by the direction of flight, so the history ends normally
    instead of crossing back and forth between two cells in zero-length flights until the
    per-particle watchdog stops it."""
    prob = P.config5()[0][32]
    assert prob["name"] == "p32_slab2d"
    p = mc.Problem(prob)
    p.run(2, 538, first_history=218024, n_batches=2, algorithm=algorithm)
    p.wait()
    c = p.counters()
    assert conserved(c) and c["flight"] < 10_000, c
    p.close()


def test_full_uneven_workload_runs_clean(torch):
    """The whole 256-problem workload (about 5.5e7 histories) on three seeds: no problem loses a
    particle or overflows (this caught crossings next to a reflecting wall that rounded to just
    outside it), and every problem conserves particles."""
    probs, nh = P.config5()
    ps = [mc.Problem(q) for q in probs]
    hs = [p.h for p in ps]
    for seed in (5, 6, 105):
        mc.run_batch(hs, nh, seed)
        for p, q in zip(ps, probs):
            p.wait()
            assert conserved(p.counters()), (seed, q["name"])
    for p in ps:
        p.close()
