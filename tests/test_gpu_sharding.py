"""History-range sharding on the CUDA path: runs of disjoint history ranges (first_history) that
cover [0, N) add up to the run of [0, N) in every tally bin's exact int64 fixed-point sum and in
every event counter.  This is the exchange step of a multi-GPU run (each GPU a history range, one
integer all-reduce of the sums) and the resume of a run cut short (run the remaining range, add);
it holds for any split because every random number is keyed by the particle's lineage, not by the
schedule, and integer sums do not depend on the order of their terms.  Bit for bit, except in the
bins of a range-walk tally (a time axis much finer than its mesh, as on the 7-group pulse): there
the track length of fully crossed time bins is formed once per statistical batch after the run,
rounded to the fixed-point unit, so shards (whose batches are other groups of histories) differ
from the whole by at most half a unit per batch and bin."""
import numpy as np
import pytest

from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _t


def _range_walk(tally):
    """The library's rule: a time axis much finer than the mesh is scored by the range walk."""
    nx, ny, nz, nt = (len(tally[k]) - 1 for k in ("x", "y", "z", "t"))
    return nt >= 3 and nt >= 4 * (nx + ny + nz)


def _sums(p, n_tallies):
    return [p.tally_sums(t)[0].copy() for t in range(n_tallies + 1)]  # mesh tallies, then leakage


@pytest.mark.parametrize("name,precision,n", [
    ("config2", "fp32", 2_000_000), ("config3", "fp32", 1_000_000),
    ("config2", "fp64", 200_000), ("config3", "fp64", 100_000),
])
def test_history_range_shards_add_up_exactly(torch, name, precision, n):
    prob = P.by_name(name)
    nt = len(prob["tallies"])
    p = mc.Problem(prob)
    seed = 31
    p.run(n, seed, precision=precision)
    whole, cw = _sums(p, nt), p.counters()
    assert np.count_nonzero(whole[0]) > 100
    cuts = [0, n // 3, n // 2 + 7, n]  # uneven shards, one of them odd
    parts, counters = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        p.run(b - a, seed, precision=precision, first_history=a)
        parts.append(_sums(p, nt))
        counters.append(p.counters())
    nb = 32  # batches of every run
    for t in range(nt + 1):
        diff = np.abs(whole[t] - sum(part[t] for part in parts))
        tal = prob["tallies"][t] if t < nt else None
        rng = tal is not None and _range_walk(tal)
        # half a unit per batch and bin of the whole run and of each shard
        assert diff.max() <= (0.5 * nb * (1 + len(parts)) if rng else 0), (t, int(diff.max()))
    for k in ("source", "secondary", "capture", "production", "leak", "census", "flight", "collision",
              "scatter", "surface", "reflect", "scores"):
        assert cw[k] == sum(c[k] for c in counters), k
    p.close()
