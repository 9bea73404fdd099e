"""Edge cases of the GPU path (through the C ABI): the largest sizes the ABI allows for groups and
surfaces, a very fine time axis, a run with no mesh tally, the smallest history count, an all-void
problem; and invalid inputs rejected on the host before any CUDA call.  Checked against the CPU
oracle, closed forms or exact counts.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu

THREADS = 16


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return _t


def combined_z(mg, sg, mo, so, rel_max=0.1):
    mg, sg, mo, so = (np.asarray(a, dtype=np.float64).ravel() for a in (mg, sg, mo, so))
    ok = (sg > 0) & (so > 0) & (sg < rel_max * np.abs(mg)) & (so < rel_max * np.abs(mo))
    return (mg[ok] - mo[ok]) / np.sqrt(sg[ok] ** 2 + so[ok] ** 2)


def test_max_groups_against_oracle(torch):
    prob = P.config2(G=mc.MAX_GROUPS, n_tbins=20)
    o = oracle.run(prob, 200_000, seed=101, threads=THREADS)
    p = mc.Problem(prob)
    p.run(2_000_000, 102)
    z = combined_z(*p.tally(0), *o.tallies[0])
    assert z.size > 200 and np.all(np.abs(z) < 4), np.abs(z).max()
    p.run(2000, 103, precision="fp64", log_first=0, log_count=2000, log_capacity=400 * 2000)
    o = oracle.run(prob, 2000, seed=103, threads=THREADS, log_first=0, log_count=2000, log_cap=400 * 2000)
    ev = p.events(400 * 2000)
    assert np.array_equal(ev["g"], o.events["g"]) and np.array_equal(ev["tag"], o.events["tag"])
    p.close()


def test_max_surfaces_against_oracle(torch):
    """254 layers: 255 planes (the ABI's limit) and 254 cells."""
    prob = P.slab_stack(thickness=5.08, n_layers=254, G=3, ww_bin=0.508, name="thin254")
    assert len(prob["surfaces"]) == mc.MAX_SURFACES
    o = oracle.run(prob, 200_000, seed=104, threads=THREADS)
    p = mc.Problem(prob)
    p.run(2_000_000, 105)
    z = combined_z(*p.tally(1), *o.tallies[1])
    assert z.size > 15 and np.all(np.abs(z) < 4), np.abs(z).max()
    z = combined_z(*p.leakage(), o.leak_mean, o.leak_std)  # the two vacuum ends (the far one faint)
    assert z.size >= 1 and np.all(np.abs(z) < 4)
    c = p.counters()
    assert c["lost"] == 0 and c["surface"] > 10 * c["source"]
    p.close()


def test_fine_time_axis_against_expm(torch):
    """4096 log-spaced time bins (the range walk): aggregated 64 bins at a time, the track length
    agrees with the matrix exponential; errors from the batch values."""
    prob = P.config2(n_tbins=4096)
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    exact = CF.multigroup_time_bins(mat, v, te).sum(axis=0).reshape(64, 64).sum(axis=1)
    p = mc.Problem(prob)
    p.run(4_096_000, 106, n_batches=64)
    b = p.tally_batches(0).reshape(64, 7, 64, 64).sum(axis=(1, 3))  # [batch][64 coarse bins]
    m, s = b.mean(axis=0), b.std(axis=0, ddof=1) / math.sqrt(64)
    ok = (s > 0) & (s < 0.1 * np.abs(m))
    z = (m[ok] - exact[ok]) / s[ok]
    assert ok.sum() > 40 and np.all(np.abs(z) < 4), np.abs(z).max()
    p.close()


def test_no_mesh_tally_leakage_closed_form(torch):
    """A slab with no mesh tally at all: only the per-surface leakage, against the E3 closed form."""
    prob = P.with_tallies(P.config1(sigma_s=0.0), [])
    pl, pr = CF.slab_leakage(1.0, 5.0, 1.0)
    p = mc.Problem(prob)
    p.run(4_000_000, 107)
    lm, ls = (a.ravel() for a in p.leakage())
    assert abs(lm[0] - pl) < 4 * ls[0] and abs(lm[1] - pr) < 4 * ls[1]
    p.close()


def test_fewest_histories_replay(torch):
    """As many histories as batches (the smallest run allowed), replayed event by event in FP64."""
    prob = P.config3()
    n = 32
    o = oracle.run(prob, n, seed=108, threads=THREADS, log_first=0, log_count=n, log_cap=2000 * n)
    p = mc.Problem(prob)
    p.run(n, 108, precision="fp64", log_first=0, log_count=n, log_capacity=2000 * n)
    ev = p.events(2000 * n)
    assert len(ev) == len(o.events) > n
    for f in ("tag", "k", "kind", "outcome", "cell", "elem", "g"):
        assert np.array_equal(ev[f], o.events[f]), f
    with pytest.raises(mc.McError) as e:
        p.run(n - 1, 108)
    assert e.value.code == mc.MC_ERR_INVALID
    p.close()


def test_all_void_slab_leaks_every_particle(torch):
    prob = P.slab_problem(5.0, 0.0, 0.0)
    p = mc.Problem(prob)
    for precision in ("fp32", "fp64"):
        p.run(1_000_000, 109, precision=precision)
        c = p.counters()
        assert c["leak"] == c["source"] == 1_000_000 and c["collision"] == 0 and c["lost"] == 0
        lm, ls = p.leakage()
        assert float(lm.sum()) == 1.0 and float(ls.sum()) == 0.0 or abs(float(lm.sum()) - 1.0) < 1e-12
    p.close()


def test_invalid_problems_rejected_on_the_host(torch):
    base = P.config1()
    bad = []
    q = dict(base); q["G"] = mc.MAX_GROUPS + 1; bad.append(q)
    q = P.with_tallies(base, [P.mesh(x=[0.0, 1.0, 0.5])]); bad.append(q)  # edges not increasing
    q = dict(base); q["surfaces"] = [dict(base["surfaces"][0], kind="SQ", coef=[0, 0, 0, -1.0])] + base["surfaces"][1:]
    bad.append(q)  # negative radius
    q = dict(base); q["surfaces"] = [dict(base["surfaces"][0], kind="CX", bc="reflect")] + base["surfaces"][1:]
    bad.append(q)  # reflection on a cylinder
    q = P.with_tallies(base, [P.mesh(x=[0.0, 5.0], t=[0.0, 1.0, math.inf], estimator="crossing")]); bad.append(q)
    for q in bad:
        with pytest.raises(mc.McError) as e:
            mc.Problem(q)
        assert e.value.code == mc.MC_ERR_INVALID


def test_tables_beyond_shared_memory_rejected_and_library_still_usable(torch):
    """The transport kernels keep the problem's tables in shared memory: 255 materials x 32 groups
    (a 1 MB scatter table) cannot fit, and the run says so with MC_ERR_INVALID before any launch;
    the failed attempt leaves nothing behind for the next calls (a run, an MLP)."""
    prob = P.config2(G=mc.MAX_GROUPS, n_tbins=4)
    prob["materials"] = prob["materials"] * 255
    p = mc.Problem(prob)
    with pytest.raises(mc.McError) as e:
        p.run(10000, 110)
    assert e.value.code == mc.MC_ERR_INVALID and "shared memory" in str(e.value)
    p.close()
    q = mc.Problem(P.config1())
    q.run(100000, 111)
    assert q.counters()["source"] == 100000
    q.close()
    net = mc.Mlp(P.mlp_init(seed=3))
    net.close()
