"""3D lattices (axial layers of pin elements) and a dog-leg duct on the GPU, through the C ABI,
against the CPU oracle and closed forms:

- FP64 replay: the axially zoned assembly (partially inserted rods, fission) and the dog-leg duct
  give the oracle's event sequence, element indices and counters;
- FP32: their mesh flux agrees with the oracle (thousands of bins: the bar is the |z| a correct
  walk exceeds anywhere with probability 1e-3, at least 4; GPU errors from 256 batches, so their
  tails are normal); point-source escape from a purely absorbing 3D lattice agrees with the
  ray-marched quadrature;
- the batched launch gives the same fixed-point tallies as separate runs;
- invalid lattices are rejected on the host.
"""
import copy
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


def replay(prob, n, seed, per_history):
    o = oracle.run(prob, n, seed=seed, threads=THREADS, log_first=0, log_count=n, log_cap=per_history * n)
    p = mc.Problem(prob)
    p.run(n, seed, precision="fp64", log_first=0, log_count=n, log_capacity=per_history * n,
          bank_capacity=1 << 20)
    ev, eo = p.events(per_history * n), o.events
    assert len(ev) == len(eo) and len(ev) > 2 * n
    for f in ("tag", "k", "kind", "outcome", "n_child", "cell", "elem", "g"):
        assert np.array_equal(ev[f], eo[f]), f
    for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
        scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
        assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, f
    c = p.counters()
    for name in oracle.COUNTER_NAMES:
        assert c[name] == o.counters[name], name
    return p, ev


def bar(n):
    from scipy.stats import norm
    return max(4.0, float(norm.isf(5e-4 / n)))


def flux_z(prob, n_gpu, n_or, seed):
    o = oracle.run(prob, n_or, seed=seed, threads=THREADS)
    p = mc.Problem(prob)
    p.run(n_gpu, seed + 1, n_batches=256, bank_capacity=1 << 22)
    mg, sg = p.tally(0)
    mo, so = o.tallies[0]
    mg, sg, mo, so = (np.asarray(a, dtype=np.float64).ravel() for a in (mg, sg, mo, so))
    ok = (sg > 0) & (so > 0) & (sg < 0.1 * np.abs(mg)) & (so < 0.1 * np.abs(mo))
    c = p.counters()
    p.close()
    return (mg[ok] - mo[ok]) / np.sqrt(sg[ok] ** 2 + so[ok] ** 2), c


def test_axial_lattice_fp64_replay(torch):
    prob = P.axial_lattice()
    p, ev = replay(prob, 2000, 85, 400)
    lat = prob["lattice"]
    walls = ev[(ev["kind"] == 1) & (ev["outcome"] == 3)]
    layers = walls["elem"] // (lat["nx"] * lat["ny"])
    assert layers.min() == 0 and layers.max() == lat["nz"] - 1
    p.close()


def test_dogleg_duct_fp64_replay(torch):
    p, _ = replay(P.dogleg_duct(), 4000, 86, 100)
    assert p.counters()["reflect"] > 0
    p.close()


def test_axial_lattice_fp32_against_oracle(torch):
    z, c = flux_z(P.axial_lattice(), 2_048_000, 100_000, 87)
    assert z.size > 1000 and np.all(np.abs(z) < bar(z.size)), (np.abs(z).max(), z.size)
    assert c["lost"] == 0


def test_dogleg_duct_fp32_against_oracle(torch):
    z, c = flux_z(P.dogleg_duct(), 4_096_000, 200_000, 88)
    assert z.size > 100 and np.all(np.abs(z) < bar(z.size)), (np.abs(z).max(), z.size)
    assert c["lost"] == 0


@pytest.mark.parametrize("point", [(1.3, 1.7, 1.2), (2.1, 1.8, 0.4), (2.1, 0.8, 0.4)])
def test_point_escape_from_3d_lattice_fp32(torch, point):
    prob = P.lattice_absorber_3d(point=point)
    exact = CF.lattice_point_escape(prob, 20000, 0.004, 0)
    p = mc.Problem(prob)
    n = 4_000_000
    p.run(n, 89)
    lm, _ = p.leakage()
    esc = float(lm.sum())
    assert abs(esc - exact) < 4 * math.sqrt(exact * (1 - exact) / n), (esc, exact)
    c = p.counters()
    assert c["lost"] == 0 and c["capture"] + c["leak"] == c["source"]
    p.close()


def test_batched_3d_lattice_equals_separate_runs(torch):
    probs = [P.axial_lattice(), P.dogleg_duct(), P.lattice_absorber_3d()]
    nh = [20000, 30000, 40000]
    ps = [mc.Problem(q) for q in probs]
    ref = []
    for i, p in enumerate(ps):
        p.run(nh[i], 90 + i, bank_capacity=1 << 20)
        ref.append((p.tally_batches(0), p.counters()))
    mc.run_batch([p.h for p in ps], nh, 90, mc.run_opts(batch_unit=64))
    for i, p in enumerate(ps):
        assert np.array_equal(p.tally_batches(0), ref[i][0]), probs[i]["name"]
        got = {k: v for k, v in p.counters().items() if k != "iterations"}
        assert got == {k: v for k, v in ref[i][1].items() if k != "iterations"}, probs[i]["name"]
    for p in ps:
        p.close()


@pytest.mark.parametrize("corner", ["low", "high"])
def test_largest_lattice_fp64_replay(torch, corner):
    """64 x 64 x 16 = 65536 elements (the most the element index holds), scattering materials, a
    point source in the first or the last element: the walk and its element indices replay the
    oracle's."""
    point = (0.03, 0.03, 0.1) if corner == "low" else (6.37, 6.37, 7.9)
    prob = P.lattice_absorber_3d(n=64, nz=16, pitch=0.1, pitch_z=0.5, radius=0.035, point=point)
    for m in prob["materials"]:
        m["sigma_s"] = [[0.6 * m["sigma_t"][0]]]
    n = 500
    p, ev = replay(prob, n, 91, 400)
    first = ev["elem"][ev["k"] == 0]
    assert np.all(first == (0 if corner == "low" else 65535))
    assert len(np.unique(ev["elem"])) > 500
    p.close()


def test_invalid_lattices_rejected_on_the_host(torch):
    base = P.axial_lattice()
    bad = []
    q = copy.deepcopy(base); q["lattice"]["pitch_z"] = 0.0; bad.append(q)
    q = copy.deepcopy(base); q["lattice"]["pin_material"][7] = 9; bad.append(q)  # no material 9
    q = copy.deepcopy(base)
    q["lattice"].update(nx=200, ny=200, nz=2, pin_material=[-1] * 80000)  # over 65536 elements
    bad.append(q)
    for q in bad:
        with pytest.raises(mc.McError) as e:
            mc.Problem(q)
        assert e.value.code == mc.MC_ERR_INVALID
