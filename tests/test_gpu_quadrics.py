"""Quadric surfaces on the GPU (spheres, cylinders along x and y, general quadrics; through the C
ABI) against the CPU oracle and closed forms:

- FP64 replay: a reflective box holding a sphere, a cylinder along x and a rotated ellipsoid, each a
  scattering region: the event sequence and every counter equal the oracle's;
- FP32: the same problem's mesh flux agrees with the oracle within 4 sigma; point-source escape
  from absorbing quadric bodies agrees with quadrature; the three cylinder orientations agree.
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


def test_quadric_assembly_fp64_replay(torch):
    prob = P.quadric_assembly()
    n = 5000
    o = oracle.run(prob, n, seed=71, threads=THREADS, log_first=0, log_count=n, log_cap=400 * n)
    p = mc.Problem(prob)
    p.run(n, 71, precision="fp64", log_first=0, log_count=n, log_capacity=400 * n)
    ev, eo = p.events(400 * n), o.events
    assert len(ev) == len(eo) and len(ev) > 5 * n
    assert np.array_equal(ev["tag"], eo["tag"]) and np.array_equal(ev["k"], eo["k"])
    for f in ("kind", "outcome", "cell", "g"):
        assert np.array_equal(ev[f], eo[f]), f
    for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
        scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
        assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, f
    c = p.counters()
    for name in oracle.COUNTER_NAMES:
        assert c[name] == o.counters[name], name
    assert c["surface"] > c["reflect"]  # quadric crossings happened
    p.close()


def test_quadric_assembly_fp32_against_oracle(torch):
    prob = P.quadric_assembly()
    o = oracle.run(prob, 400_000, seed=72, threads=THREADS)
    p = mc.Problem(prob)
    p.run(4_000_000, 73)
    mg, sg = p.tally(0)
    mo, so = o.tallies[0]
    ok = (sg > 0) & (so > 0) & (sg < 0.1 * np.abs(mg)) & (so < 0.1 * np.abs(mo))
    z = (mg[ok] - mo[ok]) / np.sqrt(sg[ok] ** 2 + so[ok] ** 2)
    assert ok.sum() > 100 and np.all(np.abs(z) < 4), np.abs(z).max()
    assert p.counters()["lost"] == 0
    p.close()


@pytest.mark.parametrize("case", ["sphere_off", "cyl_x", "cyl_y", "cyl_z", "ellipsoid_rot"])
def test_point_source_escape_fp32(torch, case):
    if case == "sphere_off":
        prob = P.sphere_absorber(1.5, 1.0, point=(1.3, 0.5, 0.2), center=(1.0, 0.4, -0.1))
        exact = CF.sphere_point_escape(1.0, 1.5, math.sqrt(0.19))
    elif case.startswith("cyl"):
        prob, exact = P.xcylinder_absorber(0.8, 1.5, 1.0, axis=case[-1]), CF.cylinder_point_escape(1.0, 0.8, 1.5)
    else:
        ang, c0, p0 = (0.7, -0.4, 1.1), (0.3, -0.5, 0.8), (0.55, -0.3, 1.1)
        prob = P.ellipsoid_absorber(1.0, 0.6, 1.5, angles=ang, center=c0, point=p0)
        exact = CF.quadric_body_point_escape(1.0, P.ellipsoid_matrix(1.0, 0.6, 1.5, ang), c0, p0)
    p = mc.Problem(prob)
    n = 4_000_000
    p.run(n, 74)
    lm, _ = p.leakage()
    esc = float(lm.sum())
    assert abs(esc - exact) < 4 * math.sqrt(exact * (1 - exact) / n), (case, esc, exact)
    c = p.counters()
    assert c["lost"] == 0 and c["capture"] + c["leak"] == c["source"]
    p.close()
