"""Pins of the oracle's quadric surfaces (spheres, cylinders along x / y, general quadrics; the paper's
quadric-surface CSG, Section 3) on the CPU:

* distances by hand: sphere from the centre, from outside, moving away, grazing; cylinders along and
  across their axes; a one-sheet hyperboloid (a concave section, leading coefficient < 0);
* escape probabilities of an isotropic point source in purely absorbing bodies against quadrature:
  a sphere (from an off-centre point), finite cylinders along x, y and z, an ellipsoid written as a
  general quadric;
* a transparent sphere inside a scattering medium leaves the flux unchanged.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import problems as P

THREADS = 8
INF = math.inf


def test_quadric_distances_by_hand():
    sph = P.sphere_absorber(1.0)
    d = lambda *a: oracle.dist_surface(sph, 0, *a)
    assert d((0, 0, 0), (1, 0, 0), -1) == pytest.approx(1.0, abs=1e-15)
    assert d((2, 0, 0), (-1, 0, 0), +1) == pytest.approx(1.0, abs=1e-15)
    assert d((2, 0, 0), (1, 0, 0), +1) == INF  # moving away
    assert d((-2, 1, 0), (1, 0, 0), +1) == INF  # grazing: a chord of length 0
    inside = d((-2, 1 - 1e-8, 0), (1, 0, 0), +1)  # a chord of 2.8e-4 cm is entered
    assert inside == pytest.approx(2.0, abs=1e-3)
    s = 1 / math.sqrt(3)
    assert d((0.1, 0.2, 0.3), (s, s, s), -1) == pytest.approx(
        -0.6 * s + math.sqrt(0.36 * s * s - (0.14 - 1)), rel=1e-12)
    cx = P.xcylinder_absorber(1.0, 2.0, axis="x")
    assert oracle.dist_surface(cx, 0, (0.5, 0, 0), (1, 0, 0), -1) == INF  # along the axis
    assert oracle.dist_surface(cx, 0, (0, 0.5, 0), (0, 1, 0), -1) == pytest.approx(0.5, abs=1e-15)
    assert oracle.dist_surface(cx, 0, (7, 0, -3), (0, 0, 1), +1) == pytest.approx(2.0, abs=1e-15)
    cy = P.xcylinder_absorber(1.0, 2.0, axis="y")
    assert oracle.dist_surface(cy, 0, (0, 3, 0.5), (0, 1, 0), -1) == INF
    assert oracle.dist_surface(cy, 0, (0, 3, 0.5), (0, 0, -1), -1) == pytest.approx(1.5, abs=1e-15)
    ell = P.ellipsoid_absorber(1.0, 0.6, 1.5)
    assert oracle.dist_surface(ell, 0, (0, 0, 0), (0, 0, 1), -1) == pytest.approx(1.5, rel=1e-14)
    assert oracle.dist_surface(ell, 0, (0, 0, 0), (0, -1, 0), -1) == pytest.approx(0.6, rel=1e-14)
    # x^2 + y^2 - z^2 - 1 = 0 (one sheet): from the origin the neck is left only sideways
    hyp = dict(sph)
    hyp["surfaces"] = [{"kind": "GQ", "coef": [1, 1, -1, 0, 0, 0, 0, 0, 0, -1], "bc": "interior"}] + sph["surfaces"][1:]
    assert oracle.dist_surface(hyp, 0, (0, 0, 0), (0, 0, 1), -1) == INF
    assert oracle.dist_surface(hyp, 0, (0, 0, 0), (1, 0, 0), -1) == pytest.approx(1.0, abs=1e-15)
    assert oracle.dist_surface(hyp, 0, (0, 0, 0), (s * math.sqrt(1.5), 0, s * math.sqrt(1.5)), -1) == INF


def escape(prob, n, seed):
    r = oracle.run(prob, n, seed=seed, threads=THREADS)
    p = r.leak_mean.sum()
    return p, math.sqrt(p * (1 - p) / n), r


@pytest.mark.parametrize("case", ["sphere", "sphere_off", "cyl_x", "cyl_y", "cyl_z", "ellipsoid", "ellipsoid_rot"])
def test_point_source_escape_from_quadric_bodies(case):
    if case == "sphere":
        prob, exact = P.sphere_absorber(1.0, 1.2), CF.sphere_point_escape(1.2, 1.0, 0.0)
    elif case == "sphere_off":
        prob = P.sphere_absorber(1.5, 1.0, point=(1.3, 0.5, 0.2), center=(1.0, 0.4, -0.1))
        exact = CF.sphere_point_escape(1.0, 1.5, math.sqrt(0.09 + 0.01 + 0.09))
    elif case.startswith("cyl"):
        prob, exact = P.xcylinder_absorber(0.8, 1.5, 1.0, axis=case[-1]), CF.cylinder_point_escape(1.0, 0.8, 1.5)
    elif case == "ellipsoid":
        prob, exact = P.ellipsoid_absorber(1.0, 0.6, 1.5), CF.ellipsoid_point_escape(1.0, 1.0, 0.6, 1.5)
    else:
        # rotated, moved and seen from an off-centre point: every coefficient of the quadric in use,
        # the exact escape from the matrix form of the body
        ang, c0, p0 = (0.7, -0.4, 1.1), (0.3, -0.5, 0.8), (0.55, -0.3, 1.1)
        prob = P.ellipsoid_absorber(1.0, 0.6, 1.5, angles=ang, center=c0, point=p0)
        exact = CF.quadric_body_point_escape(1.0, P.ellipsoid_matrix(1.0, 0.6, 1.5, ang), c0, p0)
    p, s, r = escape(prob, 400_000, 61)
    assert abs(p - exact) < 4 * s, (case, p, exact, s)
    c = r.counters
    assert c["lost"] == 0 and c["capture"] + c["leak"] == c["source"]


def test_transparent_sphere_in_a_scattering_medium():
    """A sphere that separates two cells of the same scattering material is invisible: the total
    flux of a one-group infinite medium stays 1 / Sigma_a."""
    surfs, hs = P.box_surfaces((-5, -5, -5), (5, 5, 5), "reflect")
    surfs = surfs + [{"kind": "SQ", "coef": [0.5, -0.2, 0.3, 2.0], "bc": "interior"}]
    k = len(surfs) - 1
    cells = [{"halfspaces": hs + [(k, -1)], "material": 0}, {"halfspaces": hs + [(k, +1)], "material": 0}]
    mat = P.material([1.0], [[0.6]])
    prob = P.problem("transparent", 1, [1.0], [mat], surfs, cells,
                     P.source("box", (-5, -5, -5), (5, 5, 5), "iso", 1), [P.mesh(x=(-5, 5), y=(-5, 5), z=(-5, 5))])
    r = oracle.run(prob, 200_000, seed=62, threads=THREADS)
    m, s = r.tallies[0]
    assert abs(m.ravel()[0] - 1 / 0.4) < 4 * s.ravel()[0]
    assert r.counters["lost"] == 0 and r.counters["surface"] > r.counters["reflect"]
