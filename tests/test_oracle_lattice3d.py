"""Pins of the oracle's 3D lattice (axial layers of pin elements; the paper's Section 3 lattice
geometry extended in z, toward its 3D C5G7 and Kobayashi duct configurations) on the CPU:

* escape probability of an isotropic point source in a purely absorbing 3D lattice whose layers
  differ, against a ray-marched quadrature that finds materials by point location alone (no
  distances to walls, no stored element indices); the layer order matters at many sigma;
* one layer of finite height gives the same walk as the unbounded 2D lattice;
* exact particle bookkeeping in the axially zoned assembly and the dog-leg duct; the duct carries
  the flux much farther than the shield beside it.
"""
import copy
import math

import numpy as np
import pytest

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import problems as P

THREADS = 8


def balanced(c):
    started = c["source"] + c["secondary"] + c["ww_split"] + c["pc_copies"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"] + c["pc_banked"]
    return started == ended


@pytest.mark.parametrize("point", [(1.3, 1.7, 1.2), (2.1, 1.8, 0.4), (2.1, 0.8, 0.4)])
def test_point_escape_from_3d_lattice(point):
    prob = P.lattice_absorber_3d(point=point)
    n = 400_000
    r = oracle.run(prob, n, seed=81, threads=THREADS)
    p = float(r.leak_mean.sum())
    s = math.sqrt(p * (1 - p) / n)
    exact = CF.lattice_point_escape(prob, 20000, 0.004, 0)
    assert abs(p - exact) < 4 * s, (p, exact, s)
    # the same pins with the layers in the opposite order give a clearly different answer
    w = copy.deepcopy(prob)
    w["lattice"]["pin_material"] = np.asarray(prob["lattice"]["pin_material"]).reshape(3, 9)[::-1].ravel().tolist()
    assert abs(CF.lattice_point_escape(w, 20000, 0.004, 0) - exact) > 10 * s
    c = r.counters
    assert c["lost"] == 0 and c["capture"] + c["leak"] == c["source"]


def test_ray_marched_escape_converges():
    prob = P.lattice_absorber_3d()
    a = CF.lattice_point_escape(prob, 20000, 0.004, 0)
    b = CF.lattice_point_escape(prob, 40000, 0.002, 1)
    assert abs(a - b) < 2e-5


def test_one_layer_equals_the_2d_lattice():
    prob = P.lattice_absorber_3d()
    one = copy.deepcopy(prob)
    one["lattice"].update(nz=1, pitch_z=3.0, pin_material=prob["lattice"]["pin_material"][9:18])
    flat = copy.deepcopy(one)
    flat["lattice"].update(nz=0)
    a = oracle.run(one, 20000, seed=82, threads=THREADS, log_first=0, log_count=200, log_cap=20000)
    b = oracle.run(flat, 20000, seed=82, threads=THREADS, log_first=0, log_count=200, log_cap=20000)
    assert np.array_equal(a.events, b.events) and a.counters == b.counters
    assert np.array_equal(a.leak_mean, b.leak_mean)


def test_axial_lattice_bookkeeping_and_layers():
    prob = P.axial_lattice()
    r = oracle.run(prob, 20000, seed=83, threads=THREADS, log_first=0, log_count=2000, log_cap=400000)
    c = r.counters
    assert balanced(c) and c["lost"] == 0 and c["leak"] > 0 and c["secondary"] > 0
    ev = r.events
    lat = prob["lattice"]
    per_layer = lat["nx"] * lat["ny"]
    walls = ev[(ev["kind"] == 1) & (ev["outcome"] == 3)]
    layers = walls["elem"] // per_layer
    assert layers.min() == 0 and layers.max() == lat["nz"] - 1  # every layer reached
    # the walk never reports an element outside the lattice
    assert ev["elem"].max() < per_layer * lat["nz"]
    # flux per layer: the rodded top fuel layers see less than the middle ones
    m, _ = r.tallies[0]
    layer_flux = np.asarray(m).reshape(lat["nz"], -1).sum(axis=1)
    assert layer_flux[2] > layer_flux[4]


def test_dogleg_duct_streaming():
    prob = P.dogleg_duct()
    r = oracle.run(prob, 40000, seed=84, threads=THREADS)
    c = r.counters
    assert balanced(c) and c["lost"] == 0 and c["reflect"] > 0
    m, _ = r.tallies[0]
    m = np.asarray(m).reshape(2, 10, 4, 2, -1).sum(axis=(3, 4))  # [z][y][x]
    # along the second leg (x cell 2, z < w) vs the shield beside it (x cell 0) at y in 24-32 cm
    assert m[0, 6:8, 2].sum() > 5 * m[0, 6:8, 0].sum()
