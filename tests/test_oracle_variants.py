"""Pins of the oracle's two Section 3 variants against closed forms (CPU, no GPU needed):

* the time-crossing estimator (the flux at time points, which the paper uses for its multigroup
  pulse and its C5G7 transients): a one-group infinite medium, phi(t) = v e^{-alpha t}; the
  7-group pulse, phi(t) = exp(A t) phi(0); a beam in a pure absorber, whose particles are at
  x = v t exactly, so every mesh cell but one must stay empty at each time point;
* implicit capture with a weight-cutoff roulette (the paper's Kobayashi transient): the same
  closed forms as the analog walk (P3 track length 1/Sigma_a and time bins, the AZURV1 growth with
  production, the 7-group expm), unbiasedness against analog, exact particle bookkeeping.

Statistical checks: |z| < 4 per bin with sigma from the oracle's exact per-history variance,
bins above 10% relative error excluded.
"""
import math
import os

import numpy as np

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import problems as P

THREADS = min(8, os.cpu_count() or 1)


def zscores(mean, std, exact, rel_max=0.1):
    mean, std, exact = (np.asarray(a, dtype=np.float64).ravel() for a in (mean, std, exact))
    ok = (std > 0) & (std < rel_max * np.abs(mean))
    return (mean[ok] - exact[ok]) / std[ok]


def assert_z(z, bar=4.0, min_bins=1):
    assert z.size >= min_bins, f"only {z.size} bins well sampled"
    assert np.all(np.abs(z) < bar), f"max |z| = {np.abs(z).max():.2f}"


# ----------------------------------------------------------------------------- time crossing


def test_crossing_one_group_point_flux():
    sa, v = 0.4, 2.0
    pts = np.linspace(0.0, 5.0, 11)
    prob = P.infinite_medium_1g(1.0, 1.0 - sa, speed=v)
    prob = P.with_tallies(prob, [P.mesh(x=(0, 10), y=(0, 10), z=(0, 10), t=pts, estimator="crossing")])
    r = oracle.run(prob, 200000, seed=21, threads=THREADS)
    m, s = r.tallies[0]
    assert m.shape == (1, 1, 1, 1, 11)
    # every source particle is alive at t = 0: the estimate there is exactly v
    assert m.ravel()[0] == v and s.ravel()[0] == 0.0
    assert_z(zscores(m, s, CF.infinite_point_flux(1.0, 1.0 - sa, 0.0, v, pts)), min_bins=9)


def test_crossing_multigroup_pulse_expm():
    prob = P.config2_crossing()
    mat, v = prob["materials"][0], prob["speed"]
    pts = np.asarray(prob["tallies"][1]["t"])
    live = pts < prob["t_census"]  # the census ends every particle: a point at t_census scores 0
    exact = CF.multigroup_point_flux(mat, v, pts[live])
    eig = CF.multigroup_point_flux(mat, v, pts[live], method="eig")
    big = np.abs(exact) > 1e-6 * np.abs(exact).max()
    assert np.allclose(eig[big], exact[big], rtol=1e-6)
    r = oracle.run(prob, 400000, seed=22, threads=THREADS)
    m, s = r.tallies[1]
    m, s = m.reshape(7, -1), s.reshape(7, -1)
    assert m.shape == (7, 101)
    assert m[0, 0] == v[0] and np.all(m[1:, 0] == 0.0)
    assert np.all(m[:, ~live] == 0.0)
    assert_z(zscores(m[:, live], s[:, live], exact), min_bins=250)
    # the track-length tally of the same run integrates the same flux: sum of bins = int phi dt
    tl, _ = r.tallies[0]
    assert tl.shape == (1, 1, 1, 7, 100)


def test_crossing_beam_positions():
    """Beam along +x at t = 0 in a pure absorber (Sigma_t = 1, v = 1): at time t a particle is at
    x = t exactly, alive with probability e^{-t}; the flux at t lies in the one 0.1 cm cell that
    holds x = t, every other cell is exactly zero."""
    pts = 0.05 + 0.5 * np.arange(10)  # points away from the cell edges
    prob = P.slab_problem(5.0, 1.0, 0.0, direction="beam_x", surface_source=True)
    prob = P.with_tallies(prob, [P.mesh(x=np.linspace(0, 5, 51), t=pts, estimator="crossing")])
    r = oracle.run(prob, 200000, seed=23, threads=THREADS)
    m, s = r.tallies[0]
    m, s = m.reshape(50, 10), s.reshape(50, 10)
    cell = np.floor(pts / 0.1).astype(int)
    mask = np.zeros_like(m, dtype=bool)
    mask[cell, np.arange(10)] = True
    assert np.all(m[~mask] == 0.0)
    assert_z(zscores(m[mask], s[mask], np.exp(-pts)), min_bins=10)


def test_crossing_fixed_point_counts_weight():
    """The int64 sums of a time-crossing tally count the weight (the flux is w v), so that fast
    groups do not leave the fixed-point range: fixed / 2^32 = sum of w = s1 / v."""
    v = 2e9
    prob = P.infinite_medium_1g(1.0, 0.5, speed=v)
    prob = P.with_tallies(prob, [P.mesh(x=(0, 10), y=(0, 10), z=(0, 10), t=[0.0, 1e-10, 1e-9],
                                        estimator="crossing")])
    r = oracle.run(prob, 20000, seed=24, threads=THREADS)
    assert np.allclose(r.fixed[:3] / 2.0**32, r.s1[:3] / v, rtol=1e-12)


# ----------------------------------------------------------------------------- implicit capture


def test_implicit_capture_one_group_closed_forms():
    sa = 0.4
    te = np.linspace(0, 5, 11)
    prob = P.infinite_medium_1g(1.0, 1.0 - sa, speed=2.0, t_edges=te)
    r = oracle.run(prob, 200000, seed=31, threads=THREADS, implicit_capture=True)
    m, s = r.tallies[0]
    assert_z(zscores(m, s, CF.infinite_time_bins(1.0, 1.0 - sa, 0.0, 2.0, te)), min_bins=8)
    c = r.counters
    assert c["capture"] == 0 and c["ww_kill"] == c["source"]  # only the roulette ends histories
    prob = P.infinite_medium_1g(1.0, 1.0 - sa)
    r = oracle.run(prob, 200000, seed=32, threads=THREADS, implicit_capture=True)
    m, s = r.tallies[0]
    assert abs(m.sum() - CF.infinite_total_tracklength(1.0, 1.0 - sa)) < 4 * s.sum()


def test_implicit_capture_azurv1_with_production():
    """c = 1.1 with production: each collision keeps (Ss + Sf)/St = 0.8 of the weight and gives
    it to the scattered particle or to floor(nu + xi) children; flux bins follow e^{0.1 t}, and
    the time-crossing flux at t = 20 is e^2."""
    prob = P.azurv1()
    te = prob["tallies"][0]["t"]
    pts = np.array([5.0, 10.0, 19.5])
    prob = P.with_tallies(prob, prob["tallies"] + [P.mesh(x=(0, 10), y=(0, 10), z=(0, 10), t=pts,
                                                          estimator="crossing")])
    r = oracle.run(prob, 40000, seed=33, threads=THREADS, implicit_capture=True)
    m, s = r.tallies[0]
    assert_z(zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, te)), min_bins=15)
    m, s = r.tallies[1]
    assert_z(zscores(m, s, CF.infinite_point_flux(1.0, 0.6, 0.5, 1.0, pts)), min_bins=3)
    assert r.counters["capture"] == 0 and r.counters["production"] > 0


def test_implicit_capture_multigroup_expm():
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    exact = CF.multigroup_time_bins(mat, v, te)
    r = oracle.run(prob, 300000, seed=34, threads=THREADS, implicit_capture=True)
    m, s = r.tallies[0]
    assert_z(zscores(m.reshape(7, -1), s.reshape(7, -1), exact), min_bins=250)


def test_implicit_capture_unbiased_and_conserving():
    """Slab with scattering (no closed form): implicit capture and analog agree; every particle
    started ends exactly once (roulette kills counted as ww_kill); no collision captures."""
    prob = P.config1()
    a = oracle.run(prob, 200000, seed=35, threads=THREADS)
    b = oracle.run(prob, 200000, seed=36, threads=THREADS, implicit_capture=True)
    for (ma, sa), (mb, sb) in [(a.tallies[0], b.tallies[0]), ((a.leak_mean, a.leak_std), (b.leak_mean, b.leak_std))]:
        ok = (sa > 0) & (sb > 0) & (sa < 0.1 * np.abs(ma))
        z = (ma[ok] - mb[ok]) / np.sqrt(sa[ok] ** 2 + sb[ok] ** 2)
        assert z.size > 0 and np.all(np.abs(z) < 4), np.abs(z).max()
    c = b.counters
    started = c["source"] + c["secondary"] + c["ww_split"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"]
    assert started == ended and c["capture"] == 0
    assert c["collision"] == c["scatter"] + c["capture"] + c["production"]
    # the leakage estimate gains: its variance per history drops below the analog one
    assert b.leak_std[1] < a.leak_std[1]


def test_implicit_capture_pure_absorber_is_analog():
    """With Sigma_s = Sigma_f = 0 the non-capture probability is 0: the collision captures, as in
    the analog walk, and the beam transmission is e^{-Sigma_t L}."""
    prob = P.slab_problem(5.0, 1.0, 0.0, direction="beam_x", surface_source=True)
    a = oracle.run(prob, 100000, seed=37, threads=THREADS)
    b = oracle.run(prob, 100000, seed=37, threads=THREADS, implicit_capture=True)
    assert np.array_equal(a.s1, b.s1) and a.counters == b.counters
    assert abs(b.leak_mean[1] - math.exp(-5.0)) < 4 * b.leak_std[1]
