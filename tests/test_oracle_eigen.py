"""Pins of the oracle's k-eigenvalue power iteration (the paper's C5G7 runs, Section 3) against
closed forms, on the CPU:

* one-group infinite medium: k = nu Sigma_f / (Sigma_t - Sigma_s), and every history's track length
  is 1 / Sigma_a whatever happens at its production event;
* seven-group infinite medium: k = the dominant eigenvalue of A^-1 F (A = diag(Sigma_t) - S^T,
  F = chi (nu Sigma_f)^T), and the active cycles' group flux has the shape of its eigenvector;
* the bank of fission sites keeps the population: about N k / k_prev sites per cycle;
* a symmetric pin cell has a symmetric flux (no closed form for its k);
* the result does not depend on the oracle's thread count (sites ordered by history, k summed in
  fixed point).
Statistics over the active cycles (each active cycle one batch), |z| < 4.
"""
import math

import numpy as np

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import problems as P

THREADS = 8


def test_eigen_one_group_closed_forms():
    prob = P.eigen_infinite_1g()
    r = oracle.run_eigen(prob, 20000, 5, 40, seed=41, threads=THREADS)
    k_exact = 2.4 * 0.2 / (1.0 - 0.5)
    assert abs(r.k_mean - k_exact) < 4 * r.k_std
    m, s = r.tallies[0]
    assert abs(m.ravel()[0] - 2.0) < 4 * s.ravel()[0]  # track length per history = 1 / Sigma_a
    # each cycle banks about N k / k_prev sites
    kprev = np.concatenate([[1.0], r.k_cycle[:-1]])
    ratio = r.sites_cycle / (20000 * r.k_cycle / kprev)
    assert np.all(np.abs(ratio - 1.0) < 0.05)
    assert r.counters["capture"] + r.counters["production"] == r.counters["source"]


def test_eigen_multigroup_k_and_spectrum():
    prob = P.eigen_infinite_mg()
    k_exact, phi = CF.infinite_k(prob["materials"][0])
    r = oracle.run_eigen(prob, 20000, 10, 40, seed=42, threads=THREADS)
    assert abs(r.k_mean - k_exact) < 4 * r.k_std, (r.k_mean, r.k_std, k_exact)
    spec = r.cycle_tallies[:, :7]
    spec = spec / spec.sum(axis=1, keepdims=True)  # each active cycle's normalised group flux
    mean, err = spec.mean(axis=0), spec.std(axis=0, ddof=1) / math.sqrt(spec.shape[0])
    z = (mean - phi) / err
    assert np.all(np.abs(z) < 4), z


def test_eigen_pin_cell_is_symmetric():
    """The pin cell is symmetric under x <-> y and under x -> pitch - x: so is its group flux."""
    prob = P.pin_cell()
    r = oracle.run_eigen(prob, 20000, 10, 30, seed=43, threads=THREADS)
    m, s = r.tallies[0]
    m, s = m.reshape(4, 4, 7), s.reshape(4, 4, 7)  # [y][x][g]
    for a, b, sa, sb in ((m, m.transpose(1, 0, 2), s, s.transpose(1, 0, 2)),
                         (m, m[:, ::-1], s, s[:, ::-1])):
        ok = sa > 0
        z = (a[ok] - b[ok]) / np.sqrt(sa[ok] ** 2 + sb[ok] ** 2)
        assert np.all(np.abs(z) < 4)
    assert 0.8 < r.k_mean < 1.5 and r.counters["lost"] == 0


def test_eigen_independent_of_thread_count():
    prob = P.pin_cell()
    a = oracle.run_eigen(prob, 5000, 3, 5, seed=44, threads=1)
    b = oracle.run_eigen(prob, 5000, 3, 5, seed=44, threads=7)
    assert np.array_equal(a.k_cycle, b.k_cycle)
    assert np.array_equal(a.sites_cycle, b.sites_cycle)
    assert a.counters == b.counters


def test_eigen_cycle_spread_falls_as_inverse_sqrt_n():
    """Each cycle starts N independent histories at the fission sites (systematic sampling of the
    whole bank), so the cycle-to-cycle spread of k falls as N^-1/2: 16 times the histories, a
    quarter of the spread (started from one site the spread would not fall at all)."""
    prob = P.eigen_infinite_mg()
    small = oracle.run_eigen(prob, 1000, 5, 60, seed=45, threads=THREADS)
    large = oracle.run_eigen(prob, 16000, 5, 60, seed=46, threads=THREADS)
    ratio = large.k_cycle[5:].std(ddof=1) / small.k_cycle[5:].std(ddof=1)
    assert 0.15 < ratio < 0.4, ratio
