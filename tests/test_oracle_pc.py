"""Pins of the oracle's population control at census times (splitting-roulette per independent
batch; the paper's Section 3 feature list) against closed forms, on the CPU:

* supercritical AZURV1 (c = 1.1): the flux time bins keep the closed form e^{0.1 t} while the
  population is brought back to N at every census: each census banks N e^{0.1 dt} particles;
* subcritical one-group medium: the same with decay, N e^{-0.4 dt} per census;
* the 7-group pulse (config 2) with census times inside its time range: the matrix exponential;
* exact particle bookkeeping; results independent of the thread count (batches are independent).
Combing (method "comb"): the copy counts equal the teeth (k + xi) W / N_b counted exactly in rational
arithmetic over the fixed-point weights; every census restores exactly N_b particles per batch; the
same closed forms hold.
|z| < 4 against the closed forms, errors over the independent batches.
"""
import math
from fractions import Fraction

import numpy as np

import oracle
from oracle import closed_forms as CF
from paper_2305_07636_gb300 import problems as P

THREADS = 8


def zscores(mean, std, exact, rel_max=0.1):
    mean, std, exact = (np.asarray(a, dtype=np.float64).ravel() for a in (mean, std, exact))
    ok = (std > 0) & (std < rel_max * np.abs(mean))
    return (mean[ok] - exact[ok]) / std[ok]


def balanced(c):
    started = c["source"] + c["secondary"] + c["ww_split"] + c["pc_copies"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"] + c["pc_banked"]
    return started == ended


def test_pc_azurv1_growth_and_flux():
    prob = P.azurv1()
    ct = np.arange(2.0, 20.0, 2.0)
    r = oracle.run_pc(prob, 40000, ct, 32, seed=51, threads=THREADS)
    m, s = r.tallies[0]
    z = zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, prob["tallies"][0]["t"]))
    assert z.size >= 15 and np.all(np.abs(z) < 4), z
    assert np.all(np.abs(r.banked / 40000 / math.exp(0.2) - 1) < 0.03), r.banked
    assert balanced(r.counters) and r.counters["pc_copies"] > 0


def test_pc_subcritical_decay():
    te = np.linspace(0, 6, 13)
    prob = P.infinite_medium_1g(1.0, 0.6, speed=1.0, t_edges=te, t_census=6.0)
    r = oracle.run_pc(prob, 40000, [2.0, 4.0], 32, seed=52, threads=THREADS)
    m, s = r.tallies[0]
    z = zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.0, 1.0, te))
    assert z.size >= 10 and np.all(np.abs(z) < 4), z
    assert np.all(np.abs(r.banked / 40000 / math.exp(-0.8) - 1) < 0.04), r.banked
    assert balanced(r.counters)


def test_pc_multigroup_pulse_expm():
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    r = oracle.run_pc(prob, 100000, [1e-8, 1e-7, 1e-6, 1e-5, 1e-4], 32, seed=53, threads=THREADS)
    m, s = r.tallies[0]
    z = zscores(m.reshape(7, -1), s.reshape(7, -1), CF.multigroup_time_bins(mat, v, te))
    assert z.size >= 250 and np.all(np.abs(z) < 4), np.abs(z).max()
    assert balanced(r.counters)


def test_pc_independent_of_thread_count():
    prob = P.azurv1(t_end=6.0, n_tbins=6)
    a = oracle.run_pc(prob, 4000, [2.0, 4.0], 8, seed=54, threads=1)
    b = oracle.run_pc(prob, 4000, [2.0, 4.0], 8, seed=54, threads=5)
    assert np.array_equal(a.batch_tallies, b.batch_tallies)
    assert a.counters == b.counters and np.array_equal(a.banked, b.banked)


def exact_teeth(w, n_teeth, xi):
    """Teeth (k + xi) W / N, k = 0 .. N-1, attributed to the weight intervals [C_{j-1}, C_j) of the
    fixed-point weights, in exact rational arithmetic."""
    q = [int(np.rint(x * 2**40)) for x in w]
    W = sum(q)
    C = np.cumsum([0] + q)
    out = np.zeros(len(w), np.int64)
    for k in range(n_teeth):
        pos = (Fraction(k) + Fraction(xi)) * W / n_teeth
        j = int(np.searchsorted(C, pos, side="right")) - 1
        out[min(j, len(w) - 1)] += 1
    return out


def test_comb_counts_are_the_exact_teeth():
    rng = np.random.default_rng(11)
    cases = [([1.0], 5, 0.5), ([0.5] * 8, 8, 1e-9), ([0.5] * 8, 8, 1 - 1e-9), ([1e-6, 1.0, 1e-6], 3, 0.3),
             ([2.0, 0.0, 1.0], 4, 0.75)]
    for _ in range(300):
        n = int(rng.integers(1, 40))
        cases.append((rng.exponential(1.0, n) * float(rng.choice([1e-3, 1.0, 50.0])), int(rng.integers(1, 60)),
                      float(rng.uniform())))
    for w, nt, xi in cases:
        got = oracle.comb_counts(w, nt, xi)
        assert got.sum() == nt and np.all(got >= 0)
        assert np.array_equal(got, exact_teeth(w, nt, xi)), (w, nt, xi)


def test_pc_comb_azurv1_growth_and_flux():
    prob = P.azurv1()
    ct = np.arange(2.0, 20.0, 2.0)
    n = 40000
    r = oracle.run_pc(prob, n, ct, 32, seed=55, threads=THREADS, method="comb")
    m, s = r.tallies[0]
    z = zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, prob["tallies"][0]["t"]))
    assert z.size >= 15 and np.all(np.abs(z) < 4), z
    assert np.all(np.abs(r.banked / n / math.exp(0.2) - 1) < 0.03), r.banked
    # the comb restores exactly N_b per batch at every census
    assert r.counters["pc_copies"] == len(ct) * n
    assert balanced(r.counters)


def test_pc_comb_multigroup_pulse_expm():
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    ct = [1e-8, 1e-7, 1e-6, 1e-5, 1e-4]
    r = oracle.run_pc(prob, 100000, ct, 32, seed=56, threads=THREADS, method="comb")
    m, s = r.tallies[0]
    z = zscores(m.reshape(7, -1), s.reshape(7, -1), CF.multigroup_time_bins(mat, v, te))
    assert z.size >= 250 and np.all(np.abs(z) < 4), np.abs(z).max()
    assert balanced(r.counters)


def test_pc_comb_subcritical_and_thread_independent():
    te = np.linspace(0, 6, 13)
    prob = P.infinite_medium_1g(1.0, 0.6, speed=1.0, t_edges=te, t_census=6.0)
    r = oracle.run_pc(prob, 40000, [2.0, 4.0], 32, seed=57, threads=THREADS, method="comb")
    m, s = r.tallies[0]
    z = zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.0, 1.0, te))
    assert z.size >= 10 and np.all(np.abs(z) < 4), z
    assert r.counters["pc_copies"] == 2 * 40000
    a = oracle.run_pc(P.azurv1(t_end=6.0, n_tbins=6), 4000, [2.0, 4.0], 8, seed=58, threads=1, method="comb")
    b = oracle.run_pc(P.azurv1(t_end=6.0, n_tbins=6), 4000, [2.0, 4.0], 8, seed=58, threads=5, method="comb")
    assert np.array_equal(a.batch_tallies, b.batch_tallies) and a.counters == b.counters
