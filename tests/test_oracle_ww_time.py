"""Pins of the oracle's time-binned weight windows (CPU, no GPU needed).

The paper's problems are time dependent (a pulse source and a time census, Section 3), so a
window table may depend on time: a particle takes the window of the (cell, time bin) holding its
position and its time.  Pinned here:
* a table whose time bins all hold the same x-varying windows gives, bit for bit, the run of the
  table without time bins (a transposed [t][x] index reads other cells' windows and fails);
* windows that change from one time bin to the next change the splitting and roulette (the time
  lookup is used) and keep every tally unbiased against the analog walk (|z| < 4 per bin).
"""
import os

import numpy as np

import oracle
from paper_2305_07636_gb300 import problems as P

THREADS = min(8, os.cpu_count() or 1)


def _z(ma, sa, mb, sb, rel_max=0.1):
    ma, sa, mb, sb = (np.asarray(a, np.float64).ravel() for a in (ma, sa, mb, sb))
    ok = (sa > 0) & (sb > 0) & (sa < rel_max * np.abs(ma)) & (sb < rel_max * np.abs(mb))
    return (ma[ok] - mb[ok]) / np.sqrt(sa[ok] ** 2 + sb[ok] ** 2)


def test_time_uniform_table_equals_the_untimed_table():
    prob = P.pulse_stack(thickness=8.0, n_layers=4, n_tbins=6)
    t = prob["tallies"][0]["t"]
    plain = P.exponential_ww(prob, decay=0.8)
    timed = P.exponential_ww(prob, decay=0.8, t_edges=t, t_decay=0.0)
    assert len(timed["center"]) == len(t) - 1
    a = oracle.run(prob, 20_000, seed=3, threads=THREADS, ww=plain)
    b = oracle.run(prob, 20_000, seed=3, threads=THREADS, ww=timed)
    assert a.counters == b.counters
    assert a.counters["ww_split"] > 0 and a.counters["ww_kill"] > 0
    for (ma, sa), (mb, sb) in zip(a.tallies, b.tallies):
        assert np.array_equal(ma, mb) and np.array_equal(sa, sb)


def test_time_dependent_windows_are_used_and_stay_unbiased():
    prob = P.pulse_stack(thickness=4.0, n_layers=2, n_tbins=6, ww_bin=0.5)
    t = prob["tallies"][0]["t"]
    flat = oracle.run(prob, 40_000, seed=5, threads=THREADS,
                      ww=P.exponential_ww(prob, decay=0.8, t_edges=t, t_decay=0.0))
    timed = oracle.run(prob, 40_000, seed=5, threads=THREADS,
                       ww=P.exponential_ww(prob, decay=0.8, t_edges=t, t_decay=0.5))
    assert timed.counters["ww_split"] > 2 * flat.counters["ww_split"]
    analog = oracle.run(prob, 400_000, seed=6, threads=THREADS)
    for k in (0, 1):
        mw, sw = timed.tallies[k]
        ma, sa = analog.tallies[k]
        z = _z(mw, sw, ma, sa)
        assert z.size >= (5 if k == 0 else 60), z.size
        assert np.all(np.abs(z) < 4.0), np.abs(z).max()
