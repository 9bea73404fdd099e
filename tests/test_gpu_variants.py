"""CUDA path (through the C ABI) against the CPU oracle and the closed forms for the two Section 3
variants: the time-crossing estimator and implicit capture with a weight-cutoff roulette.

- Replay: in FP64 tracking the GPU reproduces the oracle's event sequence with implicit capture
  (integer fields equal, positions, directions, times and weights within 1e-9 relative).
- Statistics: FP32-tracking tallies agree with the oracle within 4 sigma of the combined error
  (time-crossing tallies of the 7-group pulse, implicit-capture slab / pulse / lattice / AZURV1).
- Closed forms: the time-crossing flux at t = 0 is exactly v0; the 7-group point flux is
  exp(A t) phi(0); beam particles are exactly at x = v t.
- Bit identity: event- and history-based kernels, the batched launch, and the allocation-free entry
  point give the same results as a plain run with these options.
"""
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


def exact_z(mg, sg, exact, rel_max=0.1):
    mg, sg, exact = (np.asarray(a, dtype=np.float64).ravel() for a in (mg, sg, exact))
    ok = (sg > 0) & (sg < rel_max * np.abs(mg))
    return (mg[ok] - exact[ok]) / sg[ok]


def check_z(z, min_bins, bar=4.0):
    assert z.size >= min_bins, f"only {z.size} comparable bins"
    assert np.all(np.abs(z) < bar), f"max |z| = {np.abs(z).max():.2f} over {z.size} bins"


def check_z_many(z, min_bins):
    """Hundreds of bins against a closed form, every |z| < 4, with the GPU error from 256 batches:
    z is then near-Gaussian (with 32 batches it follows Student's t with 31 degrees of freedom,
    whose tail puts one of a few hundred bins beyond 4 now and then).  Neighbouring time bins share
    particles, so their z move together and no check on the spread of z over bins applies."""
    check_z(z, min_bins)


def conserved(c):
    started = c["source"] + c["secondary"] + c["ww_split"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"]
    return started == ended


# ----------------------------------------------------------------------------- time crossing


def test_crossing_pulse_against_oracle_and_expm(torch):
    prob = P.config2_crossing()
    mat, v = prob["materials"][0], prob["speed"]
    pts = np.asarray(prob["tallies"][1]["t"])
    live = pts < prob["t_census"]
    o = oracle.run(prob, 400_000, seed=51, threads=THREADS)
    p = mc.Problem(prob)
    assert mc.tally_shape(p.h, 1) == (1, 1, 1, 7, 101)
    for precision in ("fp32", "fp64"):
        # N divisible by the batch count: equal batches, so the t = 0 value has exactly zero spread
        n = 4_000_000 if precision == "fp32" else 1_024_000
        p.run(n, 52, precision=precision, n_batches=256)
        mg, sg = (a.reshape(7, 101) for a in p.tally(1))
        mo, so = (a.reshape(7, 101) for a in o.tallies[1])
        # every source particle is alive at t = 0 in group 0: exactly v0 there, 0 elsewhere
        assert mg[0, 0] == pytest.approx(v[0], rel=1e-12) and sg[0, 0] == 0.0
        assert np.all(mg[1:, 0] == 0.0) and np.all(mg[:, ~live] == 0.0)
        check_z_many(combined_z(mg, sg, mo, so), 250)
        check_z_many(exact_z(mg[:, live], sg[:, live], CF.multigroup_point_flux(mat, v, pts[live])), 250)
        # the track-length tally of the same run is unchanged by the extra tally
        check_z(combined_z(*p.tally(0), *o.tallies[0]), 200)
        assert conserved(p.counters())
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_crossing_beam_positions(torch, precision):
    """Beam along +x through a pure absorber: at time t a particle sits at x = t exactly, so only
    the 0.1 cm cell that holds x = t may score, with mean e^{-t}."""
    pts = 0.05 + 0.5 * np.arange(10)
    prob = P.slab_problem(5.0, 1.0, 0.0, direction="beam_x", surface_source=True)
    prob = P.with_tallies(prob, [P.mesh(x=np.linspace(0, 5, 51), t=pts, estimator="crossing")])
    p = mc.Problem(prob)
    p.run(2_000_000, 53, precision=precision, n_batches=256)
    m, s = (a.reshape(50, 10) for a in p.tally(0))
    cell = np.floor(pts / 0.1).astype(int)
    mask = np.zeros_like(m, dtype=bool)
    mask[cell, np.arange(10)] = True
    assert np.all(m[~mask] == 0.0)
    check_z(exact_z(m[mask], s[mask], np.exp(-pts)), 10)
    p.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_range_walks_split_runs_across_cells(torch, precision):
    """Both range walks on a mesh of several cells (40 time values over 5 cells: the tallies take
    the range walk).  A beam particle is at x = t, so each time bin [k/8, (k+1)/8) lies in cell
    floor(k/8) with track length e^{-t_k} - e^{-t_k+1}, and each time point t_j in cell floor(t_j)
    with flux e^{-t_j}; every other (cell, time) value is zero (the track tally up to rounding where
    a time edge meets a cell plane)."""
    xe = np.linspace(0, 5, 6)
    te = np.linspace(0, 5, 41)
    pts = 0.0625 + 0.125 * np.arange(40)
    prob = P.slab_problem(5.0, 1.0, 0.0, direction="beam_x", surface_source=True)
    prob = P.with_tallies(prob, [P.mesh(x=xe, t=te), P.mesh(x=xe, t=pts, estimator="crossing")])
    p = mc.Problem(prob)
    p.run(2_000_000, 54, precision=precision, n_batches=256)
    m, s = (a.reshape(5, 40) for a in p.tally(0))
    cell = np.arange(40) // 8
    mask = np.zeros_like(m, dtype=bool)
    mask[cell, np.arange(40)] = True
    assert np.all(np.abs(m[~mask]) < 1e-5 * m[mask].max())
    check_z(exact_z(m[mask], s[mask], np.exp(-te[:-1]) - np.exp(-te[1:])), 40)
    m, s = (a.reshape(5, 40) for a in p.tally(1))
    cell = np.floor(pts).astype(int)
    mask = np.zeros_like(m, dtype=bool)
    mask[cell, np.arange(40)] = True
    assert np.all(m[~mask] == 0.0)
    check_z(exact_z(m[mask], s[mask], np.exp(-pts)), 40)
    p.close()


# ----------------------------------------------------------------------------- implicit capture


def test_implicit_capture_fp64_replay(torch):
    for prob, n in ((P.config1(), 5000), (P.azurv1(t_end=5.0), 1000), (P.config3(), 2000)):
        o = oracle.run(prob, n, seed=61, threads=THREADS, log_first=0, log_count=n, log_cap=400 * n,
                       implicit_capture=True)
        p = mc.Problem(prob)
        p.run(n, 61, precision="fp64", implicit_capture=1, log_first=0, log_count=n,
              log_capacity=400 * n, bank_capacity=1 << 18)
        ev, eo = p.events(400 * n), o.events
        assert len(ev) == len(eo) and len(ev) > n
        assert np.array_equal(ev["tag"], eo["tag"]) and np.array_equal(ev["k"], eo["k"])
        for f in ("kind", "outcome", "n_child", "cell", "elem", "in_pin", "g"):
            assert np.array_equal(ev[f], eo[f]), (prob["name"], f)
        for f in ("x", "y", "z", "ux", "uy", "uz", "t", "w"):
            scale = np.maximum(np.maximum(np.abs(ev[f]), np.abs(eo[f])), 1.0)
            assert np.max(np.abs(ev[f] - eo[f]) / scale) <= 1e-9, (prob["name"], f)
        c = p.counters()
        for k in oracle.COUNTER_NAMES:
            assert c[k] == o.counters[k], (prob["name"], k)
        assert c["capture"] == 0 or prob["name"] == "config3"
        p.close()


@pytest.mark.parametrize("name,n_or,n_gpu,min_bins", [
    ("config1", 400_000, 4_000_000, 45),
    ("config2", 200_000, 2_000_000, 200),
    ("config3", 100_000, 1_000_000, 1000),
    ("azurv1", 40_000, 400_000, 15),
])
def test_implicit_capture_fp32_matches_oracle(torch, name, n_or, n_gpu, min_bins):
    prob = P.azurv1() if name == "azurv1" else P.by_name(name)
    o = oracle.run(prob, n_or, seed=62, threads=THREADS, implicit_capture=True)
    p = mc.Problem(prob)
    # without capture the supercritical population carries more (lighter) particles than analog
    p.run(n_gpu, 63, implicit_capture=1, bank_capacity=1 << 22)
    check_z(combined_z(*p.tally(0), *o.tallies[0]), min_bins)
    c = p.counters()
    assert conserved(c) and c["lost"] == 0
    if name != "config3":  # the lattice's pins have positive non-capture probability too
        assert c["capture"] == 0 and c["ww_kill"] > 0
    p.close()


def test_implicit_capture_closed_forms_and_gain(torch):
    """The 7-group pulse with implicit capture still matches the matrix exponential, and the
    slab's right leakage (config 1's target tally) has a smaller variance per history."""
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    p = mc.Problem(prob)
    p.run(4_000_000, 64, implicit_capture=1, n_batches=256)
    m, s = p.tally(0)
    check_z_many(exact_z(m.reshape(7, -1), s.reshape(7, -1), CF.multigroup_time_bins(mat, v, te)), 300)
    p.close()
    q = mc.Problem(P.config1())
    q.run(4_000_000, 65)
    _, sa = q.leakage()
    q.run(4_000_000, 65, implicit_capture=1)
    _, sb = q.leakage()
    assert sb.ravel()[1] < sa.ravel()[1]
    q.close()


def test_invalid_roulette_parameters_rejected(torch):
    p = mc.Problem(P.config1())
    for kw in ({"wr_cutoff": 0.5, "wr_survival": 0.5}, {"wr_cutoff": -1.0}, {"implicit_capture": 2}):
        with pytest.raises(mc.McError) as e:
            p.run(1000, 1, **{"implicit_capture": 1, **kw})
        assert e.value.code == mc.MC_ERR_INVALID
    p.close()


# ----------------------------------------------------------------------------- bit identity


def test_variants_identical_across_kernels_and_entry_points(torch):
    """With implicit capture and a time-crossing tally: event- and history-based runs, a batched
    launch of two problems and the allocation-free entry point all equal the plain run."""
    prob = P.config2_crossing()
    n = 300_000
    p = mc.Problem(prob)
    ref = None
    for opts in ({"algorithm": "event"}, {"algorithm": "history"}, {"algorithm": "event", "drain_threshold": 1}):
        p.run(n, 71, implicit_capture=1, **opts)
        got = (p.tally_batches(0), p.tally_batches(1), {k: v for k, v in p.counters().items() if k != "iterations"})
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), opts
            assert got[2] == ref[2], opts
    q = mc.Problem(P.azurv1(t_end=5.0))
    o = mc.run_opts(implicit_capture=1, bank_capacity=1 << 14)
    mc.run_batch([p.h, q.h], [n, 50_000], 71, o)
    assert np.array_equal(p.tally_batches(0), ref[0]) and np.array_equal(p.tally_batches(1), ref[1])
    batched_q = q.tally_batches(0)
    q.run(50_000, 72, implicit_capture=1)
    assert np.array_equal(q.tally_batches(0), batched_q)
    # the allocation-free entry point, against mc_run's mean and error of every bin
    n_bins = sum(int(np.prod(mc.tally_shape(p.h, t))) for t in range(len(prob["tallies"]) + 1))
    mean_d = torch.empty(n_bins, dtype=torch.float64, device="cuda")
    err_d = torch.empty(n_bins, dtype=torch.float64, device="cuda")
    mc.run_static(p.h, n, 71, mc.run_opts(implicit_capture=1), mean_d.data_ptr(), err_d.data_ptr(),
                  torch.cuda.current_stream())
    torch.cuda.synchronize()
    p.run(n, 71, implicit_capture=1)
    m0 = np.concatenate([mc.tally_get(p.h, t)[0].ravel() for t in range(len(prob["tallies"]) + 1)])
    e0 = np.concatenate([mc.tally_get(p.h, t)[1].ravel() for t in range(len(prob["tallies"]) + 1)])
    assert np.allclose(mean_d.cpu().numpy(), m0, rtol=1e-9, atol=0.0)
    assert np.allclose(err_d.cpu().numpy(), e0, rtol=1e-9, atol=1e-300)
    p.close()
    q.close()
