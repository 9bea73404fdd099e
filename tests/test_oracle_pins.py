"""Pins of the CPU oracle against things other than itself: closed forms, a library Philox,
exact counting identities and brute-force sampling checks.  No GPU needed.

Statistical checks use z = (oracle - exact) / sigma with sigma from the oracle's exact
per-history variance; bins whose relative error exceeds 10% are excluded (their sigma estimate
is itself unreliable), and the bar is |z| < 4 per bin (the 4-sigma rule of the method's parity).
"""
import math
import os

import numpy as np
import pytest

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


# ----------------------------------------------------------------------------- RNG


def test_philox_matches_triton_reference():
    """The oracle's Philox4x32-10 equals Triton's library implementation (run by its CPU
    interpreter) bit for bit, on random keys and full 128-bit counters."""
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    tl = pytest.importorskip("triton.language")
    torch = pytest.importorskip("torch")

    @triton.jit
    def kern(out, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                               tl.load(c3p + i), 10)
        tl.store(out + 4 * i, a)
        tl.store(out + 4 * i + 1, b)
        tl.store(out + 4 * i + 2, c)
        tl.store(out + 4 * i + 3, d)

    rng = np.random.default_rng(123)
    N = 16
    for _ in range(4):
        seed = int(rng.integers(0, 2**63))
        ctr = rng.integers(0, 2**32, size=(4, N), dtype=np.uint64)
        cts = [torch.tensor(ctr[i].astype(np.uint32).view(np.int32)).view(torch.uint32)
               for i in range(4)]
        out = torch.zeros(4 * N, dtype=torch.uint32)
        kern[(1,)](out, seed, *cts, N=N)
        ref = out.view(torch.int32).numpy().view(np.uint32).reshape(N, 4)
        for j in range(N):
            mine = oracle.philox((seed & 0xFFFFFFFF, seed >> 32), [int(c) for c in ctr[:, j]])
            assert mine == [int(v) for v in ref[j]]


def test_u01_open_interval_and_resolution():
    assert oracle.u01(0, 0) == 0.5 * 2.0**-52
    assert 0.0 < oracle.u01(0, 0) < oracle.u01(0, 64)
    top = oracle.u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and top == 1.0 - 0.5 * 2.0**-52
    # the 52 bits come from the top 26 bits of each word
    assert oracle.u01(1 << 31, 0) == 0.5 + 0.5 * 2.0**-52
    assert oracle.u01(0, 1 << 6) == 1.5 * 2.0**-52
    assert oracle.u01(0, (1 << 6) - 1) == oracle.u01(0, 0)


def test_source_positions_uniform_chi2():
    """Box source positions: chi-square of a 10x10 histogram over (x, y) is consistent with
    uniform (p > 1e-3)."""
    from scipy import stats
    prob = P.config2()
    n = 20000
    xs = np.array([oracle.source_sample(prob, 7, h)[0][:2] for h in range(n)])
    H, _, _ = np.histogram2d(xs[:, 0], xs[:, 1], bins=10, range=[[0, 10], [0, 10]])
    chi2 = ((H - n / 100) ** 2 / (n / 100)).sum()
    assert stats.chi2.sf(chi2, 99) > 1e-3


def test_direction_distributions():
    """Isotropic source: E[mu] = 0, E[mu^2] = 1/3, |u| = 1.  Cosine (isotropic-flux) surface
    source: E[mu] = 2/3, E[mu^2] = 1/2."""
    n = 20000
    iso = np.array([oracle.source_sample(P.config2(), 3, h)[0][3:6] for h in range(n)])
    assert np.allclose(np.linalg.norm(iso, axis=1), 1.0, atol=1e-12)
    for d in range(3):
        assert abs(iso[:, d].mean()) < 4 * math.sqrt(1 / 3 / n)
        assert abs((iso[:, d] ** 2).mean() - 1 / 3) < 4 * math.sqrt(4 / 45 / n)
    cos = np.array([oracle.source_sample(P.config4(), 3, h)[0][3] for h in range(n)])
    assert abs(cos.mean() - 2 / 3) < 4 * math.sqrt((0.5 - 4 / 9) / n)
    assert abs((cos ** 2).mean() - 0.5) < 4 * math.sqrt((1 / 3 - 1 / 4) / n)


def test_scatter_group_cdf_exact_on_uniform_grid():
    """Sampling g' with u on a fine uniform grid reproduces Sigma_s[g->.]/Sigma_s_tot exactly
    up to the grid resolution (brute force over all u)."""
    prob = P.config2()
    S = np.asarray(prob["materials"][0]["sigma_s"])
    n = 20000
    us = (np.arange(n) + 0.5) / n
    for g in range(prob["G"]):
        counts = np.bincount([oracle.sample_scatter_group(prob, 0, g, u) for u in us],
                             minlength=prob["G"])
        assert np.allclose(counts / n, S[g] / S[g].sum(), atol=1.5 / n)


def test_child_tags_distinct_and_lineage_only():
    tags = {oracle.child_tag(5, p, k, j) for p in range(200) for k in range(20) for j in range(5)}
    assert len(tags) == 200 * 20 * 5
    assert oracle.child_tag(5, 17, 3, 1) == oracle.child_tag(5, 17, 3, 1)
    assert oracle.child_tag(5, 17, 3, 1) != oracle.child_tag(6, 17, 3, 1)


# ----------------------------------------------------------------------------- geometry


def test_plane_distance_cases():
    assert oracle.dist_plane(1.0, 0.5, 3.0, -1) == 4.0      # x < 3, moving +x
    assert math.isinf(oracle.dist_plane(1.0, -0.5, 3.0, -1))  # moving away
    assert oracle.dist_plane(5.0, -1.0, 3.0, +1) == 2.0     # x >= 3, moving -x
    assert oracle.dist_plane(3.0 + 1e-15, 1.0, 3.0, -1) == 0.0  # overshoot clamps to 0
    assert math.isinf(oracle.dist_plane(2.0, 0.0, 3.0, -1))


def test_cylinder_distance_cases():
    d = oracle.dist_cylinder
    assert d(-2.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0) == pytest.approx(1.0, abs=1e-15)
    assert d(0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1) == pytest.approx(1.0, abs=1e-15)
    assert d(-1.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1) == pytest.approx(2.0, abs=1e-15)
    assert math.isinf(d(2.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0))     # outside, moving away
    assert math.isinf(d(-2.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0))    # grazing: tangent line
    assert math.isinf(d(-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0))    # parallel to the axis
    # oblique chord: from (-2, 0.6) along +x hits x = -0.8
    assert d(-2.0, 0.6, 1.0, 0.0, 0.0, 0.0, 1.0, 0) == pytest.approx(1.2, abs=1e-14)
    # grazing lines, on a cylinder small enough that the discriminant is resolved: a chord of
    # 5e-13 cm (below 1e-12) is not entered, a chord of 1e-11 cm is
    r = 1e-6
    y = math.sqrt(r * r - 6.25e-26)
    assert math.isinf(d(-1.5e-6, y, 1.0, 0.0, 0.0, 0.0, r, 0))
    y = math.sqrt(r * r - 2.5e-23)
    assert d(-1.5e-6, y, 1.0, 0.0, 0.0, 0.0, r, 0) == pytest.approx(1.5e-6 - 5e-12, abs=1e-16)
    # a 3D direction with a z component: distance scales by 1/sqrt(ux^2+uy^2) of the xy speed
    s = 0.6
    assert d(-2.0, 0.0, s, 0.0, 0.0, 0.0, 1.0, 0) == pytest.approx(1.0 / s, abs=1e-14)


def test_cell_after_a_crossing_next_to_a_wall():
    """Four cells of a square cut by interior planes x = L/2 and y = L/2 (surfaces 1 and 4;
    cells 0: x<h y<h, 1: x>h y<h, 2: x<h y>h, 3: x>h y>h), reflecting walls y = 0 and y = L
    (3 and 5).  After crossing x = L/2: a point exactly on y = L/2 (the corner) goes to the side
    the particle is moving into, the + side when it moves along the plane; a point rounded to
    just outside the wall y = 0 is put in the cell beyond the crossed plane, within 1e-12 of the
    terms' size; farther out it is lost; away from a crossing no tolerance applies."""
    prob = P.config5(seed=5, n_problems=3)[0][1]  # the 2D slab kind
    assert prob["name"].endswith("slab2d")
    L = prob["surfaces"][2]["coef"][0]
    h = L / 2
    fc = oracle.find_cell
    assert fc(prob, h, 1e-3, 0.0, 1, +1, (0.6, 0.8, 0.0)) == 1   # plainly in the lower right cell
    assert fc(prob, h, h - 1e-13, 0.0, 1, +1, (0.6, 0.8, 0.0)) == 1
    assert fc(prob, h, h + 1e-13, 0.0, 1, +1, (0.6, -0.8, 0.0)) == 3
    # exactly at the corner: the direction decides (this is what ends the back-and-forth of a
    # particle sitting on the corner between cells 1 and 2 and heading into cell 0)
    assert fc(prob, h, h, 0.0, 1, -1, (-0.3, -0.9, 0.3)) == 0
    assert fc(prob, h, h, 0.0, 1, -1, (-0.3, 0.9, 0.3)) == 2
    assert fc(prob, h, h, 0.0, 4, -1, (-0.3, -0.9, 0.3)) == 0     # the same corner via y = h
    assert fc(prob, h, h, 0.0, 4, -1, (0.3, -0.9, 0.3)) == 1
    assert fc(prob, h, h, 0.0, 1, +1, (0.6, 0.0, 0.8)) == 3       # along y = h: the + side
    assert fc(prob, h, -1e-13, 0.0, 1, +1, (0.6, -0.8, 0.0)) == 1  # rounded past the wall y = 0
    assert fc(prob, h, L + 1e-13, 0.0, 1, -1, (-0.6, 0.8, 0.0)) == 2  # past y = L, towards -x
    assert fc(prob, h, -1e-9, 0.0, 1, +1, (0.6, -0.8, 0.0)) == -1   # beyond rounding: lost
    assert fc(prob, 1.0, -1e-13, 0.0) == -1                  # not a crossing: exact test only
    assert fc(prob, 1.0, 1e-13, 0.0) == 0
    assert fc(prob, h, h, 0.0) == 3                          # not a crossing: the + sides


# ----------------------------------------------------------------------------- transport closed forms


def test_P1_beam_transmission():
    prob = P.slab_problem(5.0, 1.0, 0.0, direction="beam_x", surface_source=True)
    r = oracle.run(prob, 400000, seed=11, threads=THREADS)
    exact = CF.beam_transmission(1.0, 5.0)
    assert abs(r.leak_mean[1] - exact) < 4 * r.leak_std[1]
    assert r.leak_mean[0] == 0.0
    m, s = r.tallies[0]
    assert_z(zscores(m, s, CF.beam_flux_bins(1.0, np.linspace(0, 5, 51))), min_bins=40)


def test_P2_slab_isotropic_source_En():
    prob = P.config1(sigma_s=0.0)
    r = oracle.run(prob, 2_000_000, seed=12, threads=THREADS)
    pl, pr = CF.slab_leakage(1.0, 5.0, 1.0)
    assert abs(r.leak_mean[0] - pl) < 4 * r.leak_std[0]
    assert abs(r.leak_mean[1] - pr) < 4 * r.leak_std[1]
    m, s = r.tallies[0]
    exact = CF.slab_flux_bins(1.0, np.linspace(0, 5, 51))
    assert np.allclose(exact, CF.slab_flux_bins_quad(1.0, np.linspace(0, 5, 51)), rtol=1e-9)
    z = zscores(m, s, exact)
    assert_z(z, min_bins=45)
    assert 0.6 < np.mean(z**2) < 1.6


def test_P3_infinite_medium_steady_and_time():
    sa = 0.4
    prob = P.infinite_medium_1g(1.0, 1.0 - sa, speed=2.0, t_edges=np.linspace(0, 5, 11))
    r = oracle.run(prob, 300000, seed=13, threads=THREADS)
    m, s = r.tallies[0]
    exact = CF.infinite_time_bins(1.0, 1.0 - sa, 0.0, 2.0, np.linspace(0, 5, 11))
    assert_z(zscores(m, s, exact), min_bins=8)
    prob = P.infinite_medium_1g(1.0, 1.0 - sa)
    r = oracle.run(prob, 300000, seed=14, threads=THREADS)
    m, s = r.tallies[0]
    assert abs(m.sum() - 1 / sa) < 4 * s.sum()
    assert abs(m.sum() - CF.infinite_total_tracklength(1.0, 1.0 - sa)) < 4 * s.sum()


def test_P4_azurv1_population_growth():
    """Supercritical c = 1.1: the population after 20 mean-free-times is e^2 = 7.389 times the
    initial one (paper Section 3); flux time bins follow e^{0.1 t}.  Uncertainty of the census
    count from 8 seed replicates, as the paper does for its transient."""
    prob = P.azurv1()
    pops = []
    for seed in range(8):
        r = oracle.run(prob, 20000, seed=100 + seed, threads=THREADS)
        pops.append(r.counters["census"] / 20000)
    pops = np.array(pops)
    exact = CF.infinite_population(1.0, 0.6, 0.5, 1.0, 20.0)
    assert exact == pytest.approx(math.exp(2.0))
    assert abs(pops.mean() - exact) < 4 * pops.std(ddof=1) / math.sqrt(len(pops))
    m, s = r.tallies[0]
    te = prob["tallies"][0]["t"]
    assert_z(zscores(m, s, CF.infinite_time_bins(1.0, 0.6, 0.5, 1.0, te)), min_bins=15)


def test_P5_multigroup_expm_config2():
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    exact = CF.multigroup_time_bins(mat, v, te)
    eig = CF.multigroup_time_bins(mat, v, te, method="eig")
    big = np.abs(exact) > 1e-6 * np.abs(exact).max()
    assert np.allclose(eig[big], exact[big], rtol=1e-6)
    r = oracle.run(prob, 1_000_000, seed=15, threads=THREADS)
    m, s = r.tallies[0]
    z = zscores(m.reshape(7, -1), s.reshape(7, -1), exact)
    assert_z(z, min_bins=300)
    # steady totals: int_0^inf phi = -A^{-1} phi0
    A = CF.multigroup_operator(mat, v)
    phi0 = np.zeros(7)
    phi0[0] = v[0]
    tot = np.linalg.solve(A, -phi0)
    gm = m.reshape(7, -1).sum(1)
    gs = np.sqrt((s.reshape(7, -1) ** 2).sum(1))  # bins of one group are positively
    assert np.all(np.abs(gm - tot) < 4 * s.reshape(7, -1).sum(1))  # correlated: sum of sigmas
    assert gs.shape == (7,)


@pytest.mark.slow
def test_P5_vanloan_matches_radau():
    prob = P.config2()
    mat, v, te = prob["materials"][0], prob["speed"], prob["tallies"][0]["t"]
    exact = CF.multigroup_time_bins(mat, v, te)
    ode = CF.multigroup_time_bins_ode(mat, v, te)
    assert np.max(np.abs(exact - ode)) < 1e-9 * np.abs(exact).max()


@pytest.mark.parametrize("name", ["config1", "config2", "config3", "azurv1"])
def test_P6_conservation_counts(name):
    """Every particle started (primary or secondary) ends in exactly one way."""
    prob = P.azurv1() if name == "azurv1" else P.by_name(name)
    n = 3000 if name == "config3" else 20000
    c = oracle.run(prob, n, seed=16, threads=THREADS).counters
    started = c["source"] + c["secondary"] + c["ww_split"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"]
    assert started == ended
    assert c["lost"] == 0
    assert c["collision"] == c["scatter"] + c["capture"] + c["production"]


def test_P6_balance_config1():
    """Config 1 in expectation: Sigma_a * total track length + leakage = 1 per source."""
    r = oracle.run(P.config1(), 400000, seed=17, threads=THREADS)
    m, s = r.tallies[0]
    bal = 0.5 * m.sum() + r.leak_mean.sum()
    assert abs(bal - 1.0) < 4 * (0.5 * s.sum() + r.leak_std.sum())
    c = r.counters
    assert c["capture"] + c["leak"] == c["source"]


def test_P7_error_converges_as_inverse_sqrt_N():
    """RMS error against the closed form falls as N^-1/2 (paper Section 3): fitted slope over
    N = 1e3 .. 1e5 with 16 replicates per N."""
    sa = 0.5
    prob = P.infinite_medium_1g(1.0, 1.0 - sa)
    Ns = [1000, 10000, 100000]
    rms = []
    for n in Ns:
        errs = [oracle.run(prob, n, seed=1000 * n + i, threads=THREADS).tallies[0][0].sum() - 1 / sa
                for i in range(16)]
        rms.append(math.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(Ns), np.log(rms), 1)[0]
    assert -0.65 < slope < -0.35


def _uniform_lattice(n=5):
    """Lattice geometry whose three materials are identical (one group): pins and walls are
    transparent, so the medium is an infinite homogeneous one in disguise."""
    mat = P.material([1.0], [[0.6]])
    return P.lattice_problem(n=n, G=1, mats=[mat, mat, mat], mesh_n=2 * n, n_tbins=1,
                             name="uniform_lattice"), 0.4


def test_lattice_transparent_pins_flux_and_crossings():
    prob, sa = _uniform_lattice(5)
    prob["t_census"] = math.inf
    prob["tallies"][0]["t"] = [0.0, math.inf]
    side = 5 * 1.26
    r = oracle.run(prob, 40000, seed=18, threads=THREADS, log_first=0, log_count=40000,
                   log_cap=4_000_000)
    m, s = r.tallies[0]
    # uniform flux: each of the 10x10 mesh bins holds 1/100 of the total 1/Sigma_a
    assert_z(zscores(m, s, np.full(m.shape, (1 / sa) / 100)), min_bins=100)
    ev = r.events
    assert len(ev) < 4_000_000
    density = (1 / sa) / (side * side)          # track length per unit area (per unit z)
    pins = int(np.sum(np.asarray(prob["lattice"]["pin_material"]) >= 0))
    exp_pin = CF.isotropic_crossings(density, pins * 2 * math.pi * 0.54)
    exp_wall = CF.isotropic_crossings(density, 2 * 4 * 5 * 1.26)
    n_pin = np.sum((ev["kind"] == 1) & (ev["outcome"] == 4)) / 40000
    n_wall = np.sum((ev["kind"] == 1) & (ev["outcome"] == 3)) / 40000
    # crossings per history are strongly correlated within a history: allow 3% (about 6 sigma
    # of the Poisson-like spread at this N)
    assert n_pin == pytest.approx(exp_pin, rel=0.03)
    assert n_wall == pytest.approx(exp_wall, rel=0.03)


def test_lattice_pin_material_changes_result():
    """Control for the transparent-pin test: making the pin material a pure absorber must lower
    the total track length (the pins are really tracked)."""
    prob, sa = _uniform_lattice(5)
    prob["tallies"][0]["t"] = [0.0, math.inf]
    prob["t_census"] = math.inf
    prob["materials"][0] = P.material([1.0], [[0.0]])
    prob["lattice"]["pin_material"] = [0] * 25
    r = oracle.run(prob, 20000, seed=19, threads=THREADS)
    m, s = r.tallies[0]
    assert m.sum() + 4 * s.sum() < 1 / sa


# ----------------------------------------------------------------------------- sharding


def test_history_sharding_fixed_point_exact():
    """Histories are independent and keyed by their index, so running [0, N) in one piece or as
    disjoint ranges gives bit-identical int64 fixed-point tallies after summation."""
    prob = P.config3()
    one = oracle.run(prob, 600, seed=20, threads=1)
    parts = [oracle.run(prob, 200, seed=20, threads=2, first=f) for f in (0, 200, 400)]
    assert np.array_equal(one.fixed, sum(p.fixed for p in parts))
    assert one.counters == {k: sum(p.counters[k] for p in parts) for k in one.counters}


# ----------------------------------------------------------------------------- MLP reference


def test_mlp_reference_gradient_finite_differences():
    H = 8
    rng = np.random.default_rng(0)
    npar = oracle.mlp_param_count(H)
    prm = rng.normal(0, 0.5, npar)
    x = rng.uniform(-1, 1, (16, 5))
    tgt = rng.normal(0, 1, 16)
    wt = rng.uniform(0.5, 2, 16)
    loss, y, g = oracle.mlp_loss_grad(prm, x, tgt, wt, H=H)
    eps = 1e-6
    for i in rng.choice(npar, 40, replace=False):
        pp, pm = prm.copy(), prm.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (oracle.mlp_loss_grad(pp, x, tgt, wt, H=H)[0]
              - oracle.mlp_loss_grad(pm, x, tgt, wt, H=H)[0]) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)
    # forward: a zero network outputs its last bias
    z = np.zeros(npar)
    z[-1] = 0.7
    assert np.allclose(oracle.mlp_loss_grad(z, x, H=H)[1], 0.7)


# ----------------------------------------------------------------------------- weight windows


def test_weight_windows_unbiased_against_analog():
    """Splitting and roulette change only the variance: on an 8 cm slab stack the weight-window
    run's mesh tally agrees with the analog run's bin by bin within 4 sigma and its detector total
    within 4 sigma, every particle started (source, split copy) ends exactly once, and the windows
    lower the detector's relative error per history."""
    prob = P.slab_stack(thickness=8.0, n_layers=4, detector=2.0, ww_bin=1.0, name="thin")
    ww = P.exponential_ww(prob, decay=0.8)
    na, nw = 2_000_000, 400_000
    a = oracle.run(prob, na, seed=31, threads=THREADS)
    w = oracle.run(prob, nw, seed=32, threads=THREADS, ww=ww)
    ma, sa = (np.ravel(v) for v in a.tallies[1])
    mw, sw = (np.ravel(v) for v in w.tallies[1])
    ok = (sa > 0) & (sw > 0) & (sa < 0.1 * ma) & (sw < 0.1 * mw)
    z = (mw[ok] - ma[ok]) / np.sqrt(sa[ok] ** 2 + sw[ok] ** 2)
    assert ok.sum() >= 20 and np.all(np.abs(z) < 4), (ok.sum(), np.abs(z).max())
    da, dsa = a.tallies[0][0].sum(), a.tallies[0][1].sum()
    dw, dsw = w.tallies[0][0].sum(), w.tallies[0][1].sum()
    assert abs(da - dw) < 4 * (dsa + dsw)  # bins of one history are correlated: sum of sigmas
    c = w.counters
    assert c["ww_split"] > 0 and c["ww_kill"] > 0
    started = c["source"] + c["secondary"] + c["ww_split"]
    ended = c["capture"] + c["production"] + c["leak"] + c["census"] + c["lost"] + c["ww_kill"]
    assert started == ended
    assert dsw / dw * math.sqrt(nw) < dsa / da * math.sqrt(na)
