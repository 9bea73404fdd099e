"""Seeded synthetic problem generators for the multigroup time-dependent random walk.

This module only *describes* problems: cross sections, geometry, source, tally meshes
and census time, as plain Python dicts of numbers.  It contains none of the transport
arithmetic, so both the CUDA path (through the C ABI) and the CPU oracle consume the same
dicts without sharing any method code.

The paper (Section 3) states the problem class: fixed-source multigroup transport on
quadric-surface CSG with a time-dependent source, a time census and time-dependent mesh
tallies.  The five workloads below are synthetic stand-ins whose shapes follow that
statement; no benchmark cross-section data is used.

Problem dict layout (all lengths in cm, times in s, cross sections in 1/cm):

    G, speed[G]
    materials: list of {sigma_t[G], sigma_s[G][G] (from, to), sigma_f[G], nu[G], chi[G]}
    surfaces:  list of {kind: 'PX'|'PY'|'PZ'|'CZ'|'CX'|'CY'|'SQ'|'GQ', coef, bc: 'interior'|'vacuum'|'reflect'}
               coef: plane [c]; z-cylinder [x0, y0, r]; x-cylinder [y0, z0, r]; y-cylinder [x0, z0, r];
               sphere [x0, y0, z0, r]; general quadric [A..J] of
               A x^2 + B y^2 + C z^2 + D xy + E yz + F zx + G x + H y + I z + J
    cells:     list of {halfspaces: [(surface, +1|-1), ...], material: m (>=0) or -1 (lattice)}
    lattice:   None or {nx, ny, x0, y0, pitch, radius, pin_material (-1 = no pin),
                        matrix_material[, nz, z0, pitch_z]}: elements of side `pitch` holding a
               z-cylinder pin; with nz >= 2 axial layers of height pitch_z from z0, pin_material
               laid out [nz][ny][nx] (else [ny][nx], one layer unbounded in z)
    source:    {pos: 'box'|'surface_x0', lo[3], hi[3], dir: 'iso'|'beam_x'|'cos_x',
                group_pdf[G], t0, t1}
    tallies:   list of {x: edges, y: edges, z: edges, t: edges, estimator: 'track'|'crossing'}
               'track': track-length estimator over the nt time bins between the t edges;
               'crossing': time-crossing estimator of the flux at the nt+1 time points t
    t_census:  float (math.inf for steady state)
"""
from __future__ import annotations

import math

import numpy as np

INF = math.inf

# --------------------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------------------


def material(sigma_t, sigma_s, sigma_f=None, nu=None, chi=None):
    sigma_t = np.asarray(sigma_t, dtype=np.float64)
    G = sigma_t.size
    sigma_s = np.asarray(sigma_s, dtype=np.float64).reshape(G, G)
    sigma_f = np.zeros(G) if sigma_f is None else np.asarray(sigma_f, dtype=np.float64)
    nu = np.zeros(G) if nu is None else np.asarray(nu, dtype=np.float64)
    if chi is None:
        chi = np.zeros(G)
        chi[0] = 1.0
    chi = np.asarray(chi, dtype=np.float64)
    return {"sigma_t": sigma_t.tolist(), "sigma_s": sigma_s.tolist(),
            "sigma_f": sigma_f.tolist(), "nu": nu.tolist(), "chi": chi.tolist()}


def box_surfaces(lo, hi, bc, axes=(0, 1, 2)):
    """Planes bounding an axis-aligned box on the requested axes: returns (surfaces, halfspaces)."""
    kinds = ("PX", "PY", "PZ")
    surfs, hs = [], []
    for a in axes:
        surfs.append({"kind": kinds[a], "coef": [float(lo[a])], "bc": bc})
        hs.append((len(surfs) - 1, +1))
        surfs.append({"kind": kinds[a], "coef": [float(hi[a])], "bc": bc})
        hs.append((len(surfs) - 1, -1))
    return surfs, hs


def source(pos="box", lo=(0, 0, 0), hi=(0, 0, 0), direction="iso", G=1, group=0,
           group_pdf=None, t0=0.0, t1=0.0):
    if group_pdf is None:
        group_pdf = np.zeros(G)
        group_pdf[group] = 1.0
    return {"pos": pos, "lo": [float(v) for v in lo], "hi": [float(v) for v in hi],
            "dir": direction, "group_pdf": [float(v) for v in group_pdf],
            "t0": float(t0), "t1": float(t1)}


def mesh(x=(-INF, INF), y=(-INF, INF), z=(-INF, INF), t=(0.0, INF), estimator="track"):
    return {"x": [float(v) for v in x], "y": [float(v) for v in y],
            "z": [float(v) for v in z], "t": [float(v) for v in t], "estimator": estimator}


def with_tallies(prob, tallies):
    """A copy of the problem with its tally list replaced."""
    q = dict(prob)
    q["tallies"] = list(tallies)
    return q


def problem(name, G, speed, materials, surfaces, cells, src, tallies, t_census=INF,
            lattice=None):
    return {"name": name, "G": int(G), "speed": [float(v) for v in speed],
            "materials": materials, "surfaces": surfaces, "cells": cells,
            "lattice": lattice, "source": src, "tallies": tallies,
            "t_census": float(t_census)}


def log_time_edges(n_bins, t_lo=1e-9, t_hi=1e-3):
    """Edges {0} U logspace(t_lo, t_hi, n_bins): n_bins bins, the first one [0, t_lo]."""
    return [0.0] + np.logspace(math.log10(t_lo), math.log10(t_hi), n_bins).tolist()


def log_speeds(G, v_fast=2e9, v_slow=2e5):
    if G == 1:
        return [v_fast]
    return np.logspace(math.log10(v_fast), math.log10(v_slow), G).tolist()


def seeded_scatter(rng, G, sigma_t, c_lo, c_hi, upscatter_frac=0.1):
    """Downscatter-dominant scattering matrix (from, to) with per-group ratio c_g ~ U[c_lo, c_hi].

    Downscatter weights ~U[0,1] for g' >= g; the two slowest groups also get upscatter weights
    summing to at most `upscatter_frac` of their row.
    """
    S = np.zeros((G, G))
    c = rng.uniform(c_lo, c_hi, G)
    for g in range(G):
        wts = np.zeros(G)
        wts[g:] = rng.uniform(0.0, 1.0, G - g)
        wts[g] += 1e-3  # keep the self-scatter entry non-empty
        if G >= 3 and g >= G - 2:
            up = rng.uniform(0.0, 1.0, g)
            if up.sum() > 0:
                up *= upscatter_frac * wts.sum() / up.sum() * rng.uniform(0.2, 1.0)
            wts[:g] = up
        S[g] = wts / wts.sum() * c[g] * sigma_t[g]
    return S


# --------------------------------------------------------------------------------------
# closed-form pin problems (used by the oracle's tests)
# --------------------------------------------------------------------------------------


def slab_problem(L=5.0, sigma_t=1.0, sigma_s=0.5, src_hi=1.0, n_bins=50, direction="iso",
                 surface_source=False, name="slab"):
    """Config-1 family: 1D slab 0<x<L, vacuum both ends, one group, steady state."""
    surfs = [{"kind": "PX", "coef": [0.0], "bc": "vacuum"},
             {"kind": "PX", "coef": [float(L)], "bc": "vacuum"}]
    cells = [{"halfspaces": [(0, +1), (1, -1)], "material": 0}]
    mat = material([sigma_t], [[sigma_s]])
    if surface_source:
        src = source("surface_x0", (0, 0, 0), (0, 0, 0), direction, 1)
    else:
        src = source("box", (0, 0, 0), (src_hi, 0, 0), direction, 1)
    tal = [mesh(x=np.linspace(0.0, L, n_bins + 1))]
    return problem(name, 1, [1.0], [mat], surfs, cells, src, tal)


def infinite_medium_1g(sigma_t=1.0, sigma_s=0.5, sigma_f=0.0, nu=0.0, speed=1.0,
                       t_edges=(0.0, INF), t_census=INF, side=10.0, name="inf1g"):
    """One-group infinite medium: reflective cube, uniform isotropic pulse source at t=0."""
    surfs, hs = box_surfaces((0, 0, 0), (side,) * 3, "reflect")
    cells = [{"halfspaces": hs, "material": 0}]
    mat = material([sigma_t], [[sigma_s]], [sigma_f], [nu], [1.0])
    src = source("box", (0, 0, 0), (side,) * 3, "iso", 1)
    tal = [mesh(x=(0, side), y=(0, side), z=(0, side), t=t_edges)]
    return problem(name, 1, [speed], [mat], surfs, cells, src, tal, t_census)


def azurv1(c=1.1, t_end=20.0, n_tbins=20):
    """Supercritical AZURV1 stand-in (paper Section 3): c = (sigma_s + nu sigma_f)/sigma_t = 1.1,
    sigma_t = v = 1, census at t_end mean-free-times."""
    sigma_s = 0.6
    sigma_f = 0.2
    nu = (c - sigma_s) / sigma_f
    return infinite_medium_1g(1.0, sigma_s, sigma_f, nu, 1.0,
                              t_edges=np.linspace(0.0, t_end, n_tbins + 1),
                              t_census=t_end, name="azurv1")


# --------------------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------------------


def config1(sigma_s=0.5):
    """1D slab 0<x<5 cm, vacuum, 1 group, sigma_t = 1, isotropic source uniform on [0,1),
    50 x-bins + left/right leakage (leakage is reported per vacuum surface)."""
    return slab_problem(5.0, 1.0, sigma_s, 1.0, 50, name="config1")


def config2_xs(seed=2, G=7):
    rng = np.random.default_rng(seed)
    sigma_t = rng.uniform(0.2, 2.0, G)
    S = seeded_scatter(rng, G, sigma_t, 0.3, 0.9)
    return sigma_t, S


def config2(seed=2, G=7, n_tbins=100, side=10.0):
    """Infinite homogeneous medium (reflective 10 cm cube), 7 groups, pulse at t=0 in group 1,
    no secondary production; 100 log-spaced time bins; census at 1e-3 s."""
    sigma_t, S = config2_xs(seed, G)
    surfs, hs = box_surfaces((0, 0, 0), (side,) * 3, "reflect")
    cells = [{"halfspaces": hs, "material": 0}]
    mat = material(sigma_t, S)
    src = source("box", (0, 0, 0), (side,) * 3, "iso", G, 0)
    t_edges = log_time_edges(n_tbins)
    tal = [mesh(x=(0, side), y=(0, side), z=(0, side), t=t_edges)]
    return problem("config2", G, log_speeds(G), [mat], surfs, cells, src, tal, t_edges[-1])


def config2_crossing(seed=2, G=7, n_tbins=100, side=10.0):
    """Config 2 with the flux tallied by the time-crossing estimator at the 101 time points
    {0} U logspace(1e-9, 1e-3, 100) (the paper tallies its multigroup pulse this way), next to the
    track-length tally over the 100 bins between them."""
    prob = config2(seed, G, n_tbins, side)
    tl = prob["tallies"][0]
    cross = mesh(x=tl["x"], y=tl["y"], z=tl["z"], t=tl["t"], estimator="crossing")
    q = with_tallies(prob, [tl, cross])
    q["name"] = "config2_crossing"
    return q


def eigen_infinite_1g(sigma_t=1.0, sigma_s=0.5, sigma_f=0.2, nu=2.4, side=10.0):
    """One-group infinite medium with fission for k-eigenvalue runs (steady state):
    k = nu Sigma_f / (Sigma_t - Sigma_s) = 0.96."""
    q = infinite_medium_1g(sigma_t, sigma_s, sigma_f, nu, 1.0, side=side, name="eigen1g")
    return q


def eigen_infinite_mg(seed=6, G=7, side=10.0):
    """Seven-group infinite medium of one seeded fissile material (reflective cube), steady state,
    for k-eigenvalue runs; a group-flux tally."""
    rng = np.random.default_rng([seed, 2000])
    mat = _lattice_materials(rng, G, True)
    surfs, hs = box_surfaces((0, 0, 0), (side,) * 3, "reflect")
    cells = [{"halfspaces": hs, "material": 0}]
    src = source("box", (0, 0, 0), (side,) * 3, "iso", G, 0)
    tal = [mesh(x=(0, side), y=(0, side), z=(0, side))]
    return problem("eigenmg", G, log_speeds(G), [mat], surfs, cells, src, tal)


def pin_cell(seed=7, G=7, pitch=1.26, radius=0.54, mesh_n=4):
    """Infinite pin cell for k-eigenvalue runs (the paper's C5G7 UO2 pin-cell benchmark in shape
    only: seeded synthetic cross sections, no C5G7 data): a fissile pin of radius 0.54 cm in a
    1.26 cm square of a scattering moderator, reflective on all sides (z infinite), 7 groups,
    steady state, uniform initial source; a 4 x 4 group-flux mesh."""
    rng = np.random.default_rng([seed, 3000])
    fuel = _lattice_materials(rng, G, True)
    sigma_t = rng.uniform(0.3, 2.0, G)
    moderator = material(sigma_t, seeded_scatter(rng, G, sigma_t, 0.95, 0.995))  # weakly absorbing
    surfs, hs = box_surfaces((0, 0, 0), (pitch, pitch, 0), "reflect", axes=(0, 1))
    cells = [{"halfspaces": hs, "material": -1}]
    lat = {"nx": 1, "ny": 1, "x0": 0.0, "y0": 0.0, "pitch": float(pitch), "radius": float(radius),
           "pin_material": [0], "matrix_material": 1}
    src = source("box", (0, 0, 0), (pitch, pitch, 0), "iso", G, 0)
    tal = [mesh(x=np.linspace(0, pitch, mesh_n + 1), y=np.linspace(0, pitch, mesh_n + 1))]
    return problem("pincell", G, log_speeds(G), [fuel, moderator], surfs, cells, src, tal, INF, lat)


def absorber_in_void(body, sigma_t=1.0, point=(0.0, 0.0, 0.0), half=10.0, name="body", extra_cells=()):
    """A pure absorber (one group, Sigma_t) bounded by `body` = (surfaces, halfspaces) inside a void box
    [-half, half]^3 with vacuum walls, isotropic point source at `point`: the leakage through the box
    is the probability that a source particle escapes the absorber."""
    bsurfs, bhs = body
    box, box_hs = box_surfaces((-half,) * 3, (half,) * 3, "vacuum")
    surfs = list(bsurfs) + box
    nb = len(bsurfs)
    inside = {"halfspaces": list(bhs), "material": 0}
    cells = [inside]
    # the void: inside the box and outside the body (one cell per bounding half-space flipped, in order)
    for i, (s, sn) in enumerate(bhs):
        hs = [(s2, sn2) for s2, sn2 in bhs[:i]] + [(s, -sn)] + [(b + nb, sn2) for b, sn2 in box_hs]
        cells.append({"halfspaces": hs, "material": 1})
    mats = [material([sigma_t], [[0.0]]), material([0.0], [[0.0]])]
    src = source("box", point, point, "iso", 1)
    tal = [mesh(x=(-half, half), y=(-half, half), z=(-half, half))]
    return problem(name, 1, [1.0], mats, surfs, cells, src, tal)


def sphere_absorber(R=1.0, sigma_t=1.0, point=(0.0, 0.0, 0.0), center=(0.0, 0.0, 0.0)):
    s = [{"kind": "SQ", "coef": [float(c) for c in center] + [float(R)], "bc": "interior"}]
    return absorber_in_void((s, [(0, -1)]), sigma_t, point, name="sphere")


def xcylinder_absorber(R=1.0, L=2.0, sigma_t=1.0, axis="x"):
    """Finite cylinder of radius R along `axis` ('x', 'y' or 'z') between the planes at -L and +L,
    point source at the centre."""
    kind = {"x": "CX", "y": "CY", "z": "CZ"}[axis]
    plane = {"x": "PX", "y": "PY", "z": "PZ"}[axis]
    s = [{"kind": kind, "coef": [0.0, 0.0, float(R)], "bc": "interior"},
         {"kind": plane, "coef": [-float(L)], "bc": "interior"},
         {"kind": plane, "coef": [float(L)], "bc": "interior"}]
    return absorber_in_void((s, [(0, -1), (1, +1), (2, -1)]), sigma_t, name=f"cyl{axis}")


def ellipsoid_matrix(a, b, c, angles):
    """Q = R diag(1/a^2, 1/b^2, 1/c^2) R^T of an ellipsoid rotated by the z-y-x angles."""
    az, ay, ax = angles
    Rz = np.array([[math.cos(az), -math.sin(az), 0], [math.sin(az), math.cos(az), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(ay), 0, math.sin(ay)], [0, 1, 0], [-math.sin(ay), 0, math.cos(ay)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
    R = Rz @ Ry @ Rx
    return R @ np.diag([1 / a**2, 1 / b**2, 1 / c**2]) @ R.T


def ellipsoid_absorber(a=1.0, b=0.6, c=1.5, sigma_t=1.0, angles=(0.0, 0.0, 0.0), center=(0.0, 0.0, 0.0),
                       point=None):
    """Ellipsoid with semi-axes a, b, c, rotated by the z-y-x angles and centred at `center`, given as
    a general quadric (all ten coefficients in use when rotated and moved), point source at the
    centre: (p - c0)^T Q (p - c0) < 1 with Q = R diag(1/a^2, 1/b^2, 1/c^2) R^T."""
    Q = ellipsoid_matrix(a, b, c, angles)
    c0 = np.asarray(center, dtype=np.float64)
    g = -2.0 * Q @ c0
    J = float(c0 @ Q @ c0) - 1.0
    coef = [Q[0, 0], Q[1, 1], Q[2, 2], 2 * Q[0, 1], 2 * Q[1, 2], 2 * Q[0, 2], g[0], g[1], g[2], J]
    s = [{"kind": "GQ", "coef": [float(v) for v in coef], "bc": "interior"}]
    p0 = c0 if point is None else np.asarray(point, dtype=np.float64)
    return absorber_in_void((s, [(0, -1)]), sigma_t, point=tuple(float(v) for v in p0), name="ellipsoid")


def quadric_assembly(seed=8, G=2, half=4.0):
    """Scattering regions bounded by quadrics in a reflective box [-4, 4]^3: a sphere, a cylinder
    along x from wall to wall, and a rotated ellipsoid (a general quadric), each with its own seeded
    material, in a seeded background material; uniform source, steady state, a 4 x 4 x 4 mesh."""
    rng = np.random.default_rng([seed, 4000])
    mats = []
    for _ in range(4):
        st = rng.uniform(0.3, 1.5, G)
        mats.append(material(st, seeded_scatter(rng, G, st, 0.5, 0.9)))
    box, box_hs = box_surfaces((-half,) * 3, (half,) * 3, "reflect")
    Q = ellipsoid_matrix(1.0, 0.6, 1.2, (0.5, 0.3, -0.8))
    c0 = np.array([2.2, -0.5, -1.6])
    g = -2.0 * Q @ c0
    gq = [Q[0, 0], Q[1, 1], Q[2, 2], 2 * Q[0, 1], 2 * Q[1, 2], 2 * Q[0, 2], g[0], g[1], g[2], float(c0 @ Q @ c0) - 1.0]
    surfs = box + [{"kind": "SQ", "coef": [-2.0, 0.5, -1.0, 1.5], "bc": "interior"},
                   {"kind": "CX", "coef": [0.0, 2.6, 1.0], "bc": "interior"},
                   {"kind": "GQ", "coef": [float(v) for v in gq], "bc": "interior"}]
    sph, cyl, ell = 6, 7, 8
    cells = [{"halfspaces": [(sph, -1)], "material": 0},
             {"halfspaces": [(cyl, -1), box_hs[0], box_hs[1]], "material": 1},
             {"halfspaces": [(ell, -1)], "material": 2},
             {"halfspaces": box_hs + [(sph, +1), (cyl, +1), (ell, +1)], "material": 3}]
    src = source("box", (-half,) * 3, (half,) * 3, "iso", G, 0)
    tal = [mesh(x=np.linspace(-half, half, 5), y=np.linspace(-half, half, 5), z=np.linspace(-half, half, 5))]
    return problem("quadrics", G, log_speeds(G), mats, surfs, cells, src, tal)


def offspring_matrix(mat):
    """K[g][g'] = (sigma_s[g->g'] + nu sigma_f[g] chi[g']) / sigma_t[g] (mean offspring per
    collision); used only to scale the synthetic inputs."""
    st = np.asarray(mat["sigma_t"])
    S = np.asarray(mat["sigma_s"])
    F = np.outer(np.asarray(mat["nu"]) * np.asarray(mat["sigma_f"]), np.asarray(mat["chi"]))
    return (S + F) / st[:, None]


def _lattice_materials(rng, G, fissile):
    sigma_t = rng.uniform(0.3, 2.0, G)
    while True:
        S = seeded_scatter(rng, G, sigma_t, 0.3, 0.8)
        if max(abs(np.linalg.eigvals(S / sigma_t[:, None]))) <= 0.8:
            break
    if not fissile:
        return material(sigma_t, S)
    # fission in a fraction of sigma_t, fast-peaked spectrum
    room = sigma_t - S.sum(axis=1)
    sigma_f = room * rng.uniform(0.2, 0.6, G)
    nu = rng.uniform(2.3, 2.9, G)
    chi = np.zeros(G)
    chi[: max(1, G // 2)] = rng.uniform(0.1, 1.0, max(1, G // 2))
    chi /= chi.sum()
    return material(sigma_t, S, sigma_f, nu, chi)


def scale_production(mats, target=0.9, rowsum_cap=0.98):
    """Bisection on one factor lambda multiplying sigma_f of every fissile material so that
    max_m rho(K_m) = target; asserts every offspring row sum <= rowsum_cap."""
    def rho(lam):
        r = 0.0
        for m in mats:
            mm = dict(m)
            mm["sigma_f"] = (np.asarray(m["sigma_f"]) * lam).tolist()
            r = max(r, max(abs(np.linalg.eigvals(offspring_matrix(mm)))))
        return r
    lo, hi = 0.0, 1.0
    while rho(hi) < target:
        hi *= 2.0
        if hi > 1e6:
            raise ValueError("cannot reach target spectral radius")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if rho(mid) < target:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    out = []
    for m in mats:
        mm = dict(m)
        mm["sigma_f"] = (np.asarray(m["sigma_f"]) * lam).tolist()
        out.append(mm)
    rows = max(float(offspring_matrix(m).sum(axis=1).max()) for m in out)
    return out, lam, rows


def config3_materials(seed=3, G=7, target=0.9):
    for attempt in range(64):
        rng = np.random.default_rng([seed, attempt])
        mats = [_lattice_materials(rng, G, True), _lattice_materials(rng, G, True),
                _lattice_materials(rng, G, False)]
        scaled, lam, rows = scale_production(mats, target)
        if rows <= 0.98:
            return scaled
    raise RuntimeError("no seeded material set met the offspring row-sum cap")


def lattice_problem(n=17, pitch=1.26, radius=0.54, G=7, seed=3, mesh_n=34, n_tbins=50,
                    mats=None, name="config3"):
    """2D n x n lattice of z-cylinders in a reflective box (z infinite)."""
    rng = np.random.default_rng([seed, 1000])
    if mats is None:
        mats = config3_materials(seed, G)
    side = n * pitch
    surfs, hs = box_surfaces((0, 0, 0), (side, side, 0), "reflect", axes=(0, 1))
    cells = [{"halfspaces": hs, "material": -1}]
    pins = np.where(rng.uniform(size=n * n) < 0.25, 1, 0).astype(int)
    lat = {"nx": n, "ny": n, "x0": 0.0, "y0": 0.0, "pitch": float(pitch),
           "radius": float(radius), "pin_material": pins.tolist(), "matrix_material": 2}
    src = source("box", (0, 0, 0), (side, side, 0), "iso", G, 0)
    t_edges = log_time_edges(n_tbins)
    tal = [mesh(x=np.linspace(0, side, mesh_n + 1), y=np.linspace(0, side, mesh_n + 1),
                t=t_edges)]
    return problem(name, G, log_speeds(G), mats, surfs, cells, src, tal, t_edges[-1], lat)


def config3(seed=3):
    """17x17 lattice of cylinders (r=0.54, pitch 1.26) in a reflective box, 7 groups,
    3 seeded materials (two pin fills, one matrix), production scaled to spectral radius 0.9,
    uniform volumetric source, 34x34x7x50 space-group-time mesh."""
    return lattice_problem(seed=seed)


def absorber_material(rng, G):
    """A strong absorber (control-rod-like): Sigma_t in [1, 3], 10% scattering, downscatter only."""
    sigma_t = rng.uniform(1.0, 3.0, G)
    S = np.zeros((G, G))
    for g in range(G):
        S[g, g:] = 0.1 * sigma_t[g] * rng.dirichlet(np.ones(G - g))
    return material(sigma_t, S)


def axial_lattice(n=5, nz=6, pitch=1.26, pitch_z=2.0, radius=0.54, G=7, seed=9, n_rod_layers=2,
                  n_tbins=20, bc_z="vacuum", name="axial"):
    """3D lattice with axial zoning (a pin-lattice assembly in the shape of the paper's 3D C5G7
    configurations; seeded synthetic cross sections, no C5G7 data): n x n elements of pitch `pitch`,
    nz layers of height pitch_z.  Layer 0 is a bottom reflector (moderator only); layers 1..nz-2 hold
    fuel pins of two seeded fissile materials; absorber rods at a seeded eighth of the positions fill
    the top reflector layer and the top `n_rod_layers` fuel layers (partially inserted rods).
    Reflective in x and y, `bc_z` at the bottom and top; source uniform in the fuel layers, group 0,
    t = 0; mesh of one bin per element and layer over log-spaced time bins."""
    rng = np.random.default_rng([seed, 4000])
    mats = config3_materials(seed, G) + [absorber_material(rng, G)]  # fuel A, fuel B, moderator, rod
    side, height = n * pitch, nz * pitch_z
    surfs, hs = box_surfaces((0, 0, 0), (side, side, height), "reflect", axes=(0, 1))
    zs, zhs = box_surfaces((0, 0, 0), (side, side, height), bc_z, axes=(2,))
    surfs += zs
    hs += [(i + 4, sn) for i, sn in zhs]
    cells = [{"halfspaces": hs, "material": -1}]
    fuel = rng.integers(0, 2, n * n)
    rods = rng.uniform(size=n * n) < 0.125
    pins = np.full((nz, n * n), -1, dtype=int)
    for iz in range(1, nz - 1):
        pins[iz] = fuel
        if iz >= nz - 1 - n_rod_layers:
            pins[iz][rods] = 3
    pins[nz - 1][rods] = 3
    lat = {"nx": n, "ny": n, "x0": 0.0, "y0": 0.0, "pitch": float(pitch), "radius": float(radius),
           "pin_material": pins.ravel().tolist(), "matrix_material": 2,
           "nz": nz, "z0": 0.0, "pitch_z": float(pitch_z)}
    src = source("box", (0, 0, pitch_z), (side, side, height - pitch_z), "iso", G, 0)
    t_edges = log_time_edges(n_tbins)
    tal = [mesh(x=np.linspace(0, side, n + 1), y=np.linspace(0, side, n + 1),
                z=np.linspace(0, height, nz + 1), t=t_edges)]
    return problem(name, G, log_speeds(G), mats, surfs, cells, src, tal, t_edges[-1], lat)


def lattice_absorber_3d(n=3, nz=3, pitch=1.0, pitch_z=1.0, radius=0.35, point=(1.3, 1.7, 1.2),
                        sigma=(0.6, 1.5, 0.3), seed=10):
    """Purely absorbing one-group 3D lattice (n x n elements, nz layers) with vacuum walls and an
    isotropic point source at `point`: the leakage is the escape probability.  Matrix Sigma_t =
    sigma[0]; each element of each layer holds a pin of Sigma_t sigma[1] or sigma[2] or none (seeded),
    so the optical depth along a ray depends on the layer it passes through."""
    rng = np.random.default_rng([seed, 5000])
    mats = [material([v], [[0.0]]) for v in sigma]
    side, height = n * pitch, nz * pitch_z
    surfs, hs = box_surfaces((0, 0, 0), (side, side, height), "vacuum")
    cells = [{"halfspaces": hs, "material": -1}]
    pins = rng.choice([-1, 1, 2], size=nz * n * n).astype(int)
    lat = {"nx": n, "ny": n, "x0": 0.0, "y0": 0.0, "pitch": float(pitch), "radius": float(radius),
           "pin_material": pins.tolist(), "matrix_material": 0,
           "nz": nz, "z0": 0.0, "pitch_z": float(pitch_z)}
    src = source("box", point, point, "iso", 1)
    tal = [mesh(x=(0, side), y=(0, side), z=(0, height))]
    return problem("lattice3d_absorber", 1, [1.0], mats, surfs, cells, src, tal, INF, lat)


def dogleg_duct(G=2, seed=11, L=40.0, w=8.0, n_tbins=10):
    """Streaming through a dog-leg void duct in a shield (in the shape of the paper's Kobayashi
    duct-streaming benchmark; seeded synthetic cross sections, no benchmark data).  The box [0, L]^3
    is cut by planes into axis-aligned boxes, each one cell: the source block [0, w]^3, a duct leg
    along x from the source block to x = L - w, a second leg along y up to y = L - w, and shield
    elsewhere.  Reflective on x = 0, y = 0, z = 0 (a quarter model), vacuum on the far faces.
    Source uniform in the source block, group 0, t = 0; a mesh along the duct and beside it."""
    rng = np.random.default_rng([seed, 6000])
    sigma_t = rng.uniform(0.3, 0.6, G)
    shield = material(sigma_t, seeded_scatter(rng, G, sigma_t, 0.4, 0.6))
    void = material(np.zeros(G), np.zeros((G, G)))
    sigma_t = rng.uniform(0.2, 0.4, G)
    src_mat = material(sigma_t, seeded_scatter(rng, G, sigma_t, 0.5, 0.7))
    xs = [0.0, w, L - 2 * w, L - w, L]
    ys = [0.0, w, L - w, L]
    zs = [0.0, w, L]
    surfs = []
    ids = {}
    for axis, kind, cuts in ((0, "PX", xs), (1, "PY", ys), (2, "PZ", zs)):
        for j, c in enumerate(cuts):
            bc = "interior"
            if j == 0:
                bc = "reflect"
            elif j == len(cuts) - 1:
                bc = "vacuum"
            ids[(axis, j)] = len(surfs)
            surfs.append({"kind": kind, "coef": [float(c)], "bc": bc})

    def region(ix, iy, iz):
        if iz != 0:
            return 0
        if ix == 0 and iy == 0:
            return 2  # source block
        if iy == 0 and ix in (1, 2):
            return 1  # first leg along x
        if ix == 2 and iy == 1:
            return 1  # second leg along y
        return 0

    cells = []
    for iz in range(len(zs) - 1):
        for iy in range(len(ys) - 1):
            for ix in range(len(xs) - 1):
                hs = [(ids[(0, ix)], +1), (ids[(0, ix + 1)], -1), (ids[(1, iy)], +1),
                      (ids[(1, iy + 1)], -1), (ids[(2, iz)], +1), (ids[(2, iz + 1)], -1)]
                cells.append({"halfspaces": hs, "material": region(ix, iy, iz)})
    src = source("box", (0, 0, 0), (w, w, w), "iso", G, 0)
    v = log_speeds(G)
    t_edges = np.concatenate([[0.0], np.logspace(-8, -5, n_tbins)])
    tal = [mesh(x=xs, y=np.linspace(0, L, 11), z=(0, w, L), t=t_edges)]
    return problem("dogleg", G, v, [shield, void, src_mat], surfs, cells, src, tal, t_edges[-1])


def config4_materials(seed=4, G=7, n_mat=4):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(n_mat):
        sigma_t = rng.uniform(0.5, 3.0, G)
        S = seeded_scatter(rng, G, sigma_t, 0.3, 0.95)
        mats.append(material(sigma_t, S))
    return mats


def slab_stack(thickness=200.0, n_layers=40, G=7, seed=4, detector=2.0, ww_bin=5.0,
               name="config4", t_edges=(0.0, INF), t_census=INF):
    """Deep-penetration x-layered slab stack (infinite in y, z), vacuum both ends, cosine
    (isotropic-flux) surface source at x=0 in group 1 at t = 0; tally 0 = detector on the last
    `detector` cm, tally 1 = coarse space-group mesh used to train weight windows; both tallies
    take the time bins `t_edges` (one bin holding every time by default)."""
    mats = config4_materials(seed, G)
    dx = thickness / n_layers
    xs = [i * dx for i in range(n_layers + 1)]
    surfs = []
    for i, x in enumerate(xs):
        bc = "vacuum" if i in (0, n_layers) else "interior"
        surfs.append({"kind": "PX", "coef": [float(x)], "bc": bc})
    cells = [{"halfspaces": [(i, +1), (i + 1, -1)], "material": i % len(mats)}
             for i in range(n_layers)]
    src = source("surface_x0", (0, 0, 0), (0, 0, 0), "cos_x", G, 0)
    n_ww = max(1, int(round(thickness / ww_bin)))
    tal = [mesh(x=(thickness - detector, thickness), t=t_edges),
           mesh(x=np.linspace(0.0, thickness, n_ww + 1), t=t_edges)]
    return problem(name, G, log_speeds(G), mats, surfs, cells, src, tal, t_census)


def pulse_stack(thickness=10.0, n_layers=5, n_tbins=12, t_hi=1e-4, ww_bin=1.0, seed=4, name="pulse"):
    """The slab stack hit by a pulse: the cosine surface source fires at t = 0, the detector and the
    window-training mesh are resolved in n_tbins time bins ({0} U logspace(1e-9, t_hi)), and the
    census ends every history at t_hi."""
    return slab_stack(thickness=thickness, n_layers=n_layers, seed=seed, detector=2.0, ww_bin=ww_bin, name=name,
                      t_edges=log_time_edges(n_tbins, 1e-9, t_hi), t_census=t_hi)


def config4(seed=4, thickness=200.0):
    """200 cm deep-penetration stack of 40 layers (4 seeded materials), detector on the last 2 cm,
    window-training mesh of 2 cm cells."""
    return slab_stack(thickness=thickness, seed=seed, ww_bin=2.0)


def config5(seed=5, n_problems=256, n_lo=1e4, n_hi=1e6):
    """256 independent problems of uneven size: types drawn from {1D slab, 2D slab, lattice},
    G ~ U{1..7}, histories log-uniform in [n_lo, n_hi].  Returns (problems, n_histories)."""
    rng = np.random.default_rng(seed)
    probs, nh = [], []
    for i in range(n_problems):
        kind = int(rng.integers(0, 3))
        G = int(rng.integers(1, 8))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        sub = int(rng.integers(0, 2**31))
        if kind == 0:
            probs.append(_slab1d(sub, G, f"p{i}_slab1d"))
        elif kind == 1:
            probs.append(_slab2d(sub, G, f"p{i}_slab2d"))
        else:
            probs.append(_small_lattice(sub, G, f"p{i}_lattice"))
        nh.append(n)
    return probs, nh


def _slab1d(seed, G, name):
    rng = np.random.default_rng(seed)
    n_layers = int(rng.integers(1, 5))
    L = float(rng.uniform(2.0, 10.0))
    xs = np.linspace(0.0, L, n_layers + 1)
    mats = []
    for _ in range(n_layers):
        st = rng.uniform(0.2, 2.0, G)
        mats.append(material(st, seeded_scatter(rng, G, st, 0.3, 0.9)))
    surfs = [{"kind": "PX", "coef": [float(x)],
              "bc": "vacuum" if i in (0, n_layers) else "interior"} for i, x in enumerate(xs)]
    cells = [{"halfspaces": [(i, +1), (i + 1, -1)], "material": i} for i in range(n_layers)]
    src = source("box", (0, 0, 0), (L, 0, 0), "iso", G, 0)
    tal = [mesh(x=np.linspace(0.0, L, 21))]
    return problem(name, G, log_speeds(G), mats, surfs, cells, src, tal)


def _slab2d(seed, G, name):
    rng = np.random.default_rng(seed)
    L = float(rng.uniform(2.0, 10.0))
    surfs = [{"kind": "PX", "coef": [0.0], "bc": "vacuum"},
             {"kind": "PX", "coef": [L / 2], "bc": "interior"},
             {"kind": "PX", "coef": [L], "bc": "vacuum"},
             {"kind": "PY", "coef": [0.0], "bc": "reflect"},
             {"kind": "PY", "coef": [L / 2], "bc": "interior"},
             {"kind": "PY", "coef": [L], "bc": "reflect"}]
    mats, cells = [], []
    for j in range(2):
        for i in range(2):
            st = rng.uniform(0.2, 2.0, G)
            mats.append(material(st, seeded_scatter(rng, G, st, 0.3, 0.9)))
            cells.append({"halfspaces": [(i, +1), (i + 1, -1), (3 + j, +1), (4 + j, -1)],
                          "material": len(mats) - 1})
    src = source("box", (0, 0, 0), (L, L, 0), "iso", G, 0)
    tal = [mesh(x=np.linspace(0.0, L, 11), y=np.linspace(0.0, L, 11))]
    return problem(name, G, log_speeds(G), mats, surfs, cells, src, tal)


def _small_lattice(seed, G, name):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    mats = config3_materials(int(rng.integers(0, 2**31)), G)
    p = lattice_problem(n=n, G=G, seed=int(rng.integers(0, 2**31)), mesh_n=2 * n, n_tbins=10,
                        mats=mats, name=name)
    return p


def exponential_ww(prob, decay, nx=None, ref=1.0, t_edges=None, t_decay=0.0):
    """Weight-window centres w_c = ref * exp(-decay * x) on an x-mesh (edges from the problem's
    second tally, or nx equal bins over the slab), all groups alike: a fixed, seeded-free input.
    With time edges, time bin i takes w_c * exp(-t_decay * i) (center [nt][nx][G])."""
    if nx is None:
        xe = np.asarray(prob["tallies"][1]["x"], dtype=np.float64)
    else:
        L = prob["surfaces"][-1]["coef"][0]
        xe = np.linspace(0.0, L, nx + 1)
    xc = 0.5 * (xe[:-1] + xe[1:])
    G = prob["G"]
    centre = np.repeat((ref * np.exp(-decay * xc))[:, None], G, axis=1)  # [nx][G]
    ww = {"x": xe.tolist(), "y": [-INF, INF], "z": [-INF, INF]}
    if t_edges is None:
        ww["center"] = centre.tolist()
        return ww
    nt = len(t_edges) - 1
    ww["t"] = [float(v) for v in t_edges]
    ww["center"] = (np.exp(-t_decay * np.arange(nt))[:, None, None] * centre[None]).tolist()  # [nt][nx][G]
    return ww


def bf16_round(a):
    """Round to the nearest bfloat16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_init(seed=7, H=64, n_in=5, bf16=True):
    """Seeded Xavier-uniform initial parameters of the 5 -> H -> H -> H -> 1 importance network in
    the order W1, b1, W2, b2, W3, b3, W4, b4 (biases zero); optionally rounded to bfloat16 so that
    a BF16 copy of them is exact."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((n_in, H), (H, H), (H, H), (H, 1)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts)
    return bf16_round(p) if bf16 else p


def by_name(name, **kw):
    return {"config1": config1, "config2": config2, "config3": config3,
            "config4": config4}[name](**kw)
