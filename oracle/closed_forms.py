"""Closed-form and numerically exact solutions that pin the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Each function states the mathematics it
evaluates; none of them runs the random walk.

Units: cross sections 1/cm, lengths cm, speeds cm/s.  All track-length quantities are per source
particle: a mesh bin's value is the expected total track length (weight x cm) in that bin, i.e.
the space-time integral of the scalar flux over the bin.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, linalg
from scipy.special import expn

# ------------------------------------------------------------------ P1: beam transmission


def beam_transmission(sigma_t: float, L: float) -> float:
    """Normally incident beam on a pure absorber: uncollided transmission e^{-Sigma_t L}."""
    return math.exp(-sigma_t * L)


def beam_flux_bins(sigma_t: float, edges) -> np.ndarray:
    """Track length per source particle of a mu=1 beam in [a, b]: (e^{-St a} - e^{-St b})/St."""
    e = np.asarray(edges, dtype=np.float64)
    return (np.exp(-sigma_t * e[:-1]) - np.exp(-sigma_t * e[1:])) / sigma_t


# ------------------------------------------------------------------ P2: isotropic slab source


def slab_leakage(sigma_t: float, L: float, a: float = 1.0):
    """Pure absorber 0<x<L, isotropic source uniform on [0, a) (one particle in total).

    A particle born at depth d from a face escapes through it uncollided with probability
    E_2(St d)/2.  Averaging over the source and using d/du E_3(u) = -E_2(u):
        P_right = [E_3(St (L-a)) - E_3(St L)] / (2 St a)
        P_left  = [E_3(0) - E_3(St a)] / (2 St a),   E_3(0) = 1/2.
    """
    pr = (expn(3, sigma_t * (L - a)) - expn(3, sigma_t * L)) / (2.0 * sigma_t * a)
    pl = (0.5 - expn(3, sigma_t * a)) / (2.0 * sigma_t * a)
    return pl, pr


def _phi2(u, sigma_t):
    """Even second antiderivative of K(|u|) = E_1(St |u|) with Phi(0) = Phi'(0) = 0:
    Phi(u) = |u|/St - (1/2 - E_3(St |u|)) / St^2."""
    u = np.abs(np.asarray(u, dtype=np.float64))
    return u / sigma_t - (0.5 - expn(3, sigma_t * u)) / sigma_t**2


def slab_flux_bins(sigma_t: float, edges, a: float = 1.0) -> np.ndarray:
    """Track length per source particle in x-bins of the pure-absorber slab with an isotropic
    source uniform on [0, a): phi(x) = (1/a) int_0^a E_1(St |x - x'|)/2 dx', integrated over each
    bin by the double antiderivative:
        int_xa^xb int_0^a K = Phi(xb) - Phi(xa) - Phi(xb - a) + Phi(xa - a)."""
    e = np.asarray(edges, dtype=np.float64)
    xa, xb = e[:-1], e[1:]
    val = _phi2(xb, sigma_t) - _phi2(xa, sigma_t) - _phi2(xb - a, sigma_t) + _phi2(xa - a, sigma_t)
    return 0.5 * val / a


def slab_flux_bins_quad(sigma_t: float, edges, a: float = 1.0) -> np.ndarray:
    """The same bin integrals by adaptive quadrature of phi(x) (independent check of the
    antiderivative algebra).  The inner integral uses int E_1 = -E_2/St."""
    def phi(x):
        lo, hi = x - a, x  # x - x' ranges over [x-a, x]
        def F(u):  # int_0^u E_1(St s) ds for u >= 0
            return (1.0 - expn(2, sigma_t * u)) / sigma_t
        if lo >= 0.0:
            inner = F(hi) - F(lo)
        elif hi <= 0.0:
            inner = F(-lo) - F(-hi)
        else:
            inner = F(hi) + F(-lo)
        return 0.5 * inner / a
    e = np.asarray(edges, dtype=np.float64)
    out = []
    for xa, xb in zip(e[:-1], e[1:]):
        pts = [p for p in (0.0, a) if xa < p < xb]
        v, _ = integrate.quad(phi, xa, xb, points=pts or None, epsabs=1e-13, epsrel=1e-10,
                              limit=200)
        out.append(v)
    return np.array(out)


# ------------------------------------------------------------------ P3 / P4: infinite medium, 1 group


def infinite_total_tracklength(sigma_t, sigma_s, nu_sigma_f=0.0):
    """Steady infinite medium: each unit of track length is removed at rate Sigma_a = St - Ss
    and replaced at rate nu Sf, so the expected total track length per source is
    1 / (St - Ss - nu Sf) for a subcritical medium."""
    return 1.0 / (sigma_t - sigma_s - nu_sigma_f)


def infinite_time_bins(sigma_t, sigma_s, nu_sigma_f, v, t_edges):
    """Time-dependent one-group infinite medium, pulse at t = 0:
    phi(t) = v exp(-alpha t), alpha = v (St - Ss - nu Sf);
    int_ta^tb phi dt = (e^{-alpha ta} - e^{-alpha tb}) / (St - Ss - nu Sf).  For a supercritical
    medium (alpha < 0) the same formula holds."""
    e = np.asarray(t_edges, dtype=np.float64)
    sa = sigma_t - sigma_s - nu_sigma_f
    alpha = v * sa
    if sa == 0.0:
        return v * (e[1:] - e[:-1])
    return (np.exp(-alpha * e[:-1]) - np.exp(-alpha * e[1:])) / sa


def infinite_population(sigma_t, sigma_s, nu_sigma_f, v, t):
    """Expected number of particles alive at time t per source particle: exp(-alpha t)."""
    return math.exp(-v * (sigma_t - sigma_s - nu_sigma_f) * t)


def infinite_point_flux(sigma_t, sigma_s, nu_sigma_f, v, t_points):
    """One-group infinite medium after a unit pulse at t = 0: the flux at the instants t,
    phi(t) = v exp(-alpha t) (what the time-crossing estimator measures)."""
    t = np.asarray(t_points, dtype=np.float64)
    return v * np.exp(-v * (sigma_t - sigma_s - nu_sigma_f) * t)


# ------------------------------------------------------------------ P5: multigroup expm


def multigroup_operator(mat, speed):
    """A = V M with M = S^T + chi (nu Sf)^T - diag(St), V = diag(v): d phi/dt = A phi for the
    volume-integrated group flux phi_g = v_g N_g of an infinite medium."""
    st = np.asarray(mat["sigma_t"], dtype=np.float64)
    S = np.asarray(mat["sigma_s"], dtype=np.float64)
    nsf = np.asarray(mat["nu"], dtype=np.float64) * np.asarray(mat["sigma_f"], dtype=np.float64)
    chi = np.asarray(mat["chi"], dtype=np.float64)
    M = S.T + np.outer(chi, nsf) - np.diag(st)
    return np.diag(np.asarray(speed, dtype=np.float64)) @ M


def integrated_flux_vanloan(A, phi0, t):
    """int_0^t exp(A s) phi0 ds from the block exponential of Van Loan (1978):
    exp([[A, I], [0, 0]] t) = [[e^{At}, int_0^t e^{As} ds], [0, I]]  (scipy's expm does scaling
    and squaring with Pade approximants, Higham 2005)."""
    G = A.shape[0]
    B = np.zeros((2 * G, 2 * G))
    B[:G, :G] = A * t
    B[:G, G:] = np.eye(G) * t
    E = linalg.expm(B)
    return E[:G, G:] @ phi0


def integrated_flux_eig(A, phi0, t):
    """Same integral via the eigendecomposition A = W diag(lam) W^-1:
    int_0^t e^{As} ds = W diag((e^{lam t} - 1)/lam) W^-1."""
    lam, W = np.linalg.eig(A)
    f = np.where(np.abs(lam * t) > 1e-12, np.expm1(lam * t) / np.where(lam == 0, 1, lam), t)
    return np.real(W @ (f * np.linalg.solve(W, phi0.astype(complex))))


def multigroup_time_bins(mat, speed, t_edges, g0=0, method="vanloan"):
    """Per (group, time bin) track length of an infinite medium after a unit pulse in group g0
    at t = 0: phi(0) = v_g0 e_g0, bins = differences of int_0^t phi."""
    A = multigroup_operator(mat, speed)
    G = A.shape[0]
    phi0 = np.zeros(G)
    phi0[g0] = speed[g0]
    f = integrated_flux_vanloan if method == "vanloan" else integrated_flux_eig
    cum = np.array([f(A, phi0, t) if t > 0 else np.zeros(G) for t in t_edges])
    return (cum[1:] - cum[:-1]).T  # [G][nt]


def multigroup_point_flux(mat, speed, t_points, g0=0, method="expm"):
    """Group flux of an infinite medium at the instants t after a unit pulse in group g0:
    phi(t) = exp(A t) phi(0), phi(0) = v_g0 e_g0 -> [G][n_points].  method 'expm': scipy's
    scaling and squaring (Higham 2005); 'eig': the eigendecomposition of A."""
    A = multigroup_operator(mat, speed)
    G = A.shape[0]
    phi0 = np.zeros(G)
    phi0[g0] = speed[g0]
    out = []
    if method == "expm":
        for t in t_points:
            out.append(linalg.expm(A * t) @ phi0)
    else:
        lam, W = np.linalg.eig(A)
        c = np.linalg.solve(W, phi0.astype(complex))
        for t in t_points:
            out.append(np.real(W @ (np.exp(lam * t) * c)))
    return np.array(out).T


def multigroup_time_bins_ode(mat, speed, t_edges, g0=0, rtol=1e-12):
    """Third, independent route: integrate d/dt [phi, Phi] = [A phi, phi] with Radau."""
    A = multigroup_operator(mat, speed)
    G = A.shape[0]
    y0 = np.zeros(2 * G)
    y0[g0] = speed[g0]
    te = np.asarray(t_edges, dtype=np.float64)

    def rhs(t, y):
        return np.concatenate([A @ y[:G], y[:G]])

    def jac(t, y):
        J = np.zeros((2 * G, 2 * G))
        J[:G, :G] = A
        J[G:, :G] = np.eye(G)
        return J

    sol = integrate.solve_ivp(rhs, (0.0, te[-1]), y0, method="Radau", t_eval=te, rtol=rtol,
                              atol=1e-30, jac=jac)
    cum = sol.y[G:].T
    return (cum[1:] - cum[:-1]).T


# ------------------------------------------------------------------ isotropic-flux surface crossings


def isotropic_crossings(track_density: float, area: float) -> float:
    """Expected number of crossings (both directions) of a surface of the given area by a
    uniform isotropic flux of scalar value `track_density` (track length per unit volume):
    each one-way partial current is phi/4, so crossings = phi/2 per unit area."""
    return 0.5 * track_density * area


# ------------------------------------------------------------------ k-eigenvalue, infinite medium


def infinite_k(mat):
    """k of an infinite homogeneous medium and its fundamental group spectrum: the dominant
    eigenpair of A^-1 F with the removal operator A = diag(Sigma_t) - S^T (S from -> to) and the
    production operator F = chi (nu Sigma_f)^T.  Returns (k, phi) with phi >= 0 summing to 1 (the
    volume-integrated group flux shape)."""
    st = np.asarray(mat["sigma_t"], dtype=np.float64)
    S = np.asarray(mat["sigma_s"], dtype=np.float64)
    nsf = np.asarray(mat["nu"], dtype=np.float64) * np.asarray(mat["sigma_f"], dtype=np.float64)
    chi = np.asarray(mat["chi"], dtype=np.float64)
    A = np.diag(st) - S.T
    F = np.outer(chi, nsf)
    lam, V = np.linalg.eig(np.linalg.solve(A, F))
    i = int(np.argmax(lam.real))
    phi = np.abs(V[:, i].real)
    return float(lam[i].real), phi / phi.sum()


# ------------------------------------------------------------------ quadric bodies: point-source escape


def sphere_point_escape(sigma_t, R, s):
    """Escape probability of an isotropic point source at distance s from the centre of a purely
    absorbing sphere of radius R: the average over directions of exp(-Sigma_t d), d the distance to
    the surface along the direction, d(mu) = -s mu + sqrt(R^2 - s^2 (1 - mu^2))."""
    f = lambda mu: math.exp(-sigma_t * (-s * mu + math.sqrt(R * R - s * s * (1.0 - mu * mu))))
    return 0.5 * integrate.quad(f, -1.0, 1.0, epsabs=1e-13, epsrel=1e-12)[0]


def cylinder_point_escape(sigma_t, R, L):
    """Escape probability from the centre of a purely absorbing finite cylinder (radius R, length 2L):
    with mu = |cos| of the angle to the axis, uniform on [0, 1] for an isotropic source, the distance
    is min(L / mu, R / sqrt(1 - mu^2))."""
    def f(mu):
        d = min(L / mu if mu > 0 else math.inf, R / math.sqrt(1 - mu * mu) if mu < 1 else math.inf)
        return math.exp(-sigma_t * d)
    mu_c = L / math.sqrt(L * L + R * R)  # where the two distances meet
    return (integrate.quad(f, 0.0, mu_c, epsabs=1e-13, epsrel=1e-12)[0]
            + integrate.quad(f, mu_c, 1.0, epsabs=1e-13, epsrel=1e-12)[0])


def ellipsoid_point_escape(sigma_t, a, b, c):
    """Escape probability from the centre of a purely absorbing ellipsoid with semi-axes a, b, c:
    d(u) = 1 / sqrt(ux^2/a^2 + uy^2/b^2 + uz^2/c^2), averaged over the sphere of directions."""
    def f(phi, mu):
        s = math.sqrt(1 - mu * mu)
        ux, uy = s * math.cos(phi), s * math.sin(phi)
        d = 1.0 / math.sqrt(ux * ux / a**2 + uy * uy / b**2 + mu * mu / c**2)
        return math.exp(-sigma_t * d)
    return integrate.dblquad(f, -1.0, 1.0, 0.0, 2 * math.pi, epsabs=1e-11, epsrel=1e-10)[0] / (4 * math.pi)


def quadric_body_point_escape(sigma_t, Q, c0, p0):
    """Escape probability of an isotropic point source at p0 inside the purely absorbing body
    (p - c0)^T Q (p - c0) < 1 (Q symmetric positive definite): along u the distance t solves
    t^2 u.Qu + 2 t u.Q(p0 - c0) + (p0 - c0).Q(p0 - c0) - 1 = 0 (the positive root), averaged over the
    sphere of directions by 2-D quadrature.  Written from the matrix form, independently of any
    expansion into the ten coefficients of a general quadric."""
    Q = np.asarray(Q, dtype=np.float64)
    w = np.asarray(p0, dtype=np.float64) - np.asarray(c0, dtype=np.float64)
    cw = float(w @ Q @ w) - 1.0

    def f(phi, mu):
        s = math.sqrt(1 - mu * mu)
        u = np.array([s * math.cos(phi), s * math.sin(phi), mu])
        a, b = float(u @ Q @ u), float(u @ Q @ w)
        t = (-b + math.sqrt(b * b - a * cw)) / a
        return math.exp(-sigma_t * t)
    return integrate.dblquad(f, -1.0, 1.0, 0.0, 2 * math.pi, epsabs=1e-11, epsrel=1e-10)[0] / (4 * math.pi)


def lattice_point_escape(prob, n_dir=20000, h=0.004, seed=0):
    """Escape probability of an isotropic point source in a purely absorbing one-group problem made
    of one box cell filled by a (3D) pin lattice, vacuum outside: the average over directions of
    exp(-tau), tau the optical depth from the source point to the box wall.  tau is integrated along
    each ray by a Riemann sum with step h and a uniformly random offset (an unbiased estimate of the
    integral), the material at each sample found by point location alone: the element by floor
    division, the pin by the distance to its axis.  Directions: a Fibonacci lattice on the sphere.
    Shares nothing with the tracking (no distances to walls, no stored element indices)."""
    lat = prob["lattice"]
    nx, ny = lat["nx"], lat["ny"]
    nz = max(1, lat.get("nz", 0))
    p, r = lat["pitch"], lat["radius"]
    x0, y0 = lat["x0"], lat["y0"]
    z0, pz = lat.get("z0", 0.0), lat.get("pitch_z", 1.0)
    pins = np.asarray(lat["pin_material"]).reshape(nz, ny, nx)
    sig = np.array([m["sigma_t"][0] for m in prob["materials"]])
    lo = np.array([x0, y0, z0])
    hi = np.array([x0 + nx * p, y0 + ny * p, z0 + nz * pz])
    p0 = np.asarray(prob["source"]["lo"], dtype=np.float64)
    i = np.arange(n_dir) + 0.5
    mu = 1.0 - 2.0 * i / n_dir
    phi = math.pi * (1.0 + math.sqrt(5.0)) * i
    s = np.sqrt(1.0 - mu * mu)
    u = np.stack([s * np.cos(phi), s * np.sin(phi), mu], axis=1)
    with np.errstate(divide="ignore"):
        t_hi = np.where(u > 0, (hi - p0) / u, np.where(u < 0, (lo - p0) / u, np.inf)).min(axis=1)
    rng = np.random.default_rng(seed)
    total = 0.0
    for a in range(0, n_dir, 512):
        uu, L = u[a:a + 512], t_hi[a:a + 512]
        m = int(np.ceil(L.max() / h)) + 1
        t = (np.arange(m)[None, :] + rng.uniform(size=(len(uu), 1))) * h  # [ray][sample]
        inside = t < L[:, None]
        q = p0[None, None, :] + t[:, :, None] * uu[:, None, :]
        ix = np.clip(np.floor((q[..., 0] - x0) / p).astype(int), 0, nx - 1)
        iy = np.clip(np.floor((q[..., 1] - y0) / p).astype(int), 0, ny - 1)
        iz = np.clip(np.floor((q[..., 2] - z0) / pz).astype(int), 0, nz - 1) if nz > 1 else 0 * ix
        pin = pins[iz, iy, ix]
        dx = q[..., 0] - (x0 + (ix + 0.5) * p)
        dy = q[..., 1] - (y0 + (iy + 0.5) * p)
        in_pin = (pin >= 0) & (dx * dx + dy * dy < r * r)
        mat = np.where(in_pin, pin, lat["matrix_material"])
        tau = (np.where(inside, sig[mat], 0.0)).sum(axis=1) * h
        total += np.exp(-tau).sum()
    return total / n_dir
