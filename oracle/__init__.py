"""Python wrapper of the CPU oracle (plain C++17, FP64, history-based).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py`.  The product path never imports this package.

`run(problem, n, seed, ...)` takes a problem dict as written by the seeded generators and returns
per-bin means and standard errors computed from the exact per-history variance.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_HS = 16
NCOUNT = 16
COUNTER_NAMES = ["source", "secondary", "capture", "production", "leak", "census", "lost",
                 "flight", "collision", "scatter", "surface", "reflect", "ww_split", "ww_kill",
                 "pc_banked", "pc_copies"]
KIND = {"PX": 0, "PY": 1, "PZ": 2, "CZ": 3, "CX": 4, "CY": 5, "SQ": 6, "GQ": 7}
BC = {"interior": 0, "vacuum": 1, "reflect": 2}
SRC_POS = {"box": 0, "surface_x0": 1}
SRC_DIR = {"iso": 0, "beam_x": 1, "cos_x": 2}
ESTIMATOR = {"track": 0, "crossing": 1}


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (portable flags only: the same source builds on x86 and Arm)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                               os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


class OrProblem(C.Structure):
    _fields_ = [
        ("G", C.c_int), ("M", C.c_int),
        ("sigma_t", C.POINTER(C.c_double)), ("sigma_s", C.POINTER(C.c_double)),
        ("sigma_f", C.POINTER(C.c_double)), ("nu", C.POINTER(C.c_double)),
        ("chi", C.POINTER(C.c_double)), ("speed", C.POINTER(C.c_double)),
        ("n_surf", C.c_int), ("surf_kind", C.POINTER(C.c_int)),
        ("surf_coef", C.POINTER(C.c_double)), ("surf_bc", C.POINTER(C.c_int)),
        ("n_cell", C.c_int), ("cell_nhs", C.POINTER(C.c_int)),
        ("cell_hs_surf", C.POINTER(C.c_int)), ("cell_hs_sense", C.POINTER(C.c_int)),
        ("cell_mat", C.POINTER(C.c_int)),
        ("has_lattice", C.c_int), ("lat_nx", C.c_int), ("lat_ny", C.c_int),
        ("lat_x0", C.c_double), ("lat_y0", C.c_double), ("lat_pitch", C.c_double),
        ("lat_r", C.c_double), ("lat_pin_mat", C.POINTER(C.c_int)), ("lat_matrix", C.c_int),
        ("lat_nz", C.c_int), ("lat_z0", C.c_double), ("lat_pitch_z", C.c_double),
        ("src_pos", C.c_int), ("src_dir", C.c_int),
        ("src_lo", C.c_double * 3), ("src_hi", C.c_double * 3),
        ("src_group_pdf", C.POINTER(C.c_double)), ("src_t0", C.c_double), ("src_t1", C.c_double),
        ("n_tally", C.c_int), ("tally_dims", C.POINTER(C.c_int)),
        ("tally_edges", C.POINTER(C.c_double)), ("t_census", C.c_double),
        ("ww_on", C.c_int), ("ww_nx", C.c_int), ("ww_ny", C.c_int), ("ww_nz", C.c_int),
        ("ww_edges", C.POINTER(C.c_double)), ("ww_center", C.POINTER(C.c_double)),
        ("ww_upper", C.c_double), ("ww_lower", C.c_double), ("ww_split_max", C.c_int),
        ("tally_est", C.POINTER(C.c_int)),
        ("ww_nt", C.c_int), ("ww_tedges", C.POINTER(C.c_double)),
    ]


class OrEvent(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("root", C.c_uint64), ("k", C.c_uint32),
                ("kind", C.c_int32), ("outcome", C.c_int32), ("n_child", C.c_int32),
                ("cell", C.c_int32), ("elem", C.c_int32), ("in_pin", C.c_int32),
                ("g", C.c_int32),
                ("x", C.c_double), ("y", C.c_double), ("z", C.c_double),
                ("ux", C.c_double), ("uy", C.c_double), ("uz", C.c_double),
                ("t", C.c_double), ("w", C.c_double)]


class OrOpts(C.Structure):
    _fields_ = [("first_history", C.c_uint64), ("n_histories", C.c_uint64),
                ("seed", C.c_uint64), ("threads", C.c_int),
                ("log_first", C.c_uint64), ("log_count", C.c_uint64),
                ("log", C.POINTER(OrEvent)), ("log_cap", C.c_uint64),
                ("log_n", C.POINTER(C.c_uint64)), ("fixed_bits", C.c_int),
                ("implicit_capture", C.c_int), ("wr_cutoff", C.c_double), ("wr_survival", C.c_double)]


class OrEigenOpts(C.Structure):
    _fields_ = [("n_per_cycle", C.c_uint64), ("seed", C.c_uint64), ("n_inactive", C.c_int),
                ("n_active", C.c_int), ("threads", C.c_int), ("fixed_bits", C.c_int),
                ("log_first", C.c_uint64), ("log_count", C.c_uint64),
                ("log", C.POINTER(OrEvent)), ("log_cap", C.c_uint64),
                ("log_n", C.POINTER(C.c_uint64))]


class OrEigenResult(C.Structure):
    _fields_ = [("k_cycle", C.POINTER(C.c_double)), ("sites_cycle", C.POINTER(C.c_uint64)),
                ("tally_cycle", C.POINTER(C.c_double)), ("counters", C.c_int64 * NCOUNT)]


class OrPcOpts(C.Structure):
    _fields_ = [("n_histories", C.c_uint64), ("seed", C.c_uint64), ("n_batches", C.c_int),
                ("threads", C.c_int), ("n_census", C.c_int), ("census_times", C.POINTER(C.c_double)),
                ("log_first", C.c_uint64), ("log_count", C.c_uint64),
                ("log", C.POINTER(OrEvent)), ("log_cap", C.c_uint64),
                ("log_n", C.POINTER(C.c_uint64)), ("method", C.c_int)]


class OrPcResult(C.Structure):
    _fields_ = [("tally_batch", C.POINTER(C.c_double)), ("banked", C.POINTER(C.c_uint64)),
                ("counters", C.c_int64 * NCOUNT)]


class OrResult(C.Structure):
    _fields_ = [("s1", C.POINTER(C.c_double)), ("s2", C.POINTER(C.c_double)),
                ("fixed", C.POINTER(C.c_int64)), ("counters", C.c_int64 * NCOUNT)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_run.argtypes = [C.POINTER(OrProblem), C.POINTER(OrOpts), C.POINTER(OrResult)]
            L.or_run.restype = C.c_int
            L.or_run_eigen.argtypes = [C.POINTER(OrProblem), C.POINTER(OrEigenOpts),
                                       C.POINTER(OrEigenResult)]
            L.or_run_eigen.restype = C.c_int
            L.or_run_pc.argtypes = [C.POINTER(OrProblem), C.POINTER(OrPcOpts), C.POINTER(OrPcResult)]
            L.or_run_pc.restype = C.c_int
            L.or_total_bins.argtypes = [C.POINTER(OrProblem)]
            L.or_total_bins.restype = C.c_int
            L.or_philox.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32),
                                    C.POINTER(C.c_uint32)]
            L.or_u01.argtypes = [C.c_uint32, C.c_uint32]
            L.or_u01.restype = C.c_double
            L.or_dist_cylinder.argtypes = [C.c_double] * 7 + [C.c_int]
            L.or_dist_cylinder.restype = C.c_double
            L.or_dist_surface.argtypes = [C.POINTER(OrProblem), C.c_int] + [C.c_double] * 6 + [C.c_int]
            L.or_dist_surface.restype = C.c_double
            L.or_dist_plane.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
            L.or_dist_plane.restype = C.c_double
            L.or_source_sample.argtypes = [C.POINTER(OrProblem), C.c_uint64, C.c_uint64,
                                           C.POINTER(C.c_double), C.POINTER(C.c_int)]
            L.or_source_sample.restype = C.c_int
            L.or_find_cell.argtypes = [C.POINTER(OrProblem), C.c_double, C.c_double, C.c_double,
                                       C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
            L.or_find_cell.restype = C.c_int
            L.or_sample_scatter_group.argtypes = [C.POINTER(OrProblem), C.c_int, C.c_int,
                                                  C.c_double]
            L.or_sample_scatter_group.restype = C.c_int
            L.or_child_tag.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                       C.c_uint32]
            L.or_child_tag.restype = C.c_uint64
            L.or_mlp_param_count.argtypes = [C.c_int]
            L.or_mlp_param_count.restype = C.c_int
            L.or_mlp_loss_grad.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int,
                                           C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]
            L.or_mlp_loss_grad.restype = C.c_double
            _lib = L
    return _lib


def _dp(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


class Marshalled:
    """Keeps the numpy buffers alive as long as the ctypes struct that points at them."""

    def __init__(self, prob: dict, ww: dict | None = None):
        self.keep = []
        G = prob["G"]
        mats = prob["materials"]
        M = len(mats)
        s = OrProblem()
        s.G, s.M = G, M

        def dp(x):
            a, p = _dp(x)
            self.keep.append(a)
            return p

        def ip(x):
            a, p = _ip(x)
            self.keep.append(a)
            return p

        s.sigma_t = dp([m["sigma_t"] for m in mats])
        s.sigma_s = dp([m["sigma_s"] for m in mats])
        s.sigma_f = dp([m["sigma_f"] for m in mats])
        s.nu = dp([m["nu"] for m in mats])
        s.chi = dp([m["chi"] for m in mats])
        s.speed = dp(prob["speed"])
        surfs = prob["surfaces"]
        s.n_surf = len(surfs)
        s.surf_kind = ip([KIND[x["kind"]] for x in surfs])
        coef = np.zeros((len(surfs), 10))
        for i, x in enumerate(surfs):
            coef[i, : len(x["coef"])] = x["coef"]
        s.surf_coef = dp(coef)
        s.surf_bc = ip([BC[x["bc"]] for x in surfs])
        cells = prob["cells"]
        s.n_cell = len(cells)
        hs_s = np.zeros((len(cells), MAX_HS), np.int32)
        hs_n = np.zeros((len(cells), MAX_HS), np.int32)
        for i, c in enumerate(cells):
            for j, (sf, sn) in enumerate(c["halfspaces"]):
                hs_s[i, j], hs_n[i, j] = sf, sn
        s.cell_nhs = ip([len(c["halfspaces"]) for c in cells])
        s.cell_hs_surf = ip(hs_s)
        s.cell_hs_sense = ip(hs_n)
        s.cell_mat = ip([c["material"] for c in cells])
        lat = prob.get("lattice")
        if lat:
            s.has_lattice = 1
            s.lat_nx, s.lat_ny = lat["nx"], lat["ny"]
            s.lat_x0, s.lat_y0 = lat["x0"], lat["y0"]
            s.lat_pitch, s.lat_r = lat["pitch"], lat["radius"]
            s.lat_pin_mat = ip(lat["pin_material"])
            s.lat_matrix = lat["matrix_material"]
            s.lat_nz = lat.get("nz", 0)
            s.lat_z0, s.lat_pitch_z = lat.get("z0", 0.0), lat.get("pitch_z", 0.0)
        else:
            s.has_lattice = 0
            s.lat_pin_mat = ip([0])
        src = prob["source"]
        s.src_pos = SRC_POS[src["pos"]]
        s.src_dir = SRC_DIR[src["dir"]]
        for i in range(3):
            s.src_lo[i] = src["lo"][i]
            s.src_hi[i] = src["hi"][i]
        s.src_group_pdf = dp(src["group_pdf"])
        s.src_t0, s.src_t1 = src["t0"], src["t1"]
        tals = prob["tallies"]
        s.n_tally = len(tals)
        dims, edges = [], []
        self.tally_shapes = []
        est = []
        for t in tals:
            n = [len(t[k]) - 1 for k in ("x", "y", "z", "t")]
            dims += n
            for k in ("x", "y", "z", "t"):
                edges += list(t[k])
            est.append(ESTIMATOR[t.get("estimator", "track")])
            # a time-crossing tally holds one value per time point (nt + 1 of them)
            self.tally_shapes.append((n[2], n[1], n[0], G, n[3] + (1 if est[-1] == 1 else 0)))
        s.tally_dims = ip(dims)
        s.tally_est = ip(est if est else [0])
        s.tally_edges = dp(edges if edges else [0.0])
        s.t_census = prob["t_census"]
        if ww is not None:
            s.ww_on = 1
            s.ww_nx, s.ww_ny, s.ww_nz = (len(ww[k]) - 1 for k in ("x", "y", "z"))
            s.ww_edges = dp(list(ww["x"]) + list(ww["y"]) + list(ww["z"]))
            s.ww_center = dp(ww["center"])
            if "t" in ww:
                s.ww_nt = len(ww["t"]) - 1
                s.ww_tedges = dp(list(ww["t"]))
            s.ww_upper = ww.get("upper", 2.0)
            s.ww_lower = ww.get("lower", 0.5)
            s.ww_split_max = ww.get("split_max", 10)
        else:
            s.ww_on = 0
            s.ww_edges = dp([0.0])
            s.ww_center = dp([0.0])
        self.s = s
        self.n_surf = len(surfs)


class Result:
    def __init__(self, shapes, n, s1, s2, fixed, counters, n_surf, events=None):
        self.n = n
        self.counters = dict(zip(COUNTER_NAMES, [int(c) for c in counters]))
        self.s1, self.s2, self.fixed = s1, s2, fixed
        self.events = events
        mean = s1 / n
        var = np.maximum(s2 / n - mean * mean, 0.0) / max(n - 1, 1)
        self.mean_flat, self.std_flat = mean, np.sqrt(var)
        self.tallies = []
        off = 0
        for shp in shapes:
            size = int(np.prod(shp))
            self.tallies.append((mean[off:off + size].reshape(shp),
                                 np.sqrt(var[off:off + size]).reshape(shp)))
            off += size
        self.leak_mean = mean[off:off + n_surf]
        self.leak_std = np.sqrt(var[off:off + n_surf])
        self.fixed_tallies = fixed


def run(prob: dict, n: int, seed: int = 1, threads: int | None = None, first: int = 0,
        log_first: int = 0, log_count: int = 0, log_cap: int = 0, ww: dict | None = None,
        fixed_bits: int = 32, implicit_capture: bool = False, wr_cutoff: float = 0.25,
        wr_survival: float = 0.5) -> Result:
    """Runs histories [first, first + n) of the problem; implicit_capture selects the collision
    without a capture channel (weight times the non-capture probability) and the weight-cutoff
    roulette below wr_cutoff (survivors get wr_survival)."""
    L = lib()
    m = Marshalled(prob, ww)
    nb = L.or_total_bins(C.byref(m.s))
    s1 = np.zeros(nb)
    s2 = np.zeros(nb)
    fx = np.zeros(nb, np.int64)
    res = OrResult()
    res.s1 = s1.ctypes.data_as(C.POINTER(C.c_double))
    res.s2 = s2.ctypes.data_as(C.POINTER(C.c_double))
    res.fixed = fx.ctypes.data_as(C.POINTER(C.c_int64))
    o = OrOpts()
    o.first_history, o.n_histories, o.seed = first, n, seed
    o.threads = threads if threads else (os.cpu_count() or 1)
    o.fixed_bits = fixed_bits
    o.implicit_capture = 1 if implicit_capture else 0
    o.wr_cutoff, o.wr_survival = wr_cutoff, wr_survival
    events = None
    log_n = C.c_uint64(0)
    if log_count > 0:
        cap = log_cap if log_cap else 64 * log_count
        events = (OrEvent * cap)()
        o.log = events
        o.log_cap = cap
        o.log_first, o.log_count = log_first, log_count
        o.log_n = C.pointer(log_n)
    rc = L.or_run(C.byref(m.s), C.byref(o), C.byref(res))
    if rc != 0:
        raise RuntimeError(f"or_run failed: {rc}")
    ev = None
    if events is not None:
        ev = events_to_numpy(events, int(log_n.value))
    return Result(m.tally_shapes, n, s1, s2, fx, list(res.counters), m.n_surf, ev)


class EigenResult:
    """k of every cycle, the mean and standard error of k over the active cycles, sites banked per
    cycle, and every tally's mean and standard error over the active cycles (each active cycle one
    batch, as the paper's cycle statistics)."""

    def __init__(self, shapes, n_surf, k, sites, tc, n_inactive, counters, events):
        self.k_cycle, self.sites_cycle = k, sites
        ka = k[n_inactive:]
        self.k_mean = float(ka.mean())
        self.k_std = float(ka.std(ddof=1) / math.sqrt(len(ka)))
        self.counters = dict(zip(COUNTER_NAMES, [int(c) for c in counters]))
        self.events = events
        self.cycle_tallies = tc
        mean = tc.mean(axis=0)
        std = tc.std(axis=0, ddof=1) / math.sqrt(tc.shape[0])
        self.tallies = []
        off = 0
        for shp in shapes:
            size = int(np.prod(shp))
            self.tallies.append((mean[off:off + size].reshape(shp), std[off:off + size].reshape(shp)))
            off += size
        self.leak_mean, self.leak_std = mean[off:off + n_surf], std[off:off + n_surf]


def run_eigen(prob: dict, n: int, n_inactive: int, n_active: int, seed: int = 1,
              threads: int | None = None, log_first: int = 0, log_count: int = 0,
              log_cap: int = 0) -> EigenResult:
    """k-eigenvalue power iteration of the oracle (see or_run_eigen in oracle.h)."""
    L = lib()
    m = Marshalled(prob)
    nb = L.or_total_bins(C.byref(m.s))
    nc = n_inactive + n_active
    k = np.zeros(nc)
    sites = np.zeros(nc, np.uint64)
    tc = np.zeros((max(1, n_active), nb))
    o = OrEigenOpts()
    o.n_per_cycle, o.seed, o.n_inactive, o.n_active = n, seed, n_inactive, n_active
    o.threads = threads if threads else (os.cpu_count() or 1)
    o.fixed_bits = 32
    events, log_n = None, C.c_uint64(0)
    if log_count > 0:
        cap = log_cap if log_cap else 64 * log_count * nc
        events = (OrEvent * cap)()
        o.log, o.log_cap, o.log_first, o.log_count = events, cap, log_first, log_count
        o.log_n = C.pointer(log_n)
    r = OrEigenResult()
    r.k_cycle = k.ctypes.data_as(C.POINTER(C.c_double))
    r.sites_cycle = sites.ctypes.data_as(C.POINTER(C.c_uint64))
    r.tally_cycle = tc.ctypes.data_as(C.POINTER(C.c_double))
    rc = L.or_run_eigen(C.byref(m.s), C.byref(o), C.byref(r))
    if rc != 0:
        raise RuntimeError(f"or_run_eigen failed: {rc}")
    ev = events_to_numpy(events, int(log_n.value)) if events is not None else None
    return EigenResult(m.tally_shapes, m.n_surf, k, sites, tc[:n_active], n_inactive, list(r.counters), ev)


class BatchResult:
    """Mean and standard error of every tally over independent batches (per source particle)."""

    def __init__(self, shapes, n_surf, tb, counters, banked, events):
        self.batch_tallies = tb
        self.counters = dict(zip(COUNTER_NAMES, [int(c) for c in counters]))
        self.banked = banked
        self.events = events
        mean = tb.mean(axis=0)
        std = tb.std(axis=0, ddof=1) / math.sqrt(tb.shape[0])
        self.tallies = []
        off = 0
        for shp in shapes:
            size = int(np.prod(shp))
            self.tallies.append((mean[off:off + size].reshape(shp), std[off:off + size].reshape(shp)))
            off += size
        self.leak_mean, self.leak_std = mean[off:off + n_surf], std[off:off + n_surf]


def run_pc(prob: dict, n: int, census_times, n_batches: int = 32, seed: int = 1,
           threads: int | None = None, log_first: int = 0, log_count: int = 0,
           log_cap: int = 0, method: str = "split") -> BatchResult:
    """Time-dependent run with population control at the interior census times (see or_run_pc in
    oracle.h): splitting-roulette ("split") or combing ("comb"); statistics over the independent
    batches."""
    L = lib()
    m = Marshalled(prob)
    nb = L.or_total_bins(C.byref(m.s))
    ct = np.ascontiguousarray(census_times, dtype=np.float64)
    tb = np.zeros((n_batches, nb))
    banked = np.zeros(max(1, ct.size), np.uint64)
    o = OrPcOpts()
    o.n_histories, o.seed, o.n_batches = n, seed, n_batches
    o.threads = threads if threads else (os.cpu_count() or 1)
    o.n_census = ct.size
    o.census_times = ct.ctypes.data_as(C.POINTER(C.c_double))
    o.method = {"split": 0, "comb": 1}[method]
    events, log_n = None, C.c_uint64(0)
    if log_count > 0:
        cap = log_cap if log_cap else 256 * log_count
        events = (OrEvent * cap)()
        o.log, o.log_cap, o.log_first, o.log_count = events, cap, log_first, log_count
        o.log_n = C.pointer(log_n)
    r = OrPcResult()
    r.tally_batch = tb.ctypes.data_as(C.POINTER(C.c_double))
    r.banked = banked.ctypes.data_as(C.POINTER(C.c_uint64))
    rc = L.or_run_pc(C.byref(m.s), C.byref(o), C.byref(r))
    if rc != 0:
        raise RuntimeError(f"or_run_pc failed: {rc}")
    ev = events_to_numpy(events, int(log_n.value)) if events is not None else None
    return BatchResult(m.tally_shapes, m.n_surf, tb, list(r.counters), banked[:ct.size], ev)


EVENT_DTYPE = np.dtype([("tag", np.uint64), ("root", np.uint64), ("k", np.uint32),
                        ("kind", np.int32), ("outcome", np.int32), ("n_child", np.int32),
                        ("cell", np.int32), ("elem", np.int32), ("in_pin", np.int32),
                        ("g", np.int32), ("x", np.float64), ("y", np.float64),
                        ("z", np.float64), ("ux", np.float64), ("uy", np.float64),
                        ("uz", np.float64), ("t", np.float64), ("w", np.float64)], align=True)


def events_to_numpy(events, n):
    assert C.sizeof(OrEvent) == EVENT_DTYPE.itemsize
    buf = np.frombuffer(events, dtype=EVENT_DTYPE, count=len(events))[:n].copy()
    order = np.lexsort((buf["k"], buf["tag"]))
    return buf[order]


# ----------------------------------------------------------------------------- unit helpers


def philox(key, ctr):
    L = lib()
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    out = (C.c_uint32 * 4)()
    L.or_philox(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF, c, out)
    return [int(v) for v in out]


def comb_counts(weights, n_teeth: int, xi: float):
    """Copies the population-control comb gives each weight of the list, in its order."""
    L = lib()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    out = np.zeros(w.size, np.int64)
    L.or_comb_counts(w.ctypes.data_as(C.POINTER(C.c_double)), C.c_int64(w.size), C.c_uint64(n_teeth),
                     C.c_double(xi), out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def u01(a, b):
    return lib().or_u01(a, b)


def dist_cylinder(x, y, ux, uy, x0, y0, r, inside):
    return lib().or_dist_cylinder(x, y, ux, uy, x0, y0, r, int(inside))


def dist_surface(prob, s, pos, u, sense):
    """Distance to surface s of the problem at which a particle at pos moving along u leaves its
    half-space `sense`."""
    m = Marshalled(prob)
    return lib().or_dist_surface(C.byref(m.s), s, *[float(v) for v in pos], *[float(v) for v in u], sense)


def dist_plane(pos, u, c, sense):
    return lib().or_dist_plane(pos, u, c, sense)


def source_sample(prob, seed, h):
    m = Marshalled(prob)
    out = (C.c_double * 7)()
    g = C.c_int(0)
    cell = lib().or_source_sample(C.byref(m.s), seed, h, out, C.byref(g))
    return list(out), int(g.value), cell


def find_cell(prob, x, y, z, skip=-1, skip_sense=0, u=(0.0, 0.0, 0.0)):
    """Cell of a point; skip/skip_sense: the surface just crossed and the sense taken on it;
    u: the direction of flight."""
    m = Marshalled(prob)
    return int(lib().or_find_cell(C.byref(m.s), x, y, z, skip, skip_sense, *[float(v) for v in u]))


def sample_scatter_group(prob, m, g, u):
    mm = Marshalled(prob)
    return lib().or_sample_scatter_group(C.byref(mm.s), m, g, u)


def child_tag(seed, parent, k, j, marker=0x80000000):
    return int(lib().or_child_tag(seed, parent, k, j, marker))


def mlp_param_count(H=64):
    return lib().or_mlp_param_count(H)


def mlp_loss_grad(params, x, target=None, wt=None, H=64):
    """FP64 reference MLP (tanh hidden layers): returns (loss, y, grad)."""
    L = lib()
    x = np.ascontiguousarray(x, np.float64)
    n = x.shape[0]
    p = np.ascontiguousarray(params, np.float64)
    y = np.zeros(n)
    grad = np.zeros(p.size)
    tp = None if target is None else np.ascontiguousarray(target, np.float64)
    wp = None if wt is None else np.ascontiguousarray(wt, np.float64)
    dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None
    loss = L.or_mlp_loss_grad(H, dptr(p), n, dptr(x), dptr(tp), dptr(wp), dptr(y),
                              dptr(grad) if tp is not None else None)
    return loss, y, grad


def relative_error(mean, std):
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(mean != 0, std / np.abs(mean), math.inf)
