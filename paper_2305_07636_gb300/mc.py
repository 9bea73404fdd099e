"""Python binding of libmcgb (include/mc.h): argument marshalling only.

Every step of the random walk runs in the library's CUDA kernels; this module turns the problem
dicts of `problems.py` into `mc_problem_desc` structs, passes device pointers / stream handles
through, and converts status codes into exceptions.  There is no CPU fallback: if the library
cannot be loaded, or the GPU is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

# ------------------------------------------------------------------------------ constants (mc.h)
MC_OK, MC_ERR_INVALID, MC_ERR_CUDA, MC_ERR_OOM = 0, -1, -2, -3
MC_ERR_BANK_FULL, MC_ERR_TIMEOUT, MC_ERR_STATE, MC_ERR_LOST, MC_ERR_BOUNDS = -4, -5, -6, -7, -8
STATUS_NAMES = {0: "MC_OK", -1: "MC_ERR_INVALID", -2: "MC_ERR_CUDA", -3: "MC_ERR_OOM",
                -4: "MC_ERR_BANK_FULL", -5: "MC_ERR_TIMEOUT", -6: "MC_ERR_STATE",
                -7: "MC_ERR_LOST", -8: "MC_ERR_BOUNDS"}
MAX_HALFSPACES = 16
MAX_GROUPS, MAX_SURFACES, MAX_CELLS = 32, 255, 255  # MC_MAX_* of mc.h
MAX_LATTICE, MAX_LATTICE_ELEMENTS = 255, 65536
MC_FP32, MC_FP64 = 0, 1
MC_TALLY_FIXED64, MC_TALLY_FP64 = 0, 1
COUNTER_NAMES = ["source", "secondary", "capture", "production", "leak", "census", "lost",
                 "flight", "collision", "scatter", "surface", "reflect", "ww_split", "ww_kill",
                 "iterations", "scores", "ww_held", "pc_banked", "pc_copies"]
NCOUNTERS = len(COUNTER_NAMES)
KIND = {"PX": 0, "PY": 1, "PZ": 2, "CZ": 3, "CX": 4, "CY": 5, "SQ": 6, "GQ": 7}  # mc_surface_kind
BC = {"interior": 0, "vacuum": 1, "reflect": 2}
SRC_POS = {"box": 0, "surface_x0": 1}
SRC_DIR = {"iso": 0, "beam_x": 1, "cos_x": 2}


class McError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


# ------------------------------------------------------------------------------ structs (mc.h)
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int)


class mc_surface(C.Structure):
    _fields_ = [("kind", C.c_int), ("coef", C.c_double * 10), ("bc", C.c_int)]


class mc_cell(C.Structure):
    _fields_ = [("n_halfspaces", C.c_int), ("surface", C.c_int * MAX_HALFSPACES),
                ("sense", C.c_int * MAX_HALFSPACES), ("material", C.c_int)]


class mc_lattice(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("pitch", C.c_double), ("radius", C.c_double), ("pin_material", IP),
                ("matrix_material", C.c_int), ("nz", C.c_int), ("z0", C.c_double), ("pitch_z", C.c_double)]


class mc_source(C.Structure):
    _fields_ = [("pos", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("dir", C.c_int), ("group_pdf", DP), ("t0", C.c_double), ("t1", C.c_double)]


class mc_mesh_tally(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("nt", C.c_int),
                ("x", DP), ("y", DP), ("z", DP), ("t", DP), ("estimator", C.c_int)]


ESTIMATOR = {"track": 0, "crossing": 1}  # mc_estimator


class mc_problem_desc(C.Structure):
    _fields_ = [("n_groups", C.c_int), ("n_materials", C.c_int),
                ("sigma_t", DP), ("sigma_s", DP), ("sigma_f", DP), ("nu", DP), ("chi", DP),
                ("speed", DP), ("n_surfaces", C.c_int), ("surfaces", C.POINTER(mc_surface)),
                ("n_cells", C.c_int), ("cells", C.POINTER(mc_cell)),
                ("lattice", C.POINTER(mc_lattice)), ("source", mc_source),
                ("n_tallies", C.c_int), ("tallies", C.POINTER(mc_mesh_tally)),
                ("t_census", C.c_double)]


class mc_run_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tally_mode", C.c_int), ("fixed_bits", C.c_int),
                ("n_batches", C.c_int), ("bank_capacity", C.c_uint64),
                ("block_size", C.c_int), ("blocks_per_sm", C.c_int),
                ("max_iterations", C.c_uint64), ("aggregate_atomics", C.c_int),
                ("ww_enable", C.c_int), ("log_first", C.c_uint64), ("log_count", C.c_uint64),
                ("log_capacity", C.c_uint64), ("first_history", C.c_uint64),
                ("algorithm", C.c_int), ("drain_threshold", C.c_uint64),
                ("tally_stripes", C.c_int), ("batch_unit", C.c_int),
                ("implicit_capture", C.c_int), ("wr_cutoff", C.c_double), ("wr_survival", C.c_double),
                ("n_census", C.c_int), ("census_times", DP), ("pc_method", C.c_int)]


class mc_event(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("root", C.c_uint64), ("k", C.c_uint32),
                ("kind", C.c_int32), ("outcome", C.c_int32), ("n_child", C.c_int32),
                ("cell", C.c_int32), ("elem", C.c_int32), ("in_pin", C.c_int32),
                ("g", C.c_int32),
                ("x", C.c_double), ("y", C.c_double), ("z", C.c_double),
                ("ux", C.c_double), ("uy", C.c_double), ("uz", C.c_double),
                ("t", C.c_double), ("w", C.c_double)]


EVENT_DTYPE = np.dtype([("tag", np.uint64), ("root", np.uint64), ("k", np.uint32),
                        ("kind", np.int32), ("outcome", np.int32), ("n_child", np.int32),
                        ("cell", np.int32), ("elem", np.int32), ("in_pin", np.int32),
                        ("g", np.int32), ("x", np.float64), ("y", np.float64),
                        ("z", np.float64), ("ux", np.float64), ("uy", np.float64),
                        ("uz", np.float64), ("t", np.float64), ("w", np.float64)], align=True)

# every entry point declared in include/mc.h, with its ctypes signature
SIGNATURES = {
    "mc_run_opts_default": (None, [C.POINTER(mc_run_opts)]),
    "mc_problem_create": (C.c_int, [C.POINTER(mc_problem_desc), C.POINTER(C.c_void_p)]),
    "mc_run": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.POINTER(mc_run_opts), C.c_void_p]),
    "mc_run_eigen": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_int, C.c_uint64, C.POINTER(mc_run_opts),
                               C.c_void_p, DP, C.POINTER(C.c_uint64), DP, DP]),
    "mc_wait": (C.c_int, [C.c_void_p]),
    "mc_tally_shape": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64)]),
    "mc_tally_get": (C.c_int, [C.c_void_p, C.c_int, DP, DP, C.c_size_t]),
    "mc_counters_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_size_t]),
    "mc_tally_batches": (C.c_int, [C.c_void_p, C.c_int, DP, C.c_size_t, C.POINTER(C.c_int)]),
    "mc_event_log": (C.c_int, [C.c_void_p, C.POINTER(mc_event), C.c_size_t,
                               C.POINTER(C.c_size_t)]),
    "mc_run_timing": (C.c_int, [C.c_void_p, DP, DP]),
    "mc_run_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "mc_tally_layout": (C.c_int, [C.c_void_p, IP, IP, C.POINTER(C.c_uint64)]),
    "mc_tally_sums": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.c_size_t, IP]),
    "mc_trace_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                               C.POINTER(C.c_uint64), C.c_size_t, C.POINTER(C.c_size_t)]),
    "mc_problem_table_bytes": (C.c_size_t, [C.c_void_p]),
    "mc_problem_destroy": (None, [C.c_void_p]),
    "mc_last_error": (C.c_char_p, []),
    "mc_philox": (C.c_int, [C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]),
    "mc_atomic_peak": (C.c_int, [C.c_uint64, DP]),
    "mc_op_rates": (C.c_int, [DP, C.c_int]),
    "mc_ww_set_table": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, DP, DP]),
    "mc_ww_set_table_t": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, DP, DP]),
    "mc_mlp_param_count": (C.c_int, []),
    "mc_mlp_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "mc_mlp_destroy": (None, [C.c_void_p]),
    "mc_mlp_set_params": (C.c_int, [C.c_void_p, DP, C.c_size_t]),
    "mc_mlp_get_params": (C.c_int, [C.c_void_p, DP, C.c_size_t]),
    "mc_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mc_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "mc_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float,
                               C.c_void_p, C.c_void_p]),
    "mc_ww_learn": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_double,
                              C.c_double, DP]),
    "mc_ww_set_mlp": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint16), C.c_size_t]),
    "mc_ww_train": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_float]),
    "mc_run_static": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.POINTER(mc_run_opts),
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "mc_run_tune": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.POINTER(mc_run_opts), C.c_void_p,
                              C.POINTER(mc_run_opts), DP]),
    "mc_run_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_uint64), C.c_uint64,
                               C.POINTER(mc_run_opts), C.c_void_p, DP]),
    "mc_batch_tune": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_uint64), C.c_uint64,
                                C.POINTER(mc_run_opts), C.c_void_p, C.POINTER(mc_run_opts), DP]),
}

_lib = None
_lock = threading.Lock()


def lib(build_if_missing: bool = True):
    """Loads libmcgb.so (building it with nvcc first if it is missing or stale); with the
    environment variable MCGB_CHECKED=1 the bounds-checked build libmcgb_checked.so instead."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("MCGB_CHECKED") == "1"
            path = (_build.build(checked=checked) if build_if_missing
                    else (_build.LIB_CHECKED if checked else _build.LIB))
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().mc_last_error().decode(errors="replace")


def check(rc: int):
    if rc != MC_OK:
        raise McError(rc, last_error())
    return rc


def run_opts(**kw) -> mc_run_opts:
    o = mc_run_opts()
    lib().mc_run_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp32": MC_FP32, "fp64": MC_FP64}[v]
        if k == "algorithm" and isinstance(v, str):
            v = {"event": 0, "history": 1, "auto": 2}[v]
        if k == "pc_method" and isinstance(v, str):
            v = {"split": 0, "comb": 1}[v]
        if k == "tally_mode" and isinstance(v, str):
            v = {"fixed": MC_TALLY_FIXED64, "fp64": MC_TALLY_FP64}[v]
        if k == "census_times":
            # interior census times of population control; the array lives as long as the options
            o._census = np.ascontiguousarray(v, dtype=np.float64)
            o.n_census = int(o._census.size)
            v = o._census.ctypes.data_as(DP)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------------------ marshalling
class _Desc:
    """Builds an mc_problem_desc from a problem dict; keeps the arrays alive while in use."""

    def __init__(self, prob: dict):
        self.keep = []
        G = int(prob["G"])
        mats = prob["materials"]
        d = mc_problem_desc()
        d.n_groups, d.n_materials = G, len(mats)

        def dp(x):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
            self.keep.append(a)
            return a.ctypes.data_as(DP)

        def ip(x):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.int32).ravel())
            self.keep.append(a)
            return a.ctypes.data_as(IP)

        d.sigma_t = dp([m["sigma_t"] for m in mats])
        d.sigma_s = dp([m["sigma_s"] for m in mats])
        d.sigma_f = dp([m["sigma_f"] for m in mats])
        d.nu = dp([m["nu"] for m in mats])
        d.chi = dp([m["chi"] for m in mats])
        d.speed = dp(prob["speed"])
        surfs = prob["surfaces"]
        sa = (mc_surface * len(surfs))()
        for i, s in enumerate(surfs):
            sa[i].kind = KIND[s["kind"]]
            sa[i].bc = BC[s["bc"]]
            for j, c in enumerate(s["coef"]):
                sa[i].coef[j] = c
        self.keep.append(sa)
        d.n_surfaces, d.surfaces = len(surfs), sa
        cells = prob["cells"]
        ca = (mc_cell * len(cells))()
        for i, c in enumerate(cells):
            hs = c["halfspaces"]
            if len(hs) > MAX_HALFSPACES:
                raise McError(MC_ERR_INVALID, f"cell {i} has more than {MAX_HALFSPACES} half-spaces")
            ca[i].n_halfspaces = len(hs)
            for j, (s, sn) in enumerate(hs):
                ca[i].surface[j] = s
                ca[i].sense[j] = sn
            ca[i].material = c["material"]
        self.keep.append(ca)
        d.n_cells, d.cells = len(cells), ca
        lat = prob.get("lattice")
        if lat:
            L = mc_lattice()
            L.nx, L.ny = lat["nx"], lat["ny"]
            L.x0, L.y0, L.pitch, L.radius = lat["x0"], lat["y0"], lat["pitch"], lat["radius"]
            L.pin_material = ip(lat["pin_material"])
            L.matrix_material = lat["matrix_material"]
            L.nz, L.z0, L.pitch_z = lat.get("nz", 0), lat.get("z0", 0.0), lat.get("pitch_z", 0.0)
            self.keep.append(L)
            d.lattice = C.pointer(L)
        src = prob["source"]
        d.source.pos = SRC_POS[src["pos"]]
        d.source.dir = SRC_DIR[src["dir"]]
        for i in range(3):
            d.source.lo[i] = src["lo"][i]
            d.source.hi[i] = src["hi"][i]
        d.source.group_pdf = dp(src["group_pdf"])
        d.source.t0, d.source.t1 = src["t0"], src["t1"]
        tals = prob["tallies"]
        ta = (mc_mesh_tally * max(1, len(tals)))()
        for i, t in enumerate(tals):
            ta[i].nx, ta[i].ny = len(t["x"]) - 1, len(t["y"]) - 1
            ta[i].nz, ta[i].nt = len(t["z"]) - 1, len(t["t"]) - 1
            ta[i].x, ta[i].y, ta[i].z, ta[i].t = dp(t["x"]), dp(t["y"]), dp(t["z"]), dp(t["t"])
            ta[i].estimator = ESTIMATOR[t.get("estimator", "track")]
        self.keep.append(ta)
        d.n_tallies, d.tallies = len(tals), ta
        d.t_census = prob["t_census"]
        self.desc = d


def problem_create(prob: dict) -> int:
    """mc_problem_create: returns the opaque handle (an int)."""
    m = _Desc(prob)
    h = C.c_void_p()
    check(lib().mc_problem_create(C.byref(m.desc), C.byref(h)))
    return h.value


def problem_destroy(h: int):
    lib().mc_problem_destroy(C.c_void_p(h))


def run(h: int, n_histories: int, seed: int, opts: mc_run_opts | None = None, stream=None):
    """mc_run: asynchronous on `stream` (a torch.cuda.Stream, a raw handle or None)."""
    s = _stream_handle(stream)
    check(lib().mc_run(C.c_void_p(h), int(n_histories), int(seed) & (2**64 - 1),
                       C.byref(opts) if opts is not None else None, C.c_void_p(s)))


def run_tune(h: int, n_histories: int, seed: int, opts: mc_run_opts | None = None, stream=None):
    """mc_run_tune: times the kernel configurations on this problem and keeps the fastest for later
    runs with default block_size / blocks_per_sm; returns (tuned options, its time in ms)."""
    tuned = mc_run_opts()
    ms = C.c_double(0.0)
    check(lib().mc_run_tune(C.c_void_p(h), int(n_histories), int(seed) & (2**64 - 1),
                            C.byref(opts) if opts is not None else None,
                            C.c_void_p(_stream_handle(stream)), C.byref(tuned), C.byref(ms)))
    return tuned, ms.value


def run_eigen(h: int, n_per_cycle: int, n_inactive: int, n_active: int, seed: int,
              opts: mc_run_opts | None = None, stream=None):
    """mc_run_eigen: k-eigenvalue power iteration; returns (k of every cycle, fission sites banked
    per cycle, mean k over the active cycles, its standard error).  Synchronises every cycle."""
    nc = n_inactive + n_active
    k = np.zeros(nc)
    sites = np.zeros(nc, np.uint64)
    km, ke = C.c_double(0.0), C.c_double(0.0)
    check(lib().mc_run_eigen(C.c_void_p(h), int(n_per_cycle), int(n_inactive), int(n_active),
                             int(seed) & (2**64 - 1), C.byref(opts) if opts is not None else None,
                             C.c_void_p(_stream_handle(stream)), k.ctypes.data_as(DP),
                             sites.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(km), C.byref(ke)))
    return k, sites, km.value, ke.value


def wait(h: int):
    check(lib().mc_wait(C.c_void_p(h)))


def tally_shape(h: int, tally_id: int):
    shp = (C.c_int64 * 5)()
    check(lib().mc_tally_shape(C.c_void_p(h), tally_id, shp))
    return tuple(int(v) for v in shp)


def tally_get(h: int, tally_id: int):
    shp = tally_shape(h, tally_id)
    n = int(np.prod(shp))
    mean = np.zeros(n)
    err = np.zeros(n)
    check(lib().mc_tally_get(C.c_void_p(h), tally_id, mean.ctypes.data_as(DP),
                             err.ctypes.data_as(DP), n))
    return mean.reshape(shp), err.reshape(shp)


def tally_sums(h: int, tally_id: int):
    """mc_tally_sums: (exact int64 sums per bin, fixed_bits) of the last run's fixed-point tally."""
    shp = tally_shape(h, tally_id)
    out = np.zeros(int(np.prod(shp)), np.int64)
    bits = C.c_int(0)
    check(lib().mc_tally_sums(C.c_void_p(h), int(tally_id), out.ctypes.data_as(C.POINTER(C.c_int64)), out.size,
                              C.byref(bits)))
    return out.reshape(shp), bits.value


def tally_batches(h: int, tally_id: int) -> np.ndarray:
    """mc_tally_batches: per-batch per-source-particle means, shape (n_batches, *tally shape)."""
    shp = tally_shape(h, tally_id)
    nb = C.c_int(0)
    check(lib().mc_tally_batches(C.c_void_p(h), tally_id, None, 0, C.byref(nb)))
    out = np.zeros((nb.value, int(np.prod(shp))))
    check(lib().mc_tally_batches(C.c_void_p(h), tally_id, out.ctypes.data_as(DP), out.size,
                                 C.byref(nb)))
    return out.reshape((nb.value,) + shp)


def counters_get(h: int, allow_error: bool = False) -> dict:
    """mc_counters_get.  The library returns the counters even after a device error (bank
    overflow, watchdog); unless allow_error, the run's status is then raised here."""
    c = (C.c_int64 * NCOUNTERS)()
    check(lib().mc_counters_get(C.c_void_p(h), c, NCOUNTERS))
    if not allow_error:
        check(lib().mc_wait(C.c_void_p(h)))
    return dict(zip(COUNTER_NAMES, [int(v) for v in c]))


def event_log(h: int, cap: int) -> np.ndarray:
    buf = (mc_event * max(1, cap))()
    n = C.c_size_t(0)
    check(lib().mc_event_log(C.c_void_p(h), buf, cap, C.byref(n)))
    assert C.sizeof(mc_event) == EVENT_DTYPE.itemsize
    ev = np.frombuffer(buf, dtype=EVENT_DTYPE, count=max(1, cap))[: n.value].copy()
    return ev[np.lexsort((ev["k"], ev["tag"]))]


def run_static(h: int, n_histories: int, seed: int, opts: mc_run_opts | None, mean_dev_ptr: int,
               err_dev_ptr: int, stream=None):
    """mc_run_static: the run for callers that cannot allocate device memory; writes the
    per-bin mean and standard error into the given device arrays (NaN if the run failed)."""
    check(lib().mc_run_static(C.c_void_p(h), int(n_histories), int(seed) & (2**64 - 1),
                              C.byref(opts) if opts is not None else None, C.c_void_p(mean_dev_ptr),
                              C.c_void_p(err_dev_ptr), C.c_void_p(_stream_handle(stream))))


def _batch_args(handles, n_hist):
    n = len(handles)
    if len(n_hist) != n:
        raise ValueError("one history count per problem")
    hs = (C.c_void_p * n)(*[C.c_void_p(h) for h in handles])
    ns = (C.c_uint64 * n)(*[int(v) for v in n_hist])
    return n, hs, ns


def run_batch(handles, n_hist, seed: int, opts: mc_run_opts | None = None, stream=None,
              wall: bool = False):
    """mc_run_batch: the problems (handles) in one persistent launch; problem i uses seed + i.
    With wall=True it synchronises and returns each problem's completion time (s) since the
    launch started, else None."""
    n, hs, ns = _batch_args(handles, n_hist)
    out = np.zeros(n) if wall else None
    check(lib().mc_run_batch(hs, n, ns, int(seed) & (2**64 - 1),
                             C.byref(opts) if opts is not None else None,
                             C.c_void_p(_stream_handle(stream)),
                             out.ctypes.data_as(DP) if wall else None))
    return out


def batch_tune(handles, n_hist, seed: int, opts: mc_run_opts | None = None, stream=None):
    """mc_batch_tune: times the candidate configurations and stores the fastest for batches of
    this shape; returns (tuned options, its launch time in ms)."""
    n, hs, ns = _batch_args(handles, n_hist)
    tuned = mc_run_opts()
    ms = C.c_double(0.0)
    check(lib().mc_batch_tune(hs, n, ns, int(seed) & (2**64 - 1),
                              C.byref(opts) if opts is not None else None,
                              C.c_void_p(_stream_handle(stream)), C.byref(tuned), C.byref(ms)))
    return tuned, ms.value


def ww_set_table(h: int, ww: dict):
    """mc_ww_set_table from {x, y, z: edges, center: [nz][ny][nx][G]}, or mc_ww_set_table_t when
    the dict also has time edges t (center: [nt][nz][ny][nx][G])."""
    axes = "xyzt" if "t" in ww else "xyz"
    edges = np.ascontiguousarray(np.concatenate([np.asarray(ww[k], np.float64) for k in axes]))
    centre = np.ascontiguousarray(np.asarray(ww["center"], np.float64).ravel())
    n = [len(ww[k]) - 1 for k in axes]
    if "t" in ww:
        check(lib().mc_ww_set_table_t(C.c_void_p(h), n[0], n[1], n[2], n[3], edges.ctypes.data_as(DP),
                                      centre.ctypes.data_as(DP)))
    else:
        check(lib().mc_ww_set_table(C.c_void_p(h), n[0], n[1], n[2], edges.ctypes.data_as(DP),
                                    centre.ctypes.data_as(DP)))


def atomic_peak(span: int) -> float:
    """mc_atomic_peak: 64-bit atomic adds per second over `span` random slots."""
    v = C.c_double(0)
    check(lib().mc_atomic_peak(int(span), C.byref(v)))
    return v.value


def op_rates() -> dict:
    """mc_op_rates: operations per SM clock per SM of the instruction kinds the walk depends on."""
    out = np.zeros(6)
    check(lib().mc_op_rates(out.ctypes.data_as(DP), 6))
    return dict(zip(("fp32_fma", "fp64_add", "umulhi", "int_to_float", "float_to_int64", "logf"),
                    (float(v) for v in out)))


def run_timing(h: int):
    """mc_run_timing: (transport_ms, stats_ms) of the last run."""
    a, b = C.c_double(0), C.c_double(0)
    check(lib().mc_run_timing(C.c_void_p(h), C.byref(a), C.byref(b)))
    return a.value, b.value


def tally_layout(h: int):
    """mc_tally_layout: (stripes, n_batches, row) of the last run's device tallies."""
    st, nb, row = C.c_int(0), C.c_int(0), C.c_uint64(0)
    check(lib().mc_tally_layout(C.c_void_p(h), C.byref(st), C.byref(nb), C.byref(row)))
    return st.value, nb.value, row.value


def run_launches(h: int) -> int:
    """mc_run_launches: kernels the last plain mc_run launched."""
    n = C.c_int(0)
    check(lib().mc_run_launches(C.c_void_p(h), C.byref(n)))
    return n.value


def trace_get(h: int, cap: int = 65536):
    """mc_trace_get: per-iteration (t_ns, items, sources, drain) arrays of the last run."""
    t = np.zeros(cap, np.uint64)
    w = np.zeros(cap, np.uint64)
    s = np.zeros(cap, np.uint64)
    n = C.c_size_t(0)
    u64p = lambda a: a.ctypes.data_as(C.POINTER(C.c_uint64))
    check(lib().mc_trace_get(C.c_void_p(h), u64p(t), u64p(w), u64p(s), cap, C.byref(n)))
    k = n.value
    return t[:k], w[:k], s[:k] & ((1 << 63) - 1), (s[:k] >> 63).astype(bool)


def philox(seed: int, ctr_dev_ptr: int, out_dev_ptr: int, n: int, stream=None):
    """mc_philox on device arrays of 4*n uint32 words."""
    check(lib().mc_philox(int(seed) & (2**64 - 1), C.c_void_p(ctr_dev_ptr),
                          C.c_void_p(out_dev_ptr), int(n), C.c_void_p(_stream_handle(stream))))


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Problem:
    """Owning wrapper around an mc_problem handle."""

    def __init__(self, prob: dict):
        self.prob = prob
        self.h = problem_create(prob)
        self.n_tallies = len(prob["tallies"])

    def run(self, n_histories, seed=1, stream=None, **opts):
        self.opts = run_opts(**opts)
        run(self.h, n_histories, seed, self.opts, stream)
        return self

    def run_eigen(self, n_per_cycle, n_inactive, n_active, seed=1, stream=None, **opts):
        self.opts = run_opts(**opts)
        return run_eigen(self.h, n_per_cycle, n_inactive, n_active, seed, self.opts, stream)

    def wait(self):
        wait(self.h)

    def tally(self, i=0):
        return tally_get(self.h, i)

    def set_weight_windows(self, ww):
        ww_set_table(self.h, ww)

    def tally_batches(self, i=0):
        return tally_batches(self.h, i)

    def tally_sums(self, i=0):
        return tally_sums(self.h, i)

    def leakage(self):
        return tally_get(self.h, self.n_tallies)

    def counters(self):
        return counters_get(self.h)

    def table_bytes(self):
        return int(lib().mc_problem_table_bytes(C.c_void_p(self.h)))

    def trace(self):
        return trace_get(self.h)

    def timing(self):
        return run_timing(self.h)

    def launches(self):
        return run_launches(self.h)

    def events(self, cap):
        return event_log(self.h, cap)

    def close(self):
        if self.h:
            problem_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Owning wrapper around an mc_mlp handle (the weight-window importance network).  Device
    arrays are passed as raw pointers (e.g. torch tensors' data_ptr())."""

    def __init__(self, params=None):
        h = C.c_void_p()
        check(lib().mc_mlp_create(C.byref(h)))
        self.h = h.value
        self.n_params = int(lib().mc_mlp_param_count())
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        a = np.ascontiguousarray(np.asarray(params, np.float64).ravel())
        check(lib().mc_mlp_set_params(C.c_void_p(self.h), a.ctypes.data_as(DP), a.size))

    def get_params(self):
        a = np.zeros(self.n_params)
        check(lib().mc_mlp_get_params(C.c_void_p(self.h), a.ctypes.data_as(DP), a.size))
        return a

    def forward(self, x_ptr, y_ptr, n, stream=None):
        check(lib().mc_mlp_forward(C.c_void_p(self.h), C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(n),
                                   C.c_void_p(_stream_handle(stream))))

    def loss_grad(self, x_ptr, t_ptr, w_ptr, n, g_ptr, l_ptr, stream=None):
        check(lib().mc_mlp_loss_grad(C.c_void_p(self.h), C.c_void_p(x_ptr), C.c_void_p(t_ptr),
                                     C.c_void_p(w_ptr), int(n), C.c_void_p(g_ptr), C.c_void_p(l_ptr),
                                     C.c_void_p(_stream_handle(stream))))

    def train(self, x_ptr, t_ptr, w_ptr, n, epochs, lr, loss_ptr=0, stream=None):
        check(lib().mc_mlp_train(C.c_void_p(self.h), C.c_void_p(x_ptr), C.c_void_p(t_ptr),
                                 C.c_void_p(w_ptr), int(n), int(epochs), float(lr),
                                 C.c_void_p(loss_ptr), C.c_void_p(_stream_handle(stream))))

    def close(self):
        if self.h:
            lib().mc_mlp_destroy(C.c_void_p(self.h))
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ww_learn(problem_h: int, mlp: "Mlp", tally_id: int, epochs: int, lr: float,
             extrap_slope: float = 0.0, extrap_efolds: float = 0.0) -> dict:
    """mc_ww_learn: one learning round of the weight windows from the problem's last run
    (extrap_slope > 0 continues the windows past the resolved depth)."""
    info = np.zeros(5)
    check(lib().mc_ww_learn(C.c_void_p(problem_h), C.c_void_p(mlp.h), int(tally_id), int(epochs),
                            float(lr), float(extrap_slope), float(extrap_efolds),
                            info.ctypes.data_as(DP)))
    return {"points": int(info[0]), "loss": float(info[1]), "scale": float(info[2]),
            "phi_ref": float(info[3]), "extrapolated": int(info[4])}


def ww_set_mlp(problem_h: int, bf16_bits) -> None:
    """mc_ww_set_mlp: load the problem's own network from BF16 bit patterns (uint16)."""
    a = np.ascontiguousarray(np.asarray(bf16_bits, dtype=np.uint16).ravel())
    check(lib().mc_ww_set_mlp(C.c_void_p(problem_h), a.ctypes.data_as(C.POINTER(C.c_uint16)), a.size))


def ww_train(problem_h: int, tally_id: int, epochs: int, lr: float) -> None:
    """mc_ww_train: one learning round of the weight windows with the problem's own network."""
    check(lib().mc_ww_train(C.c_void_p(problem_h), int(tally_id), int(epochs), float(lr)))


def to_bf16_bits(params) -> np.ndarray:
    """BF16 bit patterns (round to nearest even) of FP64 parameters."""
    f = np.asarray(params, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (f + 0x7FFF + ((f >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)
