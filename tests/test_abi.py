"""The C-ABI library loads without a GPU, exports every entry point that include/mc.h declares,
and rejects invalid problem descriptions on the host before touching CUDA.  No compute calls."""
import ctypes as C
import math
import os
import re

import pytest

from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    # the calls of the boundary sketch, and the ones this library adds
    for core in ("mc_problem_create", "mc_run", "mc_run_batch", "mc_tally_get", "mc_tally_shape",
                 "mc_ww_set_mlp", "mc_ww_train", "mc_event_log", "mc_problem_destroy", "mc_last_error",
                 "mc_wait", "mc_counters_get", "mc_philox", "mc_run_eigen", "mc_run_tune"):
        assert core in names


def test_bf16_bit_patterns():
    import numpy as np
    x = np.array([1.0, -2.5, 3.140625, 1.0 + 2.0**-8, 1.0 + 3 * 2.0**-9, 0.0, 1e-30])
    b = mc.to_bf16_bits(x)
    back = (b.astype(np.uint32) << 16).view(np.float32)
    assert back[0] == 1.0 and back[1] == -2.5 and back[2] == 3.140625 and back[5] == 0.0
    assert back[3] == 1.0  # a tie rounds to even
    assert back[4] == 1.0 + 2.0**-7  # above the tie rounds up
    assert abs(back[6] - 1e-30) < 1e-32


def test_library_exports_every_declared_symbol():
    L = C.CDLL(mc._build.build())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(mc.SIGNATURES)


def test_run_opts_defaults():
    o = mc.run_opts()
    assert (o.precision, o.tally_mode, o.fixed_bits, o.n_batches) == (0, 0, 32, 32)
    assert o.aggregate_atomics == -1 and o.algorithm == 0


def _bad(mutator):
    prob = P.config1()
    mutator(prob)
    with pytest.raises(mc.McError) as e:
        mc.problem_create(prob)
    assert e.value.code == mc.MC_ERR_INVALID
    return str(e.value)


@pytest.mark.parametrize("case", [
    lambda p: p["materials"][0].__setitem__("sigma_s", [[1.5]]),          # channels exceed sigma_t
    lambda p: p["materials"][0].__setitem__("sigma_t", [-1.0]),
    lambda p: p["materials"][0].__setitem__("nu", [100.0]),
    lambda p: p.__setitem__("speed", [0.0]),
    lambda p: p["surfaces"][0].__setitem__("kind", "CZ") or p["surfaces"][0].__setitem__("coef", [0, 0, 1]) or p["surfaces"][0].__setitem__("bc", "reflect"),
    lambda p: p["cells"][0].__setitem__("halfspaces", [(7, 1)]),
    lambda p: p["cells"][0].__setitem__("material", -1),                    # lattice fill, no lattice
    lambda p: p["source"].__setitem__("group_pdf", [0.0]),
    lambda p: p["tallies"][0].__setitem__("x", [0.0, 2.0, 1.0]),           # edges not increasing
    lambda p: p.__setitem__("t_census", 0.0),
])
def test_invalid_descriptions_are_rejected_on_the_host(case):
    assert _bad(case)


def test_no_gpu_means_a_loud_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mc.McError) as e:
        mc.problem_create(P.config1())
    assert e.value.code in (mc.MC_ERR_CUDA, mc.MC_ERR_OOM)
    assert math.isfinite(len(str(e.value)))


def test_binding_limits_match_the_header():
    text = open(os.path.join(ROOT, "include", "mc.h")).read()
    lim = {k: int(v) for k, v in re.findall(r"#define MC_MAX_(\w+) (\d+)", text)}
    assert (lim["GROUPS"], lim["SURFACES"], lim["CELLS"], lim["HALFSPACES"]) == (
        mc.MAX_GROUPS, mc.MAX_SURFACES, mc.MAX_CELLS, mc.MAX_HALFSPACES)
    assert (lim["LATTICE"], lim["LATTICE_ELEMENTS"]) == (mc.MAX_LATTICE, mc.MAX_LATTICE_ELEMENTS)


def test_lattice_index_division_by_reciprocal():
    """The device splits a lattice element index e < 2^16 into (ix, iy, iz) with n / d =
    floor(n * ceil(2^32 / d) / 2^32): exact for every divisor an axis can have and every index."""
    import numpy as np
    n = np.arange(mc.MAX_LATTICE_ELEMENTS, dtype=np.uint64)
    for d in range(1, mc.MAX_LATTICE + 1):
        m = np.uint64(((1 << 32) + d - 1) // d)
        assert np.array_equal((n * m) >> np.uint64(32), n // np.uint64(d)), d
