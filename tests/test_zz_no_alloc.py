"""mc_run_static: the run entry point for callers that cannot allocate device memory (applications
whose device memory all belongs to their own pool, allocator or memory-pressure callbacks, hosts
that fix their device-memory budget at start-up).  It keeps its scratch in the library's static
device array, so its results must equal those of mc_run on the same problem, seed and options.
This file is collected last."""
import numpy as np
import pytest

from paper_2305_07636_gb300 import mc
from paper_2305_07636_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _all_bins(p, n_tallies):
    means, errs = [], []
    for t in range(n_tallies + 1):  # every mesh tally, then the leakage tally
        m, e = mc.tally_get(p.h, t)
        means.append(m.ravel())
        errs.append(e.ravel())
    return np.concatenate(means), np.concatenate(errs)


# (problem, histories, run options, weight windows): the pulse in FP32 with int64 tallies (its
# 100 time bins take the range walk and its reconstruction), the slab with FP64 tallies, the pulse
# tracked in FP64, and a weighted slab stack with splitting and roulette and FP64 tallies
CASES = {
    "pulse_fp32_fixed": (P.config2, 200_000, {}, False),
    "slab_fp64_tally": (P.config1, 200_000, {"tally_mode": "fp64"}, False),
    "pulse_fp64_tracking": (P.config2, 50_000, {"precision": "fp64"}, False),
    "windows_fp64_tally": (lambda: P.slab_stack(thickness=8.0, n_layers=4, detector=2.0, ww_bin=1.0, name="thin"),
                           4_000, {"tally_mode": "fp64", "ww_enable": 1, "bank_capacity": 32768}, True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_run_equals_mc_run_on_two_calls_in_a_row(case):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    make, n, extra, windows = CASES[case]
    prob = make()
    p = mc.Problem(prob)
    if windows:
        p.set_weight_windows(P.exponential_ww(prob, decay=0.8))
    n_bins = sum(int(np.prod(mc.tally_shape(p.h, t))) for t in range(len(prob["tallies"]) + 1))
    mean_d = torch.empty(n_bins, dtype=torch.float64, device="cuda")
    err_d = torch.empty(n_bins, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    fp64_tally = extra.get("tally_mode") == "fp64"
    for seed in (41, 42):  # the second call reuses the static array left by the first
        opts = mc.run_opts(n_batches=16, **extra)
        mc.run_static(p.h, n, seed, opts, mean_d.data_ptr(), err_d.data_ptr(), stream)
        torch.cuda.synchronize()
        ms, es = mean_d.cpu().numpy(), err_d.cpu().numpy()
        p.run(n, seed, n_batches=16, **extra)
        m0, e0 = _all_bins(p, len(prob["tallies"]))
        if windows:
            assert p.counters()["ww_held"] == 0  # no split held: both runs make the same copies
        assert np.isfinite(ms).all() and np.isfinite(es).all()
        assert np.count_nonzero(m0) > 20
        # integer tallies are summed exactly by both paths: only the final rounding may differ;
        # FP64 tallies add in the order the atomics arrive
        rtol = 1e-9 if fp64_tally else 1e-12
        assert np.allclose(ms, m0, rtol=rtol, atol=0.0)
        assert np.allclose(es, e0, rtol=1e-6 if fp64_tally else 1e-12, atol=1e-300)
    p.close()


def test_static_run_rejects_tallies_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    p = mc.Problem(P.config3())  # 404,604 bins: 35 x 3.2 MB does not fit 32 MB
    buf = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.McError) as e:
        mc.run_static(p.h, 100_000, 1, mc.run_opts(), buf.data_ptr(), buf.data_ptr())
    assert e.value.code == mc.MC_ERR_INVALID and "static scratch" in str(e.value)
    with pytest.raises(mc.McError) as e:
        mc.run_static(p.h, 100_000, 1, mc.run_opts(bank_capacity=1 << 20), buf.data_ptr(),
                      buf.data_ptr())
    assert e.value.code == mc.MC_ERR_INVALID
    p.close()


def test_static_run_rejects_bad_outputs_and_small_banks():
    """Host, misaligned and too-small-bank requests fail with MC_ERR_INVALID before any launch."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    p = mc.Problem(P.config1())
    dev = torch.empty(64, dtype=torch.float64, device="cuda")
    host = np.zeros(64)
    bad = [(host.ctypes.data, dev.data_ptr(), {}),          # a host array
           (dev.data_ptr() + 4, dev.data_ptr(), {}),         # misaligned
           (dev.data_ptr(), dev.data_ptr(), {"bank_capacity": 512})]
    for mean_ptr, err_ptr, extra in bad:
        with pytest.raises(mc.McError) as e:
            mc.run_static(p.h, 10_000, 1, mc.run_opts(**extra), mean_ptr, err_ptr)
        assert e.value.code == mc.MC_ERR_INVALID
    p.close()
