"""The project's Philox4x32-10 (the CUDA path's, through the C ABI, and the oracle's) equals
cuRAND's Philox4_32_10 device generator bit for bit on random keys and full 128-bit counters
(cuRAND: key = seed, counter = (block, subsequence)).  The oracle is pinned to Triton's
implementation on the CPU as well; this pins both sides to NVIDIA's library on the GPU.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2305_07636_gb300 import build as native_build
from paper_2305_07636_gb300 import mc

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_equals_curand(tmp_path):
    import torch
    so = str(tmp_path / "libcurand_ref.so")
    subprocess.check_call([native_build.nvcc(), *native_build.ARCH, "-O2", "-shared", "-Xcompiler", "-fPIC",
                           "-o", so, os.path.join(HERE, "curand_ref.cu")], timeout=600)
    ref = C.CDLL(so)
    ref.curand_ref.restype = C.c_int
    rng = np.random.default_rng(2024)
    n = 4096
    for _ in range(3):
        seed = int(rng.integers(0, 2**63))
        sub = rng.integers(0, 2**63, size=n, dtype=np.uint64)
        blk = rng.integers(0, 2**62, size=n, dtype=np.uint64)
        out = np.zeros((n, 4), np.uint32)
        assert ref.curand_ref(C.c_ulonglong(seed), sub.ctypes.data_as(C.c_void_p), blk.ctypes.data_as(C.c_void_p),
                              out.ctypes.data_as(C.c_void_p), n) == 0
        ctr = np.stack([blk & 0xFFFFFFFF, blk >> np.uint64(32), sub & 0xFFFFFFFF, sub >> np.uint64(32)],
                       axis=1).astype(np.uint32)
        # the CUDA path's generator (mc_philox), on the device
        d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        mc.philox(seed, d_ctr.data_ptr(), d_out.data_ptr(), n)
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy().view(np.uint32), out)
        for i in range(0, n, 97):  # and the oracle's
            assert oracle.philox((seed & 0xFFFFFFFF, seed >> 32), [int(v) for v in ctr[i]]) == [int(v) for v in out[i]]


def test_philox_uniformity_on_1e8_words():
    """10^8 output words of the device generator (counters (i, 0, seed-derived, 0)): chi-square of a
    1000-bin histogram and Kolmogorov-Smirnov on 10^6 of them against the uniform law, and the lag-1
    serial correlation of consecutive words, at the 10^-3 level."""
    import torch
    from scipy import stats
    n_blocks = 25_000_000  # x 4 words
    ctr = torch.zeros((n_blocks, 4), dtype=torch.int32, device="cuda")
    ctr[:, 0] = torch.arange(n_blocks, dtype=torch.int64, device="cuda").to(torch.int32)
    ctr[:, 2] = 12345
    out = torch.zeros_like(ctr)
    mc.philox(0x243F6A8885A308D3, ctr.data_ptr(), out.data_ptr(), n_blocks)
    torch.cuda.synchronize()
    w = out.view(-1).to(torch.int64) & 0xFFFFFFFF  # unsigned words
    u = (w.to(torch.float64) + 0.5) / 4294967296.0
    hist = torch.bincount((u * 1000).to(torch.int64), minlength=1000).cpu().numpy()
    e = u.numel() / 1000
    chi2 = float(((hist - e) ** 2 / e).sum())
    assert stats.chi2.sf(chi2, 999) > 1e-3, chi2
    sample = u[:: 100].cpu().numpy()
    assert stats.kstest(sample, "uniform").pvalue > 1e-3
    x = u - 0.5
    r = float((x[:-1] * x[1:]).mean() / (x * x).mean())
    assert abs(r) < 3.3 / np.sqrt(u.numel()), r  # ~1e-3 two-sided for a correlation of 0
    del ctr, out, w, u, x
