"""The bounds-checked build (libmcgb_checked.so: every index the walk computes into the tables, the
tallies and the lattice's element map is checked before use, a bad one ends the run with
MC_ERR_BOUNDS) runs small cases of every workload family (fixed source in FP32 and FP64, both
algorithms, time crossing, implicit capture, population control, lattices up to 65,536 elements,
the duct, quadrics, weight windows, k-eigenvalue cycles, the batched launch) without a single
out-of-range index, and gives the normal build's results bit for bit.  It stands in for a memory
checker on GPUs where none runs.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_cases(out, checked):
    env = dict(os.environ)
    env["MCGB_CHECKED"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_checked_build_finds_no_bad_index_and_changes_nothing(tmp_path):
    a, b = str(tmp_path / "checked.npz"), str(tmp_path / "plain.npz")
    run_cases(a, True)  # an out-of-range index would raise MC_ERR_BOUNDS here
    run_cases(b, False)
    ra, rb = np.load(a), np.load(b)
    assert sorted(ra.files) == sorted(rb.files) and len(ra.files) > 20
    for key in ra.files:
        assert np.array_equal(ra[key], rb[key]), key
