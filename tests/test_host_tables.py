"""Host logic of the library's table builder (csrc/mc_tables.h), compiled on its own with the
host C++ compiler: the first-guess rules of the tally axes (equal spacing, log-spaced time bins,
bisection otherwise; every guess within one bin of the bisection's bin) and the box-cell entries
of cells bounded by axis-aligned planes."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_table_classification(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "host_tables")
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2305_07636_gb300", "csrc"),
                           os.path.join(HERE, "host_tables.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
