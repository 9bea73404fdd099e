"""Builds libmcgb.so (the sm_103a CUDA library behind include/mc.h) in-tree with nvcc.

Each translation unit is compiled in parallel for sm_103a only, then linked into one shared
library next to this file.  No cmake; a rebuild happens only when a source is newer than the
library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmcgb.so")
LIB_CHECKED = os.path.join(HERE, "libmcgb_checked.so")  # every computed index checked (MC_ERR_BOUNDS)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         f"-I{os.path.join(ROOT, 'include')}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


# The transport translation units round every product and sum separately (no contraction into
# FMA): the compiler's contraction choices depend on the optimisation context of each kernel
# build, so with contraction the 80- and 128-register builds of the walk (and the batched kernel)
# could round a geometry expression differently and move a particle differently.  Without it every
# build computes the same bits, and the FP64 walk rounds as the CPU reference does.
NO_FMA = {"mc_transport.cu", "mc_transport_seg.cu", "mc_transport_range.cu", "mc_batch.cu", "mc_api.cu"}


def per_file_flags(src):
    return ["-fmad=false"] if os.path.basename(src) in NO_FMA else []


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "mc.h")])


def up_to_date(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in sources() + headers() + [__file__])


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libmcgb.so, or with checked=True the bounds-checked libmcgb_checked.so (the same
    sources with -DMCGB_CHECKED, objects in their own folder)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    obj_dir = os.path.join(HERE, "_build_checked" if checked else "_build")
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    procs, objs = [], []
    for src in sources():
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *per_file_flags(src), *(["-DMCGB_CHECKED"] if checked else []), "-c", src,
               "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
