"""Builds the in-tree CUDA library ``libpbad.so`` for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpbad.so")
STAGE_COUNTS = (1, 2, 3, 4, 5)  # pbad_kernels.cu is compiled once per stage count
SOURCES = ["pbad_kernels.cu", "pbad_capi.cu", "pbad_static.cu", "pbad_dense.cu"]
HEADERS = ["pbad_device.cuh", "pbad_kernels.cuh", "pbad_lp.cuh", "pbad_df64.cuh", "pbad_cta.cuh", "pbad_launch.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "pbad.h"))
    deps.append(__file__)
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles csrc/*.cu into libpbad.so (skipped when up to date)."""
    if not force and not _stale():
        return LIB
    jobs = []
    for S in STAGE_COUNTS:
        obj = os.path.join(CSRC, f"pbad_kernels_s{S}.o")
        jobs.append((obj, [NVCC, *FLAGS, f"-DPBAD_S={S}", "-c",
                           os.path.join(CSRC, "pbad_kernels.cu"), "-o", obj]))
    for src in ("pbad_capi.cu", "pbad_static.cu", "pbad_dense.cu"):
        obj = os.path.join(CSRC, src.replace(".cu", ".o"))
        jobs.append((obj, [NVCC, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]))
    procs = []
    for obj, cmd in jobs:
        if verbose:
            print(" ".join(cmd))
        procs.append(subprocess.Popen(cmd))
    rcs = [p.wait() for p in procs]
    if any(rcs):
        raise RuntimeError(f"nvcc failed: {rcs}")
    objs = [o for o, _ in jobs]
    tmp = LIB + ".tmp"  # linked aside, then renamed over the library in one step
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
