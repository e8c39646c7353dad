"""Build libpct.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libpct.so")
SOURCES = ["pct_api.cu", "pct_kernels.cu", "pct_rows.cu", "pct_grad.cu", "pct_batch.cu", "pct_noalloc.cu", "pct_peaks.cu",
           "pct_clean.cu", "pct_fbp.cu", "pct_regions.cu"]
HEADERS = ["pct_device.cuh", "pct_warp.cuh", "pct_internal.h", "pct_batch.h", "pct_bins.cuh"]

# --fmad=false: no implicit contraction of a*b+c, so every kernel that walks a
# path (fused solve, stored-row builds, row dump, batch) computes bit-identical
# MLP points; fused multiply-adds are written out with fmaf where wanted.
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "--fmad=false", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "pct.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile the CUDA sources into paper_1802_01070_b300/libpct.so (if stale)."""
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + NVCC_FLAGS + list(extra) + ["-I", INCLUDE, "-I", CSRC, "-o", tmp]
    cmd += [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
