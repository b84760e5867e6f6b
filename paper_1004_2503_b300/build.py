"""Build libaton.so (the C-ABI library of the ATON step) for sm_103a, in-tree.

    python -m paper_1004_2503_b300.build [--force] [--verbose]

nvcc cross-compiles without a GPU. The library links the CUDA runtime statically and needs
no PyTorch.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libaton.so")
SOURCES = ["aton_capi.cu", "aton_kernels.cu", "aton_tma.cu", "aton_mlp.cu", "aton_mlp_tc.cu",
           "aton_static.cu", "aton_stats.cu", "aton_sources.cu"]
HEADERS = ["aton_device.cuh", "aton_internal.h", "aton_step_common.cuh", "aton_mlp.cuh",
           "aton_stats.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The kernels use the hardware approximations of division, reciprocal square root, square root,
# exp2 and log2 (a few ulp) and flush FP32 denormals: every denominator in the kernels is
# positive and far from the FP32 limits, and the parity tests bound the effect against the
# FP64 oracle. The photon tallies stay compensated sums of FP32 values reduced in FP64.
FAST = ["--use_fast_math"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "aton.h"))
    files.append(os.path.abspath(__file__))
    return files


def stale(target=LIB):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force=False, verbose=False, ptxas_verbose=False):
    if not force and not stale():
        return LIB
    cmd = [NVCC, *ARCH, *FAST, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", INCLUDE, "-I", CSRC, "-o", LIB]
    if ptxas_verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, f) for f in SOURCES]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--verbose" in sys.argv)
