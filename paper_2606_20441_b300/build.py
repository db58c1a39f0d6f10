"""Builds libpp.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpp.so")
# The debug build: device bounds checks on tile, list, gate, region and overflow
# indices record the first failing site and skip the access (pp_kernels.cuh,
# PP_OOB); pp_propagate then returns PP_ERR_CUDA.  Load it with PP_LIBRARY.
DEBUG_LIB = os.path.join(HERE, "libpp_debug.so")
SOURCES = ["pp.cu", "pp_noalloc.cu"]
HEADERS = ["pp_device.cuh", "pp_kernels.cuh", "pp_warp.cuh", "pp_orbit.cuh", "pp_topk.cuh", "pp_result.cuh"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared", "-diag-suppress", "177"]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "pp.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = DEBUG_LIB if debug else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc] + NVCC_FLAGS + (["-DPP_DEBUG"] if debug else []) + \
          ["-I", os.path.join(ROOT, "include"), "-o", tmp] + [os.path.join(CSRC, f) for f in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
