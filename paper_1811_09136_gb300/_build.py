"""Compile the CUDA library librept.so in-tree for sm_103a (nvcc, no torch extension machinery)."""
from __future__ import annotations

import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_PATH = os.path.join(PKG, "librept.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  [os.path.join(INCLUDE, "rept.h")])


DEBUG_LIB_PATH = os.path.join(PKG, "librept_debug.so")


def build(force: bool = False, verbose_ptxas: bool = False, debug_bounds: bool = False) -> str:
    """Build librept.so if any source is newer than it.  Returns the library path.  With
    ``debug_bounds``, build librept_debug.so instead: every pool, queue and node index the kernels use
    is checked (REPT_DEBUG_BOUNDS), a failed check is recorded and the access skipped, and the next
    synchronising call reports REPT_E_INTERNAL (a stand-in for a memory checker)."""
    path = DEBUG_LIB_PATH if debug_bounds else LIB_PATH
    srcs = sources()
    if not force and os.path.exists(path):
        newest = max(os.path.getmtime(p) for p in srcs)
        if os.path.getmtime(path) >= newest:
            return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-shared", "-o", tmp,
           *sorted(glob.glob(os.path.join(CSRC, "*.cu")))]
    if verbose_ptxas:
        cmd[1:1] = ["-Xptxas", "-v"]
    if debug_bounds:
        cmd[1:1] = ["-DREPT_DEBUG_BOUNDS"]
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path
