"""CPU oracle for REPT (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it runs
on the CUDA library and fails loudly without it.

``rept_oracle.c`` is the oracle proper (plain sequential C, see its header);
this module compiles it with gcc and exposes it through ctypes with numpy
arrays.  Every function states which part of the paper it follows:

* ``splitmix64`` / ``colour``      -- the edge-partition hash h_k (Section III-A, III-B)
* ``rept_stream``                  -- Algorithm 1 per processor, the c > m grouping of
                                      Section III-B, the pair counters of Algorithm 2
* ``estimates``                    -- estimators of Section III-A, III-B.1 and Algorithm 2
* ``semitriangles``                -- the semi-triangle definition (Section III) as a static
                                      triangle enumeration, plus exact tau, tau_v, eta, eta_v
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rept_oracle.c")
_LIB = os.path.join(_HERE, "librept_oracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Load an oracle shared library from ``path`` and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.orc_splitmix64.restype = ctypes.c_uint64
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64]
    lib.orc_colour.restype = ctypes.c_uint32
    lib.orc_colour.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
    lib.orc_rept_stream.restype = ctypes.c_int
    lib.orc_rept_stream.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p, _u64p, _u64p,
                                    _u64p, _u64p, _u64p]
    lib.orc_estimates.restype = None
    lib.orc_estimates.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, _u64p, _u64p, _u64p,
                                  ctypes.c_uint32, _dp, _dp]
    lib.orc_semitriangles.restype = ctypes.c_int
    lib.orc_semitriangles.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p, _u64p, _u64p,
                                      _u64p, _u64p, _u64p, _u64p]
    lib.orc_rept_stream_parallel.restype = ctypes.c_int
    lib.orc_rept_stream_parallel.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p, _u64p, ctypes.c_int]
    lib.orc_mascot_stream.restype = ctypes.c_int
    lib.orc_mascot_stream.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p, _u64p, _u64p]
    lib.orc_mascot_estimates.restype = None
    lib.orc_mascot_estimates.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, ctypes.c_uint32,
                                         _dp, _dp]
    lib.orc_mascot_semitriangles.restype = ctypes.c_int
    lib.orc_mascot_semitriangles.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_uint64, _u64p, _u64p, _u64p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def splitmix64(x: int, lib=None) -> int:
    return int((lib or _load()).orc_splitmix64(x))


def colour(u: int, v: int, seed: int, k: int, m: int, lib=None) -> int:
    """h_k(u, v) in {0..m-1}: SplitMix64(((min << 32) | max) ^ s_k) mod m, s_k = seed + k*gamma."""
    return int((lib or _load()).orc_colour(u, v, seed, k, m))


@dataclass
class Counts:
    """Integer counters of one REPT run (0-based processors)."""
    tau_proc: np.ndarray          # [c]  tau^(i)
    local1: np.ndarray            # [n]  sum of tau_v^(i) over the full groups (all processors when c <= m)
    local2: np.ndarray            # [n]  sum over the partial last group (zeros unless c > m, c % m != 0)
    eta_proc: np.ndarray | None = None   # [c] eta^(i)
    eta_local: np.ndarray | None = None  # [n] sum_i eta_v^(i)
    tau_local_proc: np.ndarray | None = None  # [c, n]
    skipped: int = 0


def _cols(src, dst):
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    assert src.shape == dst.shape
    return src, dst


def rept_stream(src, dst, n: int, m: int, c: int, seed: int, per_proc_local: bool = False,
                pair_counters: bool = True, lib=None) -> Counts:
    """Sequential REPT over the stream (Algorithm 1 per processor; grouping of Section III-B;
    triangle-pair counters of Algorithm 2)."""
    src, dst = _cols(src, dst)
    lib = lib or _load()
    tau = np.zeros(c, dtype=np.uint64)
    eta = np.zeros(c, dtype=np.uint64) if pair_counters else None
    l1 = np.zeros(n, dtype=np.uint64)
    l2 = np.zeros(n, dtype=np.uint64)
    el = np.zeros(n, dtype=np.uint64) if pair_counters else None
    tlp = np.zeros((c, n), dtype=np.uint64) if per_proc_local else None
    sk = np.zeros(1, dtype=np.uint64)
    rc = lib.orc_rept_stream(_p(src, _u32p), _p(dst, _u32p), src.size, n, m, c, seed, _p(tau, _u64p),
                             _p(eta, _u64p), _p(l1, _u64p), _p(l2, _u64p), _p(el, _u64p), _p(tlp, _u64p),
                             _p(sk, _u64p))
    if rc != 0:
        raise ValueError(f"orc_rept_stream failed ({rc})")
    return Counts(tau, l1, l2, eta, el, tlp, int(sk[0]))


def rept_stream_parallel(src, dst, n: int, m: int, c: int, seed: int, threads: int, lib=None) -> Counts:
    """tau^(i) and the local sums the paper's multi-core way: one thread per processor, each with its
    own pass over the stream (no pair counters)."""
    src, dst = _cols(src, dst)
    lib = lib or _load()
    tau = np.zeros(c, dtype=np.uint64)
    l1 = np.zeros(n, dtype=np.uint64)
    l2 = np.zeros(n, dtype=np.uint64)
    rc = lib.orc_rept_stream_parallel(_p(src, _u32p), _p(dst, _u32p), src.size, n, m, c, seed, _p(tau, _u64p),
                                      _p(l1, _u64p), _p(l2, _u64p), int(threads))
    if rc != 0:
        raise ValueError(f"orc_rept_stream_parallel failed ({rc})")
    return Counts(tau, l1, l2)


def estimates(m: int, c: int, counts: Counts, n: int, lib=None):
    """FP64 (tau_hat, tau_hat_v[n]) from the counters (Section III-A, III-B.1, Algorithm 2)."""
    lib = lib or _load()
    g = np.zeros(1, dtype=np.float64)
    loc = np.zeros(n, dtype=np.float64)
    eta = counts.eta_proc if counts.eta_proc is not None else np.zeros(c, dtype=np.uint64)
    el = counts.eta_local if counts.eta_local is not None else np.zeros(n, dtype=np.uint64)
    lib.orc_estimates(m, c, _p(np.ascontiguousarray(counts.tau_proc, dtype=np.uint64), _u64p),
                      _p(np.ascontiguousarray(eta, dtype=np.uint64), _u64p),
                      _p(np.ascontiguousarray(counts.local1, dtype=np.uint64), _u64p),
                      _p(np.ascontiguousarray(counts.local2, dtype=np.uint64), _u64p),
                      _p(np.ascontiguousarray(el, dtype=np.uint64), _u64p), n, _p(g, _dp), _p(loc, _dp))
    return float(g[0]), loc


@dataclass
class Exact:
    """Static enumeration results: semi-triangle counters plus exact graph statistics."""
    tau_proc: np.ndarray
    local1: np.ndarray
    local2: np.ndarray
    tau_local_proc: np.ndarray | None
    triangles: int
    tri_local: np.ndarray
    eta: int
    eta_local: np.ndarray


def semitriangles(src, dst, n: int, m: int, c: int, seed: int, per_proc_local: bool = False,
                  lib=None) -> Exact:
    """Semi-triangle counts by definition (static triangle enumeration), plus tau, tau_v, eta, eta_v."""
    src, dst = _cols(src, dst)
    lib = lib or _load()
    tau = np.zeros(c, dtype=np.uint64)
    l1 = np.zeros(n, dtype=np.uint64)
    l2 = np.zeros(n, dtype=np.uint64)
    tlp = np.zeros((c, n), dtype=np.uint64) if per_proc_local else None
    tt = np.zeros(1, dtype=np.uint64)
    tl = np.zeros(n, dtype=np.uint64)
    et = np.zeros(1, dtype=np.uint64)
    el = np.zeros(n, dtype=np.uint64)
    rc = lib.orc_semitriangles(_p(src, _u32p), _p(dst, _u32p), src.size, n, m, c, seed, _p(tau, _u64p),
                               _p(l1, _u64p), _p(l2, _u64p), _p(tlp, _u64p), _p(tt, _u64p), _p(tl, _u64p),
                               _p(et, _u64p), _p(el, _u64p))
    if rc != 0:
        raise ValueError(f"orc_semitriangles failed ({rc})")
    return Exact(tau, l1, l2, tlp, int(tt[0]), tl, int(et[0]), el)


# --------------------------------------------------------------------------
# parallel MASCOT (Section I, Section III-C): c independent p = 1/m samplers
# --------------------------------------------------------------------------
def mascot_stream(src, dst, n: int, m: int, c: int, seed: int, per_proc_local: bool = False,
                  lib=None) -> Counts:
    """c independent MASCOT samplers run over the stream; sampler i stores an edge iff its
    hash-group-i colour is 0.  local1 holds sum_i tau_v^(i); local2 is zero."""
    src, dst = _cols(src, dst)
    lib = lib or _load()
    tau = np.zeros(c, dtype=np.uint64)
    l1 = np.zeros(n, dtype=np.uint64)
    tlp = np.zeros((c, n), dtype=np.uint64) if per_proc_local else None
    sk = np.zeros(1, dtype=np.uint64)
    rc = lib.orc_mascot_stream(_p(src, _u32p), _p(dst, _u32p), src.size, n, m, c, seed, _p(tau, _u64p),
                               _p(l1, _u64p), _p(tlp, _u64p), _p(sk, _u64p))
    if rc != 0:
        raise ValueError(f"orc_mascot_stream failed ({rc})")
    return Counts(tau, l1, np.zeros(n, dtype=np.uint64), None, None, tlp, int(sk[0]))


def mascot_estimates(m: int, c: int, counts: Counts, n: int, lib=None):
    """FP64 (tau_hat, tau_hat_v[n]) of parallel MASCOT: the mean of the samplers' m^2 tau^(i)."""
    lib = lib or _load()
    g = np.zeros(1, dtype=np.float64)
    loc = np.zeros(n, dtype=np.float64)
    lib.orc_mascot_estimates(m, c, _p(np.ascontiguousarray(counts.tau_proc, dtype=np.uint64), _u64p),
                             _p(np.ascontiguousarray(counts.local1, dtype=np.uint64), _u64p), n, _p(g, _dp),
                             _p(loc, _dp))
    return float(g[0]), loc


def mascot_semitriangles(src, dst, n: int, m: int, c: int, seed: int, per_proc_local: bool = False,
                         lib=None):
    """Per-sampler semi-triangle counts of parallel MASCOT by static enumeration:
    (tau_proc[c], local1[n], tau_local_proc[c, n] or None)."""
    src, dst = _cols(src, dst)
    lib = lib or _load()
    tau = np.zeros(c, dtype=np.uint64)
    l1 = np.zeros(n, dtype=np.uint64)
    tlp = np.zeros((c, n), dtype=np.uint64) if per_proc_local else None
    rc = lib.orc_mascot_semitriangles(_p(src, _u32p), _p(dst, _u32p), src.size, n, m, c, seed,
                                      _p(tau, _u64p), _p(l1, _u64p), _p(tlp, _u64p))
    if rc != 0:
        raise ValueError(f"orc_mascot_semitriangles failed ({rc})")
    return tau, l1, tlp
