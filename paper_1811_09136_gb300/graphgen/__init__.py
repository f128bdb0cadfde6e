"""Seeded synthetic edge streams shared by the oracle tests, the CUDA path and the bench.

The paper evaluates on public graphs (Section IV-A, Table II) that are not
available here; these generators produce heavy-tailed stand-ins with the same
shape of input: a stream of distinct undirected edges, uint32 node ids, no
self-loops, in a seeded uniformly random order.  The arithmetic lives in
``graphgen.c`` (PCG32 randomness, no method arithmetic); this module compiles
it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, -O2, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.gg_chung_lu.restype = ctypes.c_int64
            lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p]
            lib.gg_rmat.restype = ctypes.c_int64
            lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p]
            lib.gg_gnp.restype = ctypes.c_int64
            lib.gg_gnp.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                   _u32p, _u32p, ctypes.c_uint64]
            lib.gg_shuffle.restype = None
            lib.gg_shuffle.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_pcg32_fill.restype = None
            lib.gg_pcg32_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p, ctypes.c_uint64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


class EdgeStream:
    """A stream of undirected edges: ``src[t], dst[t]`` is edge t (0-based stream index)."""

    def __init__(self, src: np.ndarray, dst: np.ndarray, n_nodes: int, name: str = ""):
        assert src.dtype == np.uint32 and dst.dtype == np.uint32 and src.shape == dst.shape
        self.src = np.ascontiguousarray(src)
        self.dst = np.ascontiguousarray(dst)
        self.n_nodes = int(n_nodes)
        self.name = name

    def __len__(self) -> int:
        return int(self.src.shape[0])

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.uint64(self.n_nodes).tobytes())
        h.update(self.src.tobytes())
        h.update(self.dst.tobytes())
        return h.hexdigest()

    def degrees(self) -> np.ndarray:
        return (np.bincount(self.src, minlength=self.n_nodes) +
                np.bincount(self.dst, minlength=self.n_nodes)).astype(np.int64)


def chung_lu(n: int, gamma: float, n_edges: int, cap: float = 0.0, graph_seed: int = 42,
             order_seed: int = 7, max_draws: int | None = None) -> EdgeStream:
    """Chung-Lu power-law graph with ``n_edges`` distinct edges (see graphgen.c)."""
    lib = _load()
    src = np.empty(n_edges, dtype=np.uint32)
    dst = np.empty(n_edges, dtype=np.uint32)
    md = max_draws if max_draws is not None else 50 * n_edges + 1000
    ne = lib.gg_chung_lu(n, gamma, cap, n_edges, md, graph_seed, order_seed, _ptr(src), _ptr(dst))
    if ne < 0:
        raise ValueError(f"gg_chung_lu failed ({ne})")
    return EdgeStream(src[:ne].copy(), dst[:ne].copy(), n, f"chung_lu(n={n},gamma={gamma},E={ne},cap={cap})")


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         graph_seed: int = 42, order_seed: int = 7) -> EdgeStream:
    """R-MAT graph with ``edge_factor * 2**scale`` draws, deduplicated (see graphgen.c)."""
    lib = _load()
    draws = edge_factor << scale
    src = np.empty(draws, dtype=np.uint32)
    dst = np.empty(draws, dtype=np.uint32)
    ne = lib.gg_rmat(scale, draws, a, b, c, graph_seed, order_seed, _ptr(src), _ptr(dst))
    if ne < 0:
        raise ValueError(f"gg_rmat failed ({ne})")
    return EdgeStream(src[:ne].copy(), dst[:ne].copy(), 1 << scale, f"rmat(scale={scale},ef={edge_factor},E={ne})")


def gnp(n: int, q: float, graph_seed: int = 1, order_seed: int = 2) -> EdgeStream:
    """Erdos-Renyi G(n, q), for small test graphs."""
    lib = _load()
    cap = n * (n - 1) // 2 + 1
    src = np.empty(cap, dtype=np.uint32)
    dst = np.empty(cap, dtype=np.uint32)
    ne = lib.gg_gnp(n, q, graph_seed, order_seed, _ptr(src), _ptr(dst), cap)
    if ne < 0:
        raise ValueError(f"gg_gnp failed ({ne})")
    return EdgeStream(src[:ne].copy(), dst[:ne].copy(), n, f"gnp(n={n},q={q})")


def complete(n: int, order_seed: int = 3) -> EdgeStream:
    """Complete graph K_n, streamed in a seeded random order."""
    return gnp(n, 2.0, graph_seed=0, order_seed=order_seed)


def shuffled(s: EdgeStream, order_seed: int) -> EdgeStream:
    """The same edges in another seeded uniform random order."""
    lib = _load()
    src = s.src.copy()
    dst = s.dst.copy()
    lib.gg_shuffle(_ptr(src), _ptr(dst), len(s), order_seed)
    return EdgeStream(src, dst, s.n_nodes, s.name + f"+order{order_seed}")


def pcg32_stream(initstate: int, initseq: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint32)
    lib.gg_pcg32_fill(initstate, initseq, _ptr(out), n)
    return out


# ---------------------------------------------------------------------------
# Named workloads.  Graph seed 42 and order seed 7 unless stated.
# ---------------------------------------------------------------------------
def powerlaw_20k() -> EdgeStream:
    """Chung-Lu, 20,000 nodes, exponent 2.3, 200,000 distinct edges."""
    return chung_lu(20_000, 2.3, 200_000)


def rmat_s20() -> EdgeStream:
    """R-MAT (0.57, 0.19, 0.19, 0.05), scale 20, 16 * 2^20 draws before dedup."""
    return rmat(20, 16)


def powerlaw_4m() -> EdgeStream:
    """Chung-Lu, 2^22 nodes, exponent 2.1, expected degree capped at 50,000, 64 * 2^20 distinct edges."""
    return chung_lu(1 << 22, 2.1, 64 << 20, cap=50_000.0)


_CACHE_DIR = os.environ.get("REPT_STREAM_CACHE", os.path.join(tempfile.gettempdir(), "rept_stream_cache"))


def cached(name: str) -> EdgeStream:
    """A named workload, cached as .npy files (git-ignored) after the first build."""
    makers = {"powerlaw_20k": (powerlaw_20k, 20_000), "rmat_s20": (rmat_s20, 1 << 20),
              "powerlaw_4m": (powerlaw_4m, 1 << 22)}
    fn, n = makers[name]
    d = os.path.join(_CACHE_DIR, name)
    ps, pd = os.path.join(d, "src.npy"), os.path.join(d, "dst.npy")
    if os.path.exists(ps) and os.path.exists(pd) and os.path.getmtime(ps) > os.path.getmtime(_SRC):
        return EdgeStream(np.load(ps), np.load(pd), n, name)
    s = fn()
    os.makedirs(d, exist_ok=True)
    np.save(ps + f".tmp{os.getpid()}.npy", s.src)
    np.save(pd + f".tmp{os.getpid()}.npy", s.dst)
    os.replace(ps + f".tmp{os.getpid()}.npy", ps)
    os.replace(pd + f".tmp{os.getpid()}.npy", pd)
    s.name = name
    return s
