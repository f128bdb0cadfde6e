"""Thin ctypes binding of librept.so (include/rept.h): argument marshalling only.

Every step of the counting path runs in the library's CUDA kernels.  PyTorch
supplies device memory and the current CUDA stream; nothing here computes a
count or an estimate.  If the library has not been built, or there is no
GPU, the constructors raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

REPT_OK = 0
ERRORS = {-1: "REPT_E_INVAL", -2: "REPT_E_RANGE", -3: "REPT_E_CAPACITY", -4: "REPT_E_NOMEM", -5: "REPT_E_CUDA",
          -6: "REPT_E_TIMEOUT", -7: "REPT_E_INTERNAL", -8: "REPT_E_SCRATCH", -9: "REPT_E_DUPLICATE"}
FLAG_FIXED_POOL = 1
FLAG_SYNC = 2
FLAG_PROFILE = 4
FLAG_WORK_COUNTERS = 8
FLAG_LOCAL_PER_PROCESSOR = 16
FLAG_MASCOT = 32
FLAG_CHECK_DUPS = 64
KERNELS = ("classify", "plan", "commit", "insert", "intersect", "estimate", "sort")


class ReptError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_lib_strerror(code)})")


class Config(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint32), ("c", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("n_nodes", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("expected_edges", ctypes.c_uint64),
                ("max_batch", ctypes.c_uint64), ("tile_max", ctypes.c_uint32), ("proc_begin", ctypes.c_uint32),
                ("proc_end", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("reserved2", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_uint64), ("self_loops", ctypes.c_uint64), ("stored_edges", ctypes.c_uint64),
                ("pool_slots", ctypes.c_uint64), ("pool_used", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("small_entries", ctypes.c_uint64), ("small_slots", ctypes.c_uint64), ("probes", ctypes.c_uint64),
                ("probe_slots", ctypes.c_uint64), ("wedges", ctypes.c_uint64), ("counted", ctypes.c_uint64),
                ("class_items", ctypes.c_uint64 * 6), ("class_probes", ctypes.c_uint64 * 6),
                ("class_cycles", ctypes.c_uint64 * 6)]


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64


def library_path() -> str:
    """The in-tree librept.so, or the library named by REPT_LIBRARY (e.g. the bounds-checked debug
    build, paper_1811_09136_gb300/librept_debug.so)."""
    return os.environ.get("REPT_LIBRARY") or _build.LIB_PATH


def load():
    """Load librept.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import "
                               "__graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        sig = {
            "rept_create": (ctypes.c_int, [ctypes.POINTER(Config), _vp, ctypes.POINTER(_vp)]),
            "rept_reset": (ctypes.c_int, [_vp, _vp]),
            "rept_reset_async": (ctypes.c_int, [_vp, _u64, _vp]),
            "rept_ingest_batch": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp]),
            "rept_ingest_host": (ctypes.c_int, [_vp, _vp, _vp, _u64, _u64, _vp]),
            "rept_estimates": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
            "rept_estimates_host": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
            "rept_estimates_async": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "rept_counts": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "rept_pair_counts": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
            "rept_local_per_processor": (ctypes.c_int, [_vp, _vp, _vp]),
            "rept_snapshot_size": (ctypes.c_int, [_vp, _vp, _vp]),
            "rept_snapshot": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
            "rept_restore": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
            "rept_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats), _vp]),
            "rept_sync": (ctypes.c_int, [_vp, _vp]),
            "rept_kernel_times": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
            "rept_destroy": (None, [_vp]),
            "rept_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "rept_kernel_launches": (ctypes.c_uint64, []),
            "rept_ingest_multi": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "rept_estimates_from_counts": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp,
                                                          ctypes.c_uint32, ctypes.POINTER(ctypes.c_double), _vp,
                                                          _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _lib_strerror(code: int) -> str:
    try:
        return load().rept_strerror(code).decode()
    except Exception:  # pragma: no cover - only for messages
        return "?"


def kernel_launches() -> int:
    return int(load().rept_kernel_launches())


def _check(code: int, where: str):
    if code != REPT_OK:
        raise ReptError(code, where)


def _cur_stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_u32(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
            and t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32))):
        raise TypeError("expected a contiguous CUDA tensor of 32-bit node ids")
    return ctypes.c_void_p(t.data_ptr())


def _host_u32(a: np.ndarray):
    if not (isinstance(a, np.ndarray) and a.dtype == np.uint32 and a.flags.c_contiguous):
        raise TypeError("expected a contiguous numpy uint32 array")
    return ctypes.c_void_p(a.ctypes.data)


class ReptStream:
    """One edge stream counted by REPT on the current CUDA device (see include/rept.h)."""

    def __init__(self, n_nodes: int, m: int, c: int, seed: int = 1, expected_edges: int = 0,
                 max_batch: int = 1 << 20, flags: int = 0, stream=None, tile_max: int = 0,
                 proc_range: tuple[int, int] | None = None):
        """``proc_range=(b, e)`` keeps processors b..e-1 only (a colour shard, see rept_config)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ReptStream needs a CUDA device; there is no CPU fallback")
        lib = load()
        self.n_nodes, self.m, self.c, self.seed = int(n_nodes), int(m), int(c), int(seed)
        self.flags = int(flags)
        b, e = proc_range if proc_range is not None else (0, 0)
        cfg = Config(self.m, self.c, self.seed, self.n_nodes, flags, expected_edges, max_batch, tile_max, b, e, 0, 0)
        h = ctypes.c_void_p()
        _check(lib.rept_create(ctypes.byref(cfg), _cur_stream(stream), ctypes.byref(h)), "rept_create")
        self._h = h
        self._lib = lib

    # ------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rept_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def reset(self, stream=None):
        _check(self._lib.rept_reset(self._h, _cur_stream(stream)), "rept_reset")

    def reset_async(self, seed: int | None = None, stream=None):
        """Clear the whole state without waiting (enqueued on `stream`); the next stream uses hash
        seed `seed` (default: unchanged)."""
        if seed is not None:
            self.seed = int(seed)
        _check(self._lib.rept_reset_async(self._h, self.seed, _cur_stream(stream)), "rept_reset_async")

    def ingest(self, src, dst, stream=None):
        """Append device edges (torch int32/uint32 CUDA tensors) as one batch (asynchronous)."""
        if src.numel() != dst.numel():
            raise ValueError("src and dst differ in length")
        _check(self._lib.rept_ingest_batch(self._h, _dev_u32(src), _dev_u32(dst), src.numel(),
                                           _cur_stream(stream)), "rept_ingest_batch")

    def ingest_host(self, src: np.ndarray, dst: np.ndarray, batch: int = 0, stream=None):
        """Append host edges (numpy uint32), copied and ingested in chunks of ``batch`` edges."""
        if src.size != dst.size:
            raise ValueError("src and dst differ in length")
        _check(self._lib.rept_ingest_host(self._h, _host_u32(src), _host_u32(dst), src.size, batch,
                                          _cur_stream(stream)), "rept_ingest_host")

    def sync(self, stream=None):
        _check(self._lib.rept_sync(self._h, _cur_stream(stream)), "rept_sync")

    def estimates(self, local: bool = True, stream=None):
        """(tau_hat, tau_hat_v as a float64 CUDA tensor or None)."""
        import torch
        g = ctypes.c_double()
        out = torch.empty(self.n_nodes, dtype=torch.float64, device="cuda") if local else None
        ptr = ctypes.c_void_p(out.data_ptr()) if local else None
        _check(self._lib.rept_estimates(self._h, ctypes.byref(g), ptr, _cur_stream(stream)), "rept_estimates")
        return g.value, out

    def estimates_host(self, out: np.ndarray | None = None, stream=None):
        """(tau_hat, tau_hat_v as a numpy float64 array written by the library)."""
        g = ctypes.c_double()
        if out is None:
            out = np.empty(self.n_nodes, dtype=np.float64)
        _check(self._lib.rept_estimates_host(self._h, ctypes.byref(g), ctypes.c_void_p(out.ctypes.data),
                                             _cur_stream(stream)), "rept_estimates_host")
        return g.value, out

    def estimates_async(self, h_global: np.ndarray, h_proc: np.ndarray, h_status: np.ndarray, stream=None):
        """Enqueue tau_hat, tau^(i) and the status word for copy into the given (pinned) numpy arrays
        of 1 float64, c uint64 and 1 uint32; they are valid once the stream passes this point."""
        _check(self._lib.rept_estimates_async(self._h, ctypes.c_void_p(h_global.ctypes.data),
                                              ctypes.c_void_p(h_proc.ctypes.data),
                                              ctypes.c_void_p(h_status.ctypes.data), _cur_stream(stream)),
               "rept_estimates_async")

    def counts(self, stream=None, allow_error: bool = False):
        """(tau^(i) as numpy uint64 [c], sum_i tau_v^(i) as an int64 CUDA tensor [n_nodes]).
        With ``allow_error`` the handle's sticky error code is returned as a third value
        instead of raised (the counters are those of the last batch that was applied)."""
        import torch
        proc = np.zeros(self.c, dtype=np.uint64)
        local = torch.empty(self.n_nodes, dtype=torch.int64, device="cuda")
        rc = self._lib.rept_counts(self._h, ctypes.c_void_p(proc.ctypes.data), ctypes.c_void_p(local.data_ptr()),
                                   _cur_stream(stream))
        if allow_error:
            return proc, local, rc
        _check(rc, "rept_counts")
        return proc, local

    def local_per_processor(self, stream=None):
        """tau_v^(i) of every processor as an int64 CUDA tensor [c, n_nodes] (needs FLAG_LOCAL_PER_PROCESSOR)."""
        import torch
        out = torch.empty((self.c, self.n_nodes), dtype=torch.int64, device="cuda")
        _check(self._lib.rept_local_per_processor(self._h, ctypes.c_void_p(out.data_ptr()), _cur_stream(stream)),
               "rept_local_per_processor")
        return out

    def snapshot(self, stream=None) -> np.ndarray:
        """The whole stream state as a host byte array (see rept_snapshot)."""
        n = ctypes.c_uint64()
        _check(self._lib.rept_snapshot_size(self._h, ctypes.byref(n), _cur_stream(stream)), "rept_snapshot_size")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(self._lib.rept_snapshot(self._h, ctypes.c_void_p(buf.ctypes.data), n.value, _cur_stream(stream)),
               "rept_snapshot")
        return buf

    def restore(self, buf: np.ndarray, stream=None):
        """Replace the state with a snapshot taken from a handle of the same configuration."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self._lib.rept_restore(self._h, ctypes.c_void_p(buf.ctypes.data), buf.size, _cur_stream(stream)),
               "rept_restore")

    def pair_counts(self, stream=None):
        """c > m with c mod m != 0 (Algorithm 2): (eta^(i) numpy uint64 [c], sum_i eta_v^(i),
        full-group local counts, partial-group local counts), the last three int64 CUDA tensors."""
        import torch
        eta = np.zeros(self.c, dtype=np.uint64)
        el, l1, l2 = (torch.empty(self.n_nodes, dtype=torch.int64, device="cuda") for _ in range(3))
        _check(self._lib.rept_pair_counts(self._h, ctypes.c_void_p(eta.ctypes.data), ctypes.c_void_p(el.data_ptr()),
                                          ctypes.c_void_p(l1.data_ptr()), ctypes.c_void_p(l2.data_ptr()),
                                          _cur_stream(stream)), "rept_pair_counts")
        return eta, el, l1, l2

    def stats(self, stream=None) -> dict:
        st = Stats()
        _check(self._lib.rept_get_stats(self._h, ctypes.byref(st), _cur_stream(stream)), "rept_get_stats")
        out = {}
        for k, _ in Stats._fields_:
            v = getattr(st, k)
            out[k] = [int(x) for x in v] if hasattr(v, "__len__") else int(v)
        return out

    def kernel_times(self, clear: bool = False) -> dict:
        """{kernel: (milliseconds, launches)} from CUDA events (needs FLAG_PROFILE)."""
        ms = (ctypes.c_double * len(KERNELS))()
        n = (ctypes.c_uint64 * len(KERNELS))()
        _check(self._lib.rept_kernel_times(self._h, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p),
                                           int(clear)), "rept_kernel_times")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}


def estimates_from_counts(m: int, c: int, proc: np.ndarray, local=None, flags: int = 0, stream=None):
    """rept_estimates_from_counts: (tau_hat, tau_hat_v as a float64 CUDA tensor or None) from integer
    counts, e.g. summed over colour shards.  ``proc``: numpy uint64 [c]; ``local``: int64 CUDA tensor
    of sum_i tau_v^(i) or None."""
    import torch
    lib = load()
    proc = np.ascontiguousarray(proc, dtype=np.uint64)
    if proc.size != c:
        raise ValueError("proc must hold c counters")
    g = ctypes.c_double()
    out = None
    if local is not None:
        out = torch.empty(local.numel(), dtype=torch.float64, device=local.device)
    _check(lib.rept_estimates_from_counts(m, c, flags, ctypes.c_void_p(proc.ctypes.data),
                                          ctypes.c_void_p(local.data_ptr()) if local is not None else None,
                                          local.numel() if local is not None else 0, ctypes.byref(g),
                                          ctypes.c_void_p(out.data_ptr()) if out is not None else None,
                                          _cur_stream(stream) if local is not None else None),
           "rept_estimates_from_counts")
    return g.value, out


def ingest_multi(handles, srcs, dsts, stream=None):
    """rept_ingest_multi: one batch per handle (srcs[i]/dsts[i] CUDA int32 tensors, possibly empty)
    through the library's own group for the current device."""
    lib = load()
    k = len(handles)
    hs = (ctypes.c_void_p * k)(*[h.handle.value for h in handles])
    a = (ctypes.c_void_p * k)(*[x.data_ptr() if x.numel() else None for x in srcs])
    b = (ctypes.c_void_p * k)(*[x.data_ptr() if x.numel() else None for x in dsts])
    n = (ctypes.c_uint64 * k)(*[x.numel() for x in srcs])
    _check(lib.rept_ingest_multi(ctypes.cast(hs, ctypes.c_void_p), ctypes.cast(a, ctypes.c_void_p),
                                 ctypes.cast(b, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p), k,
                                 _cur_stream(stream)), "rept_ingest_multi")
