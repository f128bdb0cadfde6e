"""Many independent streams counted side by side: the batched path and its plain-loop comparison.

`ReptGroup` binds the C ABI's rept_group (one kernel launch per step of the batch path for all
streams, optionally replayed from a CUDA graph).  `run_batched` feeds every stream of a mix chunk
by chunk through one group; `run_plain` counts the same streams one after the other with the
single-stream path.  Both admit streams in waves that fit a device-memory budget, keep the
handles' state resident while a stream is open, and return each stream's integer counts and
estimates, which must be identical between the two.

The stream mix follows the batched workload: each stream is an R-MAT graph (a, b, c, d) =
(0.57, 0.19, 0.19, 0.05) or a Chung-Lu graph with exponent in [2.1, 2.5], with a node count
log-uniform in [1e4, 2e6] and 10-40 edges per node, and p drawn from {0.1, 0.05, 0.01} with
c = m = 1/p.  The draws come from PCG32 so that the mix is the same on every machine.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import graphgen, rept

GROUP_GRAPH = 1
GROUP_PERSISTENT = 2
GROUP_TEST_TIMEOUT = 4


class ReptGroup:
    """Binding of rept_group_create / rept_group_ingest / rept_group_destroy.  With `persistent`
    every call is one cooperative launch running all steps for all streams (REPT_GROUP_PERSISTENT);
    `test_timeout` is the test hook that makes its first grid-wide wait run out."""

    def __init__(self, max_streams: int, graph: bool = True, persistent: bool = False, test_timeout: bool = False):
        lib = rept.load()
        lib.rept_group_create.restype = ctypes.c_int
        lib.rept_group_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]
        lib.rept_group_ingest.restype = ctypes.c_int
        lib.rept_group_ingest.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
        lib.rept_group_destroy.restype = None
        lib.rept_group_destroy.argtypes = [ctypes.c_void_p]
        self._lib = lib
        self.max_streams = int(max_streams)
        h = ctypes.c_void_p()
        flags = (GROUP_GRAPH if graph else 0) | (GROUP_PERSISTENT if persistent else 0) | \
            (GROUP_TEST_TIMEOUT if test_timeout else 0)
        rept._check(lib.rept_group_create(max_streams, flags, ctypes.byref(h)), "rept_group_create")
        self._h = h
        self._hs = (ctypes.c_void_p * max_streams)()
        self._src = (ctypes.c_void_p * max_streams)()
        self._dst = (ctypes.c_void_p * max_streams)()
        self._n = (ctypes.c_uint64 * max_streams)()

    def ingest(self, handles, srcs, dsts, stream=None):
        """One batch per handle: srcs[i]/dsts[i] are CUDA int32 tensors (possibly empty)."""
        k = len(handles)
        if k > self.max_streams:
            raise ValueError("more streams than the group was created for")
        for i, (h, a, b) in enumerate(zip(handles, srcs, dsts)):
            self._hs[i] = h.handle.value
            n = a.numel()
            self._n[i] = n
            self._src[i] = a.data_ptr() if n else None
            self._dst[i] = b.data_ptr() if n else None
        rept._check(self._lib.rept_group_ingest(self._h, ctypes.cast(self._hs, ctypes.c_void_p),
                                                ctypes.cast(self._src, ctypes.c_void_p),
                                                ctypes.cast(self._dst, ctypes.c_void_p),
                                                ctypes.cast(self._n, ctypes.c_void_p), k,
                                                rept._cur_stream(stream)), "rept_group_ingest")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rept_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- workload mix
@dataclass
class StreamSpec:
    index: int
    kind: str          # "rmat" or "chung_lu"
    n_nodes: int
    edges_per_node: float
    gamma: float       # Chung-Lu exponent (unused for R-MAT)
    m: int             # 1/p; c = m
    graph_seed: int
    order_seed: int
    hash_seed: int

    def generate(self) -> graphgen.EdgeStream:
        if self.kind == "rmat":
            scale = max(1, int(round(math.log2(self.n_nodes))))
            s = graphgen.rmat(scale, int(round(self.edges_per_node)), graph_seed=self.graph_seed,
                              order_seed=self.order_seed)
        else:
            s = graphgen.chung_lu(self.n_nodes, self.gamma, int(round(self.n_nodes * self.edges_per_node)),
                                  graph_seed=self.graph_seed, order_seed=self.order_seed)
        s.name = f"{self.kind}#{self.index}"
        return s


def mix_specs(n_streams: int = 256, seed: int = 1000, n_min: float = 1e4, n_max: float = 2e6,
              epn=(10.0, 40.0)) -> list[StreamSpec]:
    """The batched workload's stream parameters, drawn from PCG32(seed)."""
    r = graphgen.pcg32_stream(seed, 77, 8 * n_streams).astype(np.float64) / 4294967296.0
    specs = []
    for i in range(n_streams):
        u = r[8 * i: 8 * i + 8]
        kind = "rmat" if u[0] < 0.5 else "chung_lu"
        n = int(round(math.exp(math.log(n_min) + u[1] * (math.log(n_max) - math.log(n_min)))))
        e = epn[0] + u[2] * (epn[1] - epn[0])
        gamma = 2.1 + 0.4 * u[3]
        m = (10, 20, 100)[min(2, int(u[4] * 3))]
        specs.append(StreamSpec(i, kind, n, e, gamma, m, graph_seed=seed + 2 * i, order_seed=seed + 2 * i + 1,
                                hash_seed=seed + i))
    return specs


def _gen(spec: StreamSpec):
    s = spec.generate()
    return spec.index, s.src, s.dst, s.n_nodes


def generate_all(specs: list[StreamSpec], processes: int | None = None) -> list[graphgen.EdgeStream]:
    """Generate every stream of a mix, in parallel worker processes (spawned, never forked)."""
    import multiprocessing as mp
    graphgen.build()
    out = [None] * len(specs)
    procs = processes or min(len(specs), os.cpu_count() or 1)
    if procs <= 1 or len(specs) == 1:
        for sp in specs:
            out[sp.index - specs[0].index] = sp.generate()
        return out
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for idx, src, dst, n in pool.imap_unordered(_gen, sorted(specs, key=lambda s: -s.n_nodes * s.edges_per_node)):
            out[idx - specs[0].index] = graphgen.EdgeStream(src, dst, n, f"stream#{idx}")
    return out


# --------------------------------------------------------------------------- runners
@dataclass
class StreamResult:
    proc: np.ndarray      # tau^(i), uint64 [c]
    local: np.ndarray     # sum_i tau_v^(i), uint64 [n]
    tau_hat: float
    local_hat: np.ndarray | None


def _state_bytes(n_nodes: int, edges: int, batch: int) -> int:
    """Device bytes a stream's state needs: per-node arrays, per-batch scratch, and the pool at the
    guaranteed bound (32 slots of 8 bytes per edge)."""
    return 28 * n_nodes + 200_000 + 96 * batch + 256 * edges + (1 << 20)


def _waves(streams, batch, budget):
    wave, used = [], 0
    for i, s in enumerate(streams):
        b = _state_bytes(s.n_nodes, len(s), min(batch, len(s))) + 8 * len(s)
        if wave and used + b > budget:
            yield wave
            wave, used = [], 0
        wave.append(i)
        used += b
    if wave:
        yield wave


def _device_budget(frac=0.6):
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free * frac)


def _collect(h, local_estimates):
    proc, local = h.counts()
    g, loc = h.estimates(local=local_estimates)
    return StreamResult(proc, local.cpu().numpy().view(np.uint64), g,
                        None if loc is None else loc.cpu().numpy())


def _pinned(a: np.ndarray):
    import torch
    return torch.from_numpy(a.view(np.int32)).pin_memory()


def _result_buffers(c: int):
    """Pinned host buffers for rept_estimates_async: tau_hat, tau^(i), status word."""
    import torch
    return (torch.empty(1, dtype=torch.float64).pin_memory().numpy(),
            torch.empty(c, dtype=torch.int64).pin_memory().numpy().view(np.uint64),
            torch.empty(1, dtype=torch.int32).pin_memory().numpy().view(np.uint32))


def run_batched(streams, params, batch: int = 1 << 18, tile_max: int = 32, graph: bool = True,
                budget: int | None = None, local_estimates: bool = False, presize: bool = True,
                host_io: bool = False, persistent: bool = False):
    """All streams through one rept_group, batch edges per stream per round.  `params[i]` is
    (m, c, seed).  With `presize` every pool is sized for its whole stream up front (no round needs
    a pool check); without it pools start small and grow (one host check per round).  With
    `host_io` the timed region also holds the copy of every stream's edges from pinned host memory
    to the device and the copy of each stream's tau_hat, tau^(i) and status word back to pinned
    host memory (end to end).  With `persistent` each round is one cooperative launch of every step
    for every stream.  Returns (results, seconds of device work incl. per-round host launch cost)."""
    import torch
    budget = budget or _device_budget()
    results = [None] * len(streams)
    total = 0.0
    for wave in _waves(streams, batch, budget):
        handles, srcs, dsts, hsrc, hdst, outs = [], [], [], [], [], []
        for i in wave:
            s = streams[i]
            m, c, seed = params[i]
            handles.append(rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=len(s) if presize else 0,
                                           max_batch=min(batch, max(1, len(s))), tile_max=tile_max))
            if host_io:
                hsrc.append(_pinned(s.src))
                hdst.append(_pinned(s.dst))
                outs.append(_result_buffers(c))
            else:
                srcs.append(torch.from_numpy(s.src.view(np.int32)).cuda())
                dsts.append(torch.from_numpy(s.dst.view(np.int32)).cuda())
        group = ReptGroup(len(wave), graph=graph, persistent=persistent)
        rounds = max((len(streams[i]) + batch - 1) // batch for i in wave)
        torch.cuda.synchronize()
        t = time.perf_counter()
        if host_io:
            srcs = [x.to("cuda", non_blocking=True) for x in hsrc]
            dsts = [x.to("cuda", non_blocking=True) for x in hdst]
        for r in range(rounds):
            # only the streams that still have edges take part, so the finished ones free their SMs
            live = [j for j, x in enumerate(srcs) if r * batch < x.numel()]
            group.ingest([handles[j] for j in live], [srcs[j][r * batch:(r + 1) * batch] for j in live],
                         [dsts[j][r * batch:(r + 1) * batch] for j in live])
        if host_io:
            for h, o in zip(handles, outs):
                h.estimates_async(*o)
        for h in handles:
            h.sync()
        torch.cuda.synchronize()
        total += time.perf_counter() - t
        for j, i in enumerate(wave):
            if host_io:
                assert int(outs[j][2][0]) == 0, "device error"
            results[i] = _collect(handles[j], local_estimates)
            handles[j].close()
        group.close()
        del srcs, dsts, hsrc, hdst
    return results, total


def run_plain(streams, params, batch: int = 1 << 18, tile_max: int = 32, budget: int | None = None,
              local_estimates: bool = False):
    """The same streams counted one after the other with the single-stream path."""
    import torch
    budget = budget or _device_budget()
    results = [None] * len(streams)
    total = 0.0
    for wave in _waves(streams, batch, budget):
        handles, srcs, dsts = [], [], []
        for i in wave:
            s = streams[i]
            m, c, seed = params[i]
            handles.append(rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=len(s),
                                           max_batch=min(batch, max(1, len(s))), tile_max=tile_max))
            srcs.append(torch.from_numpy(s.src.view(np.int32)).cuda())
            dsts.append(torch.from_numpy(s.dst.view(np.int32)).cuda())
        torch.cuda.synchronize()
        t = time.perf_counter()
        for h, a, b in zip(handles, srcs, dsts):
            for off in range(0, a.numel(), batch):
                h.ingest(a[off:off + batch], b[off:off + batch])
        for h in handles:
            h.sync()
        torch.cuda.synchronize()
        total += time.perf_counter() - t
        for j, i in enumerate(wave):
            results[i] = _collect(handles[j], local_estimates)
            handles[j].close()
        del srcs, dsts
    return results, total


# --------------------------------------------------------------------------- autotuner
_CACHE = os.environ.get("REPT_AUTOTUNE_CACHE",
                        os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json"))


def _device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}"


def autotune(streams, params, batches=(1 << 16, 1 << 18, 1 << 20), tiles=(16, 32), key: str = "mix",
             use_cache: bool = True, repeat: int = 2):
    """Pick (batch, tile_max) for the batched path by timing each candidate on `streams` (a sample of
    the workload); the winner is cached per device and key in a JSON file."""
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    ck = f"{_device_key()}|{key}"
    if use_cache and ck in cache:
        return cache[ck]["batch"], cache[ck]["tile_max"], cache[ck]["timings"]
    timings = {}
    for b in batches:
        for tm in tiles:
            best = min(run_batched(streams, params, batch=b, tile_max=tm)[1] for _ in range(repeat))
            timings[f"{b},{tm}"] = best
    b, tm = min(timings, key=timings.get).split(",")
    cache[ck] = {"batch": int(b), "tile_max": int(tm), "timings": timings}
    if use_cache:
        tmp = _CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, _CACHE)
    return int(b), int(tm), timings
