"""Serving many REPT streams with continuous batching.

Requests (one edge stream each, with its own m, c and hash seed) arrive over time.  The server
admits a request as soon as it has arrived, a slot is free and its device state fits the HBM
budget (the paper's memory rule c* = min(c, floor(M / (p |E|))) read for whole streams: a stream is
admitted only if its state fits what is left of M); admitted streams stay resident and are fed in
chunks, all of them together through one rept_group per round, so requests that arrive while
others are on the GPU join the next round.  A finished stream's estimates are read back and its
memory released at once.

Each request's counts equal those of counting its stream alone (the streams share nothing on the
device but the launches).  The report gives per-request completion latency (arrival to estimates
on the host), its p50 / p99, and aggregate edges/s over the whole trace.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import batched, graphgen, rept


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the trace starts
    stream: graphgen.EdgeStream
    m: int
    c: int
    seed: int
    chunk: int = 1 << 18      # edges fed per round
    cancel_after: float = math.inf  # the client gives up this many seconds after arrival
    # filled in by the server
    cancelled: bool = False
    admitted: float = math.nan
    done: float = math.nan
    tau_hat: float = math.nan
    proc: np.ndarray | None = None
    local: np.ndarray | None = None


@dataclass
class _Live:
    req: Request
    handle: rept.ReptStream
    src: object
    dst: object
    fed: int = 0
    bytes: int = 0
    ready: object = None       # CUDA event: edges uploaded
    waited: bool = False       # the compute stream already waits for the upload
    out: tuple = ()            # pinned result buffers (tau_hat, tau^(i), status)
    done_ev: object = None     # CUDA event: results copied to the host (or, if cancelled, its rounds done)


@dataclass
class ServeReport:
    requests: list = field(default_factory=list)
    cancelled: list = field(default_factory=list)
    makespan: float = 0.0
    edges: int = 0
    rounds: int = 0
    max_live: int = 0

    def latencies(self) -> np.ndarray:
        return np.array([r.done - r.arrival for r in self.requests])

    def summary(self) -> dict:
        lat = self.latencies()
        return {"requests": len(self.requests), "cancelled": len(self.cancelled), "edges": self.edges,
                "makespan_s": self.makespan,
                "edges_per_s": self.edges / self.makespan if self.makespan > 0 else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "rounds": self.rounds, "max_live": self.max_live}


def poisson_arrivals(n: int, rate: float, seed: int = 5) -> np.ndarray:
    """Arrival times of a Poisson process with `rate` requests per second (exponential gaps from PCG32)."""
    u = graphgen.pcg32_stream(seed, 99, n).astype(np.float64)
    u = (u + 0.5) / 4294967296.0
    return np.cumsum(-np.log(u) / rate)


def serve(requests: list[Request], max_live: int = 256, budget_bytes: int | None = None,
          graph: bool = False, keep_local: bool = False, clock=time.perf_counter,
          free_batch: int = 16) -> ServeReport:
    """Run the trace.  Requests must be sorted by arrival time.

    A finished stream's estimates are requested asynchronously (rept_estimates_async into pinned
    memory, completion seen through a CUDA event), so the next round starts at once.  Finished
    handles are kept and reused (rept_reset_async) by later streams of the same shape; they are
    destroyed only when admission needs their memory, because releasing device memory waits for
    the whole device.

    A request whose client gives up (``cancel_after`` seconds after its arrival) before its last
    chunk was fed is cancelled: dropped if it is still waiting, otherwise no longer fed, and its
    handle becomes a spare once its rounds already on the GPU have finished.  Cancelled requests
    are listed in ``report.cancelled`` with no estimates; the others are unaffected."""
    import torch

    torch.cuda.synchronize()
    budget = budget_bytes if budget_bytes is not None else batched._device_budget()
    group = batched.ReptGroup(max_live, graph=graph)
    copy_stream = torch.cuda.Stream()
    compute = torch.cuda.current_stream()
    pending = list(requests)
    pending.reverse()          # pop() from the end = earliest arrival
    live: list[_Live] = []
    completing: list[_Live] = []
    graveyard: list[_Live] = []
    used = 0
    rep = ServeReport()
    pinned: dict[int, tuple] = {}
    spare: dict[tuple, list] = {}   # finished handles kept for reuse, by shape

    def feed(r):
        # edges fed per round: the request's chunk, raised for long streams so that a stream needs at
        # most about 256 rounds, and never above 2^20
        return min(max(1, len(r.stream)), max(r.chunk, min(1 << 20, len(r.stream) // 256)))

    def shape(r):
        return (r.stream.n_nodes, r.m, r.c, len(r.stream), feed(r))

    def release_graveyard():
        # finished handles become spares for a later stream of the same shape (their memory stays
        # counted); spares are destroyed only when admission needs the memory
        for x in graveyard:
            spare.setdefault(shape(x.req), []).append(x)
        graveyard.clear()

    def destroy_spares():
        nonlocal used
        for lst in spare.values():
            for x in lst:
                x.handle.close()
                used -= x.bytes
        spare.clear()

    def host_edges(r):
        key = id(r.stream)
        if key not in pinned:
            pinned[key] = (torch.from_numpy(r.stream.src.view(np.int32)).pin_memory(),
                           torch.from_numpy(r.stream.dst.view(np.int32)).pin_memory())
        return pinned[key]

    t0 = clock()
    while pending or live or completing:
        now = clock() - t0
        # cancellations: live requests stop being fed; their rounds in flight finish first
        for x in [x for x in live if now >= x.req.arrival + x.req.cancel_after]:
            x.req.cancelled = True
            x.done_ev = torch.cuda.Event()
            x.done_ev.record(compute)
            x.src = x.dst = None
            live.remove(x)
            completing.append(x)
        # results whose copies have landed
        for x in [x for x in completing if x.done_ev.query()]:
            r = x.req
            if r.cancelled:
                r.done = clock() - t0
                rep.cancelled.append(r)
                completing.remove(x)
                graveyard.append(x)
                continue
            g, proc, status = x.out
            if int(status[0]) != 0:
                x.handle.sync()  # raises the handle's REPT_E_* error
            r.tau_hat = float(g[0])
            r.proc = proc.copy()
            if keep_local:
                _, local = x.handle.counts()
                r.local = local.cpu().numpy().view(np.uint64)
            r.done = clock() - t0
            rep.edges += len(r.stream)
            rep.requests.append(r)
            completing.remove(x)
            graveyard.append(x)
        if len(graveyard) >= free_batch:
            release_graveyard()
        # admission: arrived, a slot free, state fits the remaining budget (FIFO, no overtaking)
        while pending and pending[-1].arrival <= now and len(live) < max_live:
            r = pending[-1]
            if now >= r.arrival + r.cancel_after:  # given up before it was admitted
                pending.pop()
                r.cancelled = True
                r.done = now
                rep.cancelled.append(r)
                continue
            need = batched._state_bytes(r.stream.n_nodes, len(r.stream), feed(r)) + 8 * len(r.stream)
            reuse = spare.get(shape(r))
            if reuse:
                pending.pop()
                old = reuse.pop()
                h = old.handle
                need = old.bytes
                used -= old.bytes
                h.reset_async(seed=r.seed, stream=copy_stream)
            else:
                if (live or completing or spare) and used + need > budget:
                    if graveyard or spare:
                        release_graveyard()
                        destroy_spares()
                        continue
                    break
                pending.pop()
                # state set-up and the edge upload go on the copy stream, next to the running rounds
                h = rept.ReptStream(r.stream.n_nodes, r.m, r.c, r.seed, expected_edges=len(r.stream),
                                    max_batch=feed(r), stream=copy_stream)
            hsrc, hdst = host_edges(r)
            with torch.cuda.stream(copy_stream):
                src = hsrc.to("cuda", non_blocking=True)
                dst = hdst.to("cuda", non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            src.record_stream(compute)
            dst.record_stream(compute)
            r.admitted = clock() - t0
            live.append(_Live(r, h, src, dst, bytes=need, ready=ev))
            used += need
        rep.max_live = max(rep.max_live, len(live))
        ready = [x for x in live if x.waited or x.ready.query()]
        if not ready:
            if live:
                live[0].ready.synchronize()
            elif completing:
                completing[0].done_ev.synchronize()
            elif pending:
                wait = pending[-1].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
            continue
        # one round: every ready stream gets its next chunk, all in one group launch sequence
        hs, a, b = [], [], []
        for x in ready:
            if not x.waited:
                compute.wait_event(x.ready)
                x.waited = True
            n = min(feed(x.req), len(x.req.stream) - x.fed)
            hs.append(x.handle)
            a.append(x.src[x.fed:x.fed + n])
            b.append(x.dst[x.fed:x.fed + n])
            x.fed += n
        group.ingest(hs, a, b)
        rep.rounds += 1
        for x in [x for x in ready if x.fed >= len(x.req.stream)]:
            x.out = (torch.empty(1, dtype=torch.float64).pin_memory().numpy(),
                     torch.empty(x.req.c, dtype=torch.int64).pin_memory().numpy().view(np.uint64),
                     torch.empty(1, dtype=torch.int32).pin_memory().numpy().view(np.uint32))
            x.handle.estimates_async(*x.out)
            x.done_ev = torch.cuda.Event()
            x.done_ev.record(compute)
            x.src = x.dst = None
            live.remove(x)
            completing.append(x)
    torch.cuda.synchronize()
    rep.makespan = clock() - t0
    release_graveyard()
    destroy_spares()
    group.close()
    rep.requests.sort(key=lambda r: r.rid)
    rep.cancelled.sort(key=lambda r: r.rid)
    return rep


def count_alone(r: Request):
    """The request's stream counted on its own with the single-stream path (for comparison)."""
    import torch
    with rept.ReptStream(r.stream.n_nodes, r.m, r.c, r.seed, expected_edges=len(r.stream),
                         max_batch=min(r.chunk, max(1, len(r.stream)))) as h:
        src = torch.from_numpy(r.stream.src.view(np.int32)).cuda()
        dst = torch.from_numpy(r.stream.dst.view(np.int32)).cuda()
        for off in range(0, len(r.stream), r.chunk):
            h.ingest(src[off:off + r.chunk], dst[off:off + r.chunk])
        g, _ = h.estimates(local=False)
        proc, local = h.counts()
        return g, proc, local.cpu().numpy().view(np.uint64)


def build_trace(n_requests: int = 1000, rate: float = 200.0, distinct: int = 64, big_every: int = 50,
                big_scale: int = 24, seed: int = 5, chunk_choices=(1 << 16, 1 << 18, 1 << 20),
                mix_kwargs=None, processes=None) -> list[Request]:
    """The serving workload: Poisson arrivals at `rate`/s; each request's stream is drawn from
    `distinct` streams of the batched mix (its own hash seed, p from the mix with c = m), and every
    `big_every`-th request is an R-MAT scale-`big_scale`, edge-factor-16 stream with p = 0.01,
    c = 100.  Chunk sizes are drawn from `chunk_choices`."""
    mix_kwargs = mix_kwargs or {}
    specs = batched.mix_specs(distinct, seed=seed * 1000, **mix_kwargs)
    streams = batched.generate_all(specs, processes=processes)
    big = graphgen.rmat(big_scale, 16, graph_seed=seed, order_seed=seed + 1) if big_every else None
    arrivals = poisson_arrivals(n_requests, rate, seed)
    pick = graphgen.pcg32_stream(seed, 123, 2 * n_requests)
    reqs = []
    for i in range(n_requests):
        chunk = chunk_choices[int(pick[2 * i + 1]) % len(chunk_choices)]
        if big_every and (i + 1) % big_every == 0:
            reqs.append(Request(i, float(arrivals[i]), big, 100, 100, 7000 + i, chunk))
        else:
            sp = specs[int(pick[2 * i]) % distinct]
            reqs.append(Request(i, float(arrivals[i]), streams[sp.index], sp.m, sp.m, 7000 + i, chunk))
    return reqs
