"""Colour sharding: one stream counted by several GPUs, each keeping a share of the processors.

REPT's processors share nothing until the final sums (Algorithm 1: processor i keeps the edges of
its colour and counts the wedges of its own edges).  So c processors can be split among G GPUs:
GPU g keeps processors J_g (a range of colours, or whole hash groups when c > m), ingests the whole
stream, stores only the edges its processors keep and counts only their semi-triangles.  One
exchange step remains: tau^(i) comes from the GPU that keeps i, and sum_i tau_v^(i) is the sum over
GPUs of their local counts, a uint64 all-reduce.  The estimates are then formed from the summed
counts exactly as one GPU holding every processor would form them (rept_estimates_from_counts).
Algorithm 2's case (c > m, c mod m != 0) combines its counts non-linearly and is not sharded.

This module holds the host side: the partition rule, the reduction over a torch.distributed
process group (NCCL for CUDA tensors, gloo for CPU tensors), and a stream wrapper that does both
around a rept handle created with its processor range.
"""
from __future__ import annotations

import numpy as np


def shard_range(c: int, m: int, world: int, rank: int, mascot: bool = False) -> tuple[int, int]:
    """Processors [b, e) of rank `rank` out of `world`: whole hash groups (m processors each, one
    for parallel MASCOT) when there are at least as many groups as ranks, else near-equal ranges of
    processors.  The ranges of ranks 0..world-1 are disjoint and cover 0..c-1; a range may be empty
    when world > c."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    stride = 1 if mascot else m
    groups = -(-c // stride)
    if groups >= world and groups > 1:
        g0, g1 = groups * rank // world, groups * (rank + 1) // world
        return min(c, g0 * stride), min(c, g1 * stride)
    return c * rank // world, c * (rank + 1) // world


def reduce_counts(proc: np.ndarray, local, pg, device=None):
    """Sum the shards' counts over the process group `pg` (torch.distributed): `proc` (numpy uint64
    [c], zero outside the rank's processors) and `local` (int64 tensor [n_nodes] holding uint64
    values; reduced in place).  uint64 sums are exact modulo 2^64 through int64 two's complement.
    Returns the summed (proc, local)."""
    import torch
    if pg is None:
        return proc, local
    dev = device if device is not None else local.device
    p = torch.from_numpy(np.ascontiguousarray(proc, dtype=np.uint64).view(np.int64).copy()).to(dev)
    pg.all_reduce(p, op=pg.ReduceOp.SUM)
    pg.all_reduce(local, op=pg.ReduceOp.SUM)
    return p.cpu().numpy().view(np.uint64), local


class ShardedStream:
    """A stream whose c processors are spread over the ranks of `pg`; every rank ingests the whole
    stream into a handle that keeps its own processors (rept_config.proc_begin / proc_end)."""

    def __init__(self, n_nodes: int, m: int, c: int, seed: int, world: int, rank: int, pg=None,
                 flags: int = 0, **kw):
        from . import rept
        self.n_nodes, self.m, self.c, self.flags = n_nodes, m, c, flags
        self.pg = pg
        self.range = shard_range(c, m, world, rank, mascot=bool(flags & rept.FLAG_MASCOT))
        b, e = self.range
        # an empty share (more ranks than processors) ingests nothing and adds zeros
        self.h = rept.ReptStream(n_nodes, m, c, seed, flags=flags, proc_range=(b, e), **kw) if e > b else None

    def ingest(self, src, dst, stream=None):
        if self.h is not None:
            self.h.ingest(src, dst, stream=stream)

    def reset(self):
        if self.h is not None:
            self.h.reset()

    def counts(self):
        """The counts summed over all ranks: (tau^(i) numpy uint64 [c], sum_i tau_v^(i) int64 CUDA tensor)."""
        import torch
        if self.h is not None:
            proc, local = self.h.counts()
        else:
            proc = np.zeros(self.c, dtype=np.uint64)
            local = torch.zeros(self.n_nodes, dtype=torch.int64, device="cuda")
        return reduce_counts(proc, local, self.pg)

    def estimates(self, local: bool = True):
        """(tau_hat, tau_hat_v or None) of the whole stream, from the summed counts."""
        from . import rept
        proc, loc = self.counts()
        return rept.estimates_from_counts(self.m, self.c, proc, loc if local else None, flags=self.flags)

    def close(self):
        if self.h is not None:
            self.h.close()
            self.h = None
