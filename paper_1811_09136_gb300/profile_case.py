"""One pass of a stream through the C ABI and nothing else: the command to run under a profiler.

  python -m paper_1811_09136_gb300.profile_case --workload rmat_s20 --m 100 --c 100
  python -m paper_1811_09136_gb300.profile_case --chung-lu 1048576 2.1 16777216 50000 --m 20 --c 100
  python -m paper_1811_09136_gb300.profile_case --mix 32 --batch 1048576 --mode group

The stream is ingested once in batches of --batch edges into a handle whose pool grows as needed, so
that the device holds little beyond the state the stream needs.  Kernel launches per batch follow
the library's launch order (classify, plan, commit, two block-move kernels, insert, two sort
kernels, intersect), which is what a profiler's launch skip count (-s) refers to.  With --mix N the
first N streams of the batched workload's mix (seed 1000) are counted instead, each with its own
m = c and hash seed, through one rept_group (--mode group: one launch per step for all streams;
persistent: one cooperative launch per round) or one stream after the other (--mode plain).
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default=None, help="a named workload of graphgen.cached")
    ap.add_argument("--chung-lu", nargs=4, type=float, default=None, metavar=("N", "GAMMA", "EDGES", "CAP"))
    ap.add_argument("--m", type=int, default=100)
    ap.add_argument("--c", type=int, default=100)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--batch", type=int, default=1 << 20)
    ap.add_argument("--work", action="store_true",
                    help="with work counters (REPT_FLAG_WORK_COUNTERS), printing each batch's scanned entries")
    ap.add_argument("--mix", type=int, default=0, help="count the first N streams of the batched mix instead")
    ap.add_argument("--mode", default="group", choices=["group", "persistent", "plain"])
    args = ap.parse_args()

    import torch
    from . import graphgen, rept

    if args.mix:
        from . import batched
        specs = batched.mix_specs(args.mix, seed=1000)
        streams = batched.generate_all(specs)
        params = [(sp.m, sp.m, sp.hash_seed) for sp in specs]
        if args.mode == "plain":
            res, t = batched.run_plain(streams, params, batch=args.batch)
        else:
            res, t = batched.run_batched(streams, params, batch=args.batch, graph=False,
                                         persistent=args.mode == "persistent")
        print(f"{sum(len(x) for x in streams)} edges in {len(streams)} streams, "
              f"{sum(int(r.proc.sum()) for r in res)} semi-triangles, {t:.3f} s", flush=True)
        return

    if args.chung_lu:
        n, gamma, e, cap = args.chung_lu
        s = graphgen.chung_lu(int(n), gamma, int(e), cap=cap)
    else:
        s = graphgen.cached(args.workload or "rmat_s20")
    src = torch.from_numpy(s.src.view(np.int32)).cuda()
    dst = torch.from_numpy(s.dst.view(np.int32)).cuda()
    flags = rept.FLAG_WORK_COUNTERS if args.work else 0
    with rept.ReptStream(s.n_nodes, args.m, args.c, args.seed, max_batch=args.batch, flags=flags) as r:
        prev = 0
        for b, off in enumerate(range(0, len(s), args.batch)):
            r.ingest(src[off:off + args.batch], dst[off:off + args.batch])
            if args.work:  # the intersection's scanned entries of this batch (one launch)
                st = r.stats()
                print(f"batch {b}: {st['small_entries'] - prev} small-side entries, probes so far {st['probes']}")
                prev = st["small_entries"]
        proc, _ = r.counts()
        st = r.stats()
    print(f"{len(s)} edges, {int(proc.sum())} semi-triangles, pool {st['pool_used']} slots used", flush=True)


if __name__ == "__main__":
    main()
