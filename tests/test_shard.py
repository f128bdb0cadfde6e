"""Colour sharding (processors split among GPUs, Algorithm 1's processors being independent until the
final sums): the partition rule, the uint64 reduction over two gloo ranks on CPU, and, on the GPU,
shards run one after another whose summed counts equal one unsharded handle's and the oracle's."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1811_09136_gb300 import graphgen as gg
from paper_1811_09136_gb300 import shard

CASES = [(10, 10, False), (4, 3, False), (4, 8, False), (5, 20, False), (4, 6, True)]


@pytest.mark.parametrize("m,c,mascot", CASES)
def test_shard_ranges_cover_every_processor_once(m, c, mascot):
    for world in (1, 2, 3, 4, 7, 25):
        seen = np.zeros(c, dtype=int)
        for r in range(world):
            b, e = shard.shard_range(c, m, world, r, mascot)
            assert 0 <= b <= e <= c
            seen[b:e] += 1
            stride = 1 if mascot else m
            if -(-c // stride) >= world > 1:      # whole hash groups
                assert b % stride == 0 and (e % stride == 0 or e == c)
        assert (seen == 1).all(), (m, c, world, seen)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle as O
    from paper_1811_09136_gb300 import graphgen as gg
    from paper_1811_09136_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    s = gg.chung_lu(1500, 2.2, 9000, graph_seed=5, order_seed=6)
    for m, c, mascot in CASES:
        run = O.mascot_stream if mascot else O.rept_stream
        kw = {} if mascot else {"pair_counters": False}
        full = run(s.src, s.dst, s.n_nodes, m, c, 17, per_proc_local=True, **kw)
        # this rank's shard: the processors of its range (the oracle's per-processor counts)
        b, e = shard.shard_range(c, m, world, rank, mascot)
        proc = np.zeros(c, dtype=np.uint64)
        proc[b:e] = full.tau_proc[b:e]
        local = torch.from_numpy(full.tau_local_proc[b:e].sum(axis=0).astype(np.uint64).view(np.int64).copy())
        # a count above 2^63 must survive the int64 reduction
        if rank == 0:
            local[0] += torch.tensor(-(1 << 62), dtype=torch.int64) * 2  # + 2^63 as uint64
        rp, rl = shard.reduce_counts(proc, local, dist, device="cpu")
        rl = rl.numpy().view(np.uint64).copy()
        rl[0] -= np.uint64(1 << 63)
        out.append((bool(np.array_equal(rp, full.tau_proc)), bool(np.array_equal(rl, full.local1))))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_reduce_shard_counts_to_the_unsharded_oracle():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out in res:
        assert all(a and b for a, b in out), (rank, out)


def test_estimates_from_summed_counts_equal_the_oracle():
    """The global estimate formed by the library from summed shard counts is the oracle's."""
    from paper_1811_09136_gb300 import rept
    s = gg.chung_lu(1500, 2.2, 9000, graph_seed=5, order_seed=6)
    for m, c, mascot in CASES:
        if mascot:
            a = O.mascot_stream(s.src, s.dst, s.n_nodes, m, c, 17)
            ref_g, _ = O.mascot_estimates(m, c, a, s.n_nodes)
        else:
            a = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 17, pair_counters=False)
            ref_g, _ = O.estimates(m, c, a, s.n_nodes)
        g, _ = rept.estimates_from_counts(m, c, a.tau_proc, None, flags=rept.FLAG_MASCOT if mascot else 0)
        assert abs(g - ref_g) <= 1e-12 * max(abs(ref_g), 1.0), (m, c, g, ref_g)


@pytest.mark.gpu
@pytest.mark.parametrize("m,c,mascot", CASES)
def test_shards_one_after_another_sum_to_the_unsharded_counts(m, c, mascot):
    import torch
    from paper_1811_09136_gb300 import rept
    from gpu_helpers import device_edges
    s = gg.cached("powerlaw_20k")
    flags = rept.FLAG_MASCOT if mascot else 0
    src, dst = device_edges(s)
    with rept.ReptStream(s.n_nodes, m, c, 3, flags=flags, max_batch=1 << 16) as r:
        for off in range(0, len(s), 1 << 16):
            r.ingest(src[off:off + (1 << 16)], dst[off:off + (1 << 16)])
        full_proc, full_local = r.counts()
        full_g, full_loc = r.estimates()
    if mascot:
        ref = O.mascot_stream(s.src, s.dst, s.n_nodes, m, c, 3)
        ref_g, ref_loc = O.mascot_estimates(m, c, ref, s.n_nodes)
    else:
        ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 3, pair_counters=False)
        ref_g, ref_loc = O.estimates(m, c, ref, s.n_nodes)
    assert np.array_equal(full_proc, ref.tau_proc)
    for world in (2, 3):
        proc = np.zeros(c, dtype=np.uint64)
        local = torch.zeros(s.n_nodes, dtype=torch.int64, device="cuda")
        stored = []
        for rank in range(world):
            b, e = shard.shard_range(c, m, world, rank, mascot)
            if e == b:
                continue
            with rept.ReptStream(s.n_nodes, m, c, 3, flags=flags, max_batch=1 << 16, proc_range=(b, e)) as h:
                for off in range(0, len(s), 1 << 16):
                    h.ingest(src[off:off + (1 << 16)], dst[off:off + (1 << 16)])
                p, l = h.counts()
                stored.append(h.stats()["stored_edges"])
            assert (p[:b] == 0).all() and (p[e:] == 0).all()
            proc += p
            local += l
        assert np.array_equal(proc, ref.tau_proc), (world, proc, ref.tau_proc)
        assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1), world
        g, loc = rept.estimates_from_counts(m, c, proc, local, flags=flags)
        assert abs(g - ref_g) <= 1e-12 * max(abs(ref_g), 1.0)
        np.testing.assert_allclose(loc.cpu().numpy(), ref_loc, rtol=1e-12, atol=0)
        assert g == full_g
        # with one hash group each shard stores only the edges of its colours: the shards split them
        if not mascot and c <= m:
            with rept.ReptStream(s.n_nodes, m, c, 3, max_batch=1 << 16) as r1:
                for off in range(0, len(s), 1 << 16):
                    r1.ingest(src[off:off + (1 << 16)], dst[off:off + (1 << 16)])
                assert sum(stored) == r1.stats()["stored_edges"] and max(stored) < len(s)
