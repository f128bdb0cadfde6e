"""CUDA path vs the CPU oracle: bit-exact integer counts, FP64 estimates within 1e-12 relative.

Every GPU call goes through the C-ABI (librept.so) via the ctypes binding.
"""
import math

import numpy as np
import pytest

import oracle as O
from gpu_helpers import assert_counts_equal, assert_estimates_close, device_edges, gpu_run
from paper_1811_09136_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

SUPPORTED_SMALL = [(2, 1), (2, 2), (3, 2), (4, 4), (5, 3), (2, 4), (3, 6), (1, 1), (1, 3), (7, 7)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    from paper_1811_09136_gb300 import rept
    rept.load()


@pytest.mark.parametrize("n,q,gs", [(9, 0.7, 1), (23, 0.4, 2), (40, 0.3, 3)])
@pytest.mark.parametrize("m,c", SUPPORTED_SMALL)
def test_small_graphs_every_batch_split(n, q, gs, m, c):
    s = gg.gnp(n, q, graph_seed=gs, order_seed=gs + 10)
    ref = O.rept_stream(s.src, s.dst, n, m, c, 5)
    ref_g, ref_loc = O.estimates(m, c, ref, n)
    for batch in (1, 7, len(s)):
        proc, local, g, loc, _ = gpu_run(s, m, c, 5, batch=batch)
        assert_counts_equal(proc, local, ref.tau_proc, ref.local1, f"batch={batch}")
        assert_estimates_close(g, loc, ref_g, ref_loc)


def test_complete_graph_closed_form():
    for n in (3, 4, 12, 64):
        s = gg.complete(n, order_seed=n)
        proc, local, g, loc, _ = gpu_run(s, 1, 1, 3, batch=5)
        assert int(proc[0]) == math.comb(n, 3)
        assert np.all(local == math.comb(n - 1, 2))
        assert g == float(math.comb(n, 3))


@pytest.mark.parametrize("m,c", [(10, 10), (10, 3), (4, 8), (1, 1), (300, 300), (300, 120)])
def test_powerlaw_20k(m, c):
    """Chung-Lu, 20,000 nodes, exponent 2.3, 200,000 edges: whole stream, 2^10 and 2^16 batches.
    m = 300 keeps a colour word per list entry (too many colours for the entry's top 8 bits)."""
    s = gg.cached("powerlaw_20k")
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 1, pair_counters=False)
    ref_g, ref_loc = O.estimates(m, c, ref, s.n_nodes)
    for batch in (len(s), 1 << 10, 1 << 16):
        proc, local, g, loc, st = gpu_run(s, m, c, 1, batch=batch)
        assert_counts_equal(proc, local, ref.tau_proc, ref.local1, f"batch={batch}")
        assert_estimates_close(g, loc, ref_g, ref_loc)
        assert st["edges"] == len(s) and st["self_loops"] == 0


def test_pool_growth_matches_presized_pool():
    """A pool that starts small and grows gives the same counts as one sized up front."""
    s = gg.chung_lu(30_000, 2.1, 150_000, graph_seed=5, order_seed=6)
    a = gpu_run(s, 8, 8, 2, batch=4096, expected_edges=0, max_batch=4096)
    b = gpu_run(s, 8, 8, 2, batch=4096, expected_edges=len(s))
    assert_counts_equal(a[0], a[1], b[0], b[1])
    assert a[4]["pool_slots"] < b[4]["pool_slots"] or a[4]["pool_slots"] >= a[4]["pool_used"]
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, 8, 8, 2, pair_counters=False)
    assert_counts_equal(a[0], a[1], ref.tau_proc, ref.local1)


def test_self_loops_skipped():
    s = gg.gnp(30, 0.4, 7, 8)
    src = np.insert(s.src, [3, 50, 50, len(s)], np.array([5, 9, 9, 2], dtype=np.uint32))
    dst = np.insert(s.dst, [3, 50, 50, len(s)], np.array([5, 9, 9, 2], dtype=np.uint32))
    loops = gg.EdgeStream(src, dst, 30)
    ref = O.rept_stream(src, dst, 30, 3, 3, 4)
    proc, local, _, _, st = gpu_run(loops, 3, 3, 4, batch=17)
    assert_counts_equal(proc, local, ref.tau_proc, ref.local1)
    assert st["self_loops"] == 4 == ref.skipped


def test_empty_batch_and_ingest_host_equal_device():
    from paper_1811_09136_gb300.rept import ReptStream
    import torch
    s = gg.chung_lu(5000, 2.3, 40_000, graph_seed=9, order_seed=10)
    with ReptStream(s.n_nodes, 5, 5, 11) as r:
        empty = torch.empty(0, dtype=torch.int32, device="cuda")
        r.ingest(empty, empty)
        r.ingest_host(s.src, s.dst, batch=3000)
        proc, local = r.counts()
        st = r.stats()
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, 5, 5, 11, pair_counters=False)
    assert_counts_equal(proc, local.cpu().numpy().view(np.uint64), ref.tau_proc, ref.local1)
    assert st["edges"] == len(s)


def test_range_error_leaves_state_unchanged_and_reset_recovers():
    from paper_1811_09136_gb300.rept import ReptStream, ReptError
    import torch
    s = gg.gnp(40, 0.3, 12, 13)
    half = len(s) // 2
    src, dst = device_edges(s)
    with ReptStream(s.n_nodes, 3, 3, 1) as r:
        r.ingest(src[:half], dst[:half])
        bad = torch.tensor([1, 40, 2], dtype=torch.int32, device="cuda")  # 40 >= n_nodes
        ok = torch.tensor([2, 3, 4], dtype=torch.int32, device="cuda")
        r.ingest(ok, bad)
        r.ingest(src[half:], dst[half:])  # also dropped: the error is sticky
        proc, local, rc = r.counts(allow_error=True)
        assert rc == -2
        with pytest.raises(ReptError):
            r.sync()
        ref = O.rept_stream(s.src[:half], s.dst[:half], 40, 3, 3, 1)
        assert_counts_equal(proc, local.cpu().numpy().view(np.uint64), ref.tau_proc, ref.local1)
        r.reset()
        r.ingest(src, dst)
        proc, local = r.counts()
        full = O.rept_stream(s.src, s.dst, 40, 3, 3, 1)
        assert_counts_equal(proc, local.cpu().numpy().view(np.uint64), full.tau_proc, full.local1)


def test_fixed_pool_capacity_error():
    from paper_1811_09136_gb300.rept import ReptStream, FLAG_FIXED_POOL
    s = gg.chung_lu(20_000, 2.2, 100_000, graph_seed=14, order_seed=15)
    src, dst = device_edges(s)
    # pool sized for 2,000 edges: the first batch fits, a later one cannot
    with ReptStream(s.n_nodes, 4, 4, 3, expected_edges=2000, max_batch=1000, flags=FLAG_FIXED_POOL) as r:
        r.ingest(src[:1000], dst[:1000])
        r.sync()
        good = r.counts()
        for off in range(1000, len(s), 1000):
            r.ingest(src[off:off + 1000], dst[off:off + 1000])
        proc, local, rc = r.counts(allow_error=True)
        assert rc == -3
    # counts are those of a prefix that ended at a batch boundary, and never exceed the full stream's
    ref_full = O.rept_stream(s.src, s.dst, s.n_nodes, 4, 4, 3, pair_counters=False)
    assert int(proc.sum()) <= int(ref_full.tau_proc.sum())
    assert int(proc.sum()) >= int(good[0].sum())
    found = False
    for end in range(1000, len(s) + 1, 1000):
        ref = O.rept_stream(s.src[:end], s.dst[:end], s.n_nodes, 4, 4, 3, pair_counters=False)
        if np.array_equal(ref.tau_proc, proc):
            assert_counts_equal(proc, local.cpu().numpy().view(np.uint64), ref.tau_proc, ref.local1)
            found = True
            break
        if int(ref.tau_proc.sum()) > int(proc.sum()):
            break
    assert found


@pytest.mark.parametrize("n", [1 << 24, 1 << 27])
def test_large_node_ids(n):
    """Ids near the top of a 2^24-node space (the largest whose list entries carry colours in their
    top 8 bits) and of a 2^27-node space (colours in a word per list entry; node records and local
    counts of 2 GB and 1 GB)."""
    base = gg.gnp(60, 0.25, 16, 17)
    off = np.uint32(n - 64)
    s = gg.EdgeStream(base.src + off, base.dst + off, n)
    proc, local, g, loc, _ = gpu_run(s, 3, 3, 8, batch=37)
    ref = O.rept_stream(s.src, s.dst, n, 3, 3, 8, pair_counters=False)
    assert_counts_equal(proc, local, ref.tau_proc, ref.local1)
    assert int(local[: n - 64].sum()) == 0


@pytest.mark.parametrize("m,c", [(3, 7), (4, 9), (2, 3), (5, 12), (3, 4)])
def test_partial_group_algorithm2(m, c):
    """c > m with c mod m != 0: tau^(i), the split local counts, the triangle-pair counters eta^(i)
    and sum_i eta_v^(i), and the combined estimates all match the oracle, for every batch split."""
    s = gg.chung_lu(3000, 2.2, 25_000, graph_seed=m, order_seed=c)
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 7)
    ref_g, ref_loc = O.estimates(m, c, ref, s.n_nodes)
    from paper_1811_09136_gb300.rept import ReptStream
    src, dst = device_edges(s)
    for batch in (len(s), 997, 1 << 13):
        with ReptStream(s.n_nodes, m, c, 7, max_batch=batch) as r:
            for off in range(0, len(s), batch):
                r.ingest(src[off:off + batch], dst[off:off + batch])
            proc, local = r.counts()
            eta, el, l1, l2 = r.pair_counts()
            g, loc = r.estimates()
        u64 = lambda t: t.cpu().numpy().view(np.uint64)
        assert np.array_equal(proc, ref.tau_proc), batch
        assert np.array_equal(u64(l1), ref.local1) and np.array_equal(u64(l2), ref.local2), batch
        assert np.array_equal(u64(local), ref.local1 + ref.local2), batch
        assert np.array_equal(eta, ref.eta_proc), (batch, eta, ref.eta_proc)
        assert np.array_equal(u64(el), ref.eta_local), batch
        assert_estimates_close(g, loc.cpu().numpy(), ref_g, ref_loc)


def test_work_counters_match_the_graph():
    """With m = c = 1 every edge is stored, so the intersection finds every triangle exactly once
    (at its last edge): wedges == counted == tau.  Probes read whole 4-slot buckets and the tables
    stay at most half full, so a probe reads few slots on average."""
    from paper_1811_09136_gb300.rept import ReptStream, FLAG_WORK_COUNTERS
    s = gg.cached("powerlaw_20k")
    exact = O.semitriangles(s.src, s.dst, s.n_nodes, 1, 1, 1)
    src, dst = device_edges(s)
    with ReptStream(s.n_nodes, 1, 1, 1, max_batch=1 << 15, flags=FLAG_WORK_COUNTERS) as r:
        for off in range(0, len(s), 1 << 15):
            r.ingest(src[off:off + (1 << 15)], dst[off:off + (1 << 15)])
        st = r.stats()
    assert st["wedges"] == exact.triangles == st["counted"]
    assert st["probes"] <= st["small_entries"] <= st["small_slots"]
    assert 4 * st["probes"] <= st["probe_slots"] < 6 * st["probes"]


@pytest.mark.parametrize("m,c", [(4, 4), (5, 3), (3, 6), (3, 7)])
def test_local_per_processor(m, c):
    """Every processor's tau_v^(i) equals the oracle's, and sums to 3 tau^(i) per processor."""
    from paper_1811_09136_gb300.rept import ReptStream, FLAG_LOCAL_PER_PROCESSOR
    s = gg.chung_lu(1500, 2.2, 12_000, graph_seed=c, order_seed=m)
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 3, per_proc_local=True)
    src, dst = device_edges(s)
    with ReptStream(s.n_nodes, m, c, 3, max_batch=2048, flags=FLAG_LOCAL_PER_PROCESSOR) as r:
        for off in range(0, len(s), 2048):
            r.ingest(src[off:off + 2048], dst[off:off + 2048])
        lp = r.local_per_processor().cpu().numpy().view(np.uint64)
        proc, _ = r.counts()
    assert np.array_equal(lp, ref.tau_local_proc)
    assert np.array_equal(lp.sum(axis=1), 3 * proc)


@pytest.mark.parametrize("m,c,flags", [(10, 10, 0), (3, 7, 0), (4, 4, 16)])
def test_snapshot_restore_resumes_exactly(m, c, flags):
    """Half the stream, a snapshot to host memory, a fresh handle restored from it, the other half:
    the same counts (and pair counters / per-processor locals when kept) as one uninterrupted run."""
    from paper_1811_09136_gb300.rept import ReptStream, ReptError
    s = gg.chung_lu(4000, 2.2, 30_000, graph_seed=m + c, order_seed=5)
    src, dst = device_edges(s)
    half = 13_337
    with ReptStream(s.n_nodes, m, c, 9, max_batch=4096, flags=flags) as a:
        for off in range(0, half, 4096):
            e = min(half, off + 4096)
            a.ingest(src[off:e], dst[off:e])
        snap = a.snapshot()
    with ReptStream(s.n_nodes, m, c, 9, max_batch=4096, flags=flags) as b:
        b.restore(snap)
        for off in range(half, len(s), 4096):
            b.ingest(src[off:off + 4096], dst[off:off + 4096])
        proc, local = b.counts()
        g, _ = b.estimates(local=False)
        extra = b.pair_counts()[0] if c > m and c % m else None
        lp = b.local_per_processor().cpu().numpy() if flags else None
        st = b.stats()
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 9, per_proc_local=bool(flags))
    ref_g, _ = O.estimates(m, c, ref, s.n_nodes)
    assert np.array_equal(proc, ref.tau_proc)
    assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1 + ref.local2)
    assert abs(g - ref_g) <= 1e-12 * abs(ref_g)
    assert st["edges"] == len(s)
    if extra is not None:
        assert np.array_equal(extra, ref.eta_proc)
    if lp is not None:
        assert np.array_equal(lp.view(np.uint64), ref.tau_local_proc)
    with ReptStream(s.n_nodes, m, c, 10, max_batch=4096, flags=flags) as wrong_seed:
        with pytest.raises(ReptError):
            wrong_seed.restore(snap)


@pytest.mark.parametrize("m,c", [(1, 3), (3, 1), (4, 4), (10, 7), (4, 10), (100, 20)])
def test_parallel_mascot_matches_oracle(m, c):
    """FLAG_MASCOT: c independent p = 1/m samplers (hash group i, colour 0).  tau^(i), the local
    sums, every tau_v^(i) and the (m^2/c)-scaled estimates match the oracle for several batch splits."""
    from paper_1811_09136_gb300.rept import ReptStream, FLAG_MASCOT, FLAG_LOCAL_PER_PROCESSOR
    s = gg.chung_lu(2500, 2.2, 20_000, graph_seed=m, order_seed=c)
    ref = O.mascot_stream(s.src, s.dst, s.n_nodes, m, c, 17, per_proc_local=True)
    ref_g, ref_loc = O.mascot_estimates(m, c, ref, s.n_nodes)
    src, dst = device_edges(s)
    for batch in (len(s), 1009):
        with ReptStream(s.n_nodes, m, c, 17, max_batch=batch, flags=FLAG_MASCOT | FLAG_LOCAL_PER_PROCESSOR) as r:
            for off in range(0, len(s), batch):
                r.ingest(src[off:off + batch], dst[off:off + batch])
            proc, local = r.counts()
            lp = r.local_per_processor().cpu().numpy().view(np.uint64)
            g, loc = r.estimates()
        assert np.array_equal(proc, ref.tau_proc), (batch, proc, ref.tau_proc)
        assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1), batch
        assert np.array_equal(lp, ref.tau_local_proc), batch
        assert_estimates_close(g, loc.cpu().numpy(), ref_g, ref_loc)


def test_check_dups_flags_repeats_and_leaves_the_state():
    """REPT_FLAG_CHECK_DUPS: a batch holding an edge twice, or repeating a stored edge of an earlier
    batch (either orientation), fails with REPT_E_DUPLICATE and is not applied; a clean stream gives
    the oracle's counts with the check on."""
    import torch
    from paper_1811_09136_gb300.rept import ReptStream, ReptError, FLAG_CHECK_DUPS, FLAG_SYNC
    s = gg.chung_lu(3000, 2.2, 20_000, graph_seed=3, order_seed=4)
    src, dst = device_edges(s)
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, 4, 4, 2)
    with ReptStream(s.n_nodes, 4, 4, 2, max_batch=4096, flags=FLAG_CHECK_DUPS) as r:
        for off in range(0, len(s), 4096):
            r.ingest(src[off:off + 4096], dst[off:off + 4096])
        proc, local = r.counts()
    assert np.array_equal(proc, ref.tau_proc)
    assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1)
    half = 10_000
    for case in ("same_batch", "earlier_batch"):
        with ReptStream(s.n_nodes, 1, 1, 2, max_batch=4096, flags=FLAG_CHECK_DUPS | FLAG_SYNC) as r:
            r.ingest(src[:half], dst[:half])
            before = r.counts()[0].copy()
            if case == "same_batch":
                a = torch.cat([src[half:half + 50], src[half + 7:half + 8]])
                b = torch.cat([dst[half:half + 50], dst[half + 7:half + 8]])
            else:  # edge 123 again, reversed
                a = torch.cat([src[half:half + 50], dst[123:124]])
                b = torch.cat([dst[half:half + 50], src[123:124]])
            with pytest.raises(ReptError) as ei:
                r.ingest(a, b)
            assert ei.value.code == -9, ei.value
            proc, _, rc = r.counts(allow_error=True)
            assert rc == -9 and np.array_equal(proc, before), case
