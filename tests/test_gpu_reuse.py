"""A handle reused for another stream after rept_reset / rept_reset_async.

The pool is not cleared between streams: blocks are handed out again from its start, over the lists
and tables of the previous stream, and each new table gets its empty keys when its block is handed
out.  These cases fill a handle with one stream (tables of every size, moved by the thread, warp and
block paths), reset it, and count a different stream whose blocks land on that memory; the counts
must equal the oracle's for the second stream alone.  They cover the three table layouts (colours in
the entries, colour words, split tables without colours) and both entry points of the batch path
(a pool known to fit, and one checked per batch).
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_09136_gb300 import graphgen as gg
from gpu_helpers import assert_counts_equal, assert_estimates_close, device_edges

pytestmark = pytest.mark.gpu


def _count(r, s, batch):
    src, dst = device_edges(s)
    for off in range(0, len(s), batch):
        r.ingest(src[off:off + batch], dst[off:off + batch])
    proc, local = r.counts()
    g, loc = r.estimates()
    return proc, local.cpu().numpy().view(np.uint64), g, loc.cpu().numpy()


# (m, c, n_nodes): one group with colours in the entries; one group with 2^24 < n (colour words);
# five groups (split tables, every candidate probed)
CASES = [(10, 10, 6000), (6, 6, (1 << 24) + 7), (4, 20, 6000)]


@pytest.mark.parametrize("m,c,n", CASES)
@pytest.mark.parametrize("presize", [True, False])
def test_reset_then_other_stream(m, c, n, presize):
    from paper_1811_09136_gb300.rept import ReptStream
    # the first stream: a dense power-law graph, so that tables of every size are built and moved
    a = gg.chung_lu(5000, 2.1, 60_000, cap=2000.0, graph_seed=3, order_seed=4)
    # the second stream: other nodes (shifted ids), other structure
    b0 = gg.chung_lu(5000, 2.4, 40_000, graph_seed=8, order_seed=9)
    shift = 1000
    b_src = (b0.src.astype(np.int64) + shift).astype(np.uint32)
    b_dst = (b0.dst.astype(np.int64) + shift).astype(np.uint32)
    b = gg.EdgeStream(b_src, b_dst, n)
    a = gg.EdgeStream(a.src, a.dst, n)
    expected = max(len(a), len(b)) if presize else 0
    with ReptStream(n, m, c, 17, expected_edges=expected, max_batch=1 << 14) as r:
        _count(r, a, 1 << 14)
        r.reset()
        proc, local, g, loc = _count(r, b, 1 << 12)
    ref = O.rept_stream(b.src, b.dst, n, m, c, 17, pair_counters=False)
    assert_counts_equal(proc, local, ref.tau_proc, ref.local1, f"m={m} c={c} presize={presize}")
    ref_g, ref_loc = O.estimates(m, c, ref, n)
    assert_estimates_close(g, loc, ref_g, ref_loc)


def test_reset_async_new_seed():
    from paper_1811_09136_gb300.rept import ReptStream
    a = gg.chung_lu(5000, 2.1, 60_000, cap=2000.0, graph_seed=5, order_seed=6)
    b = gg.rmat(12, 8, graph_seed=7, order_seed=8)
    n = max(a.n_nodes, b.n_nodes)
    a = gg.EdgeStream(a.src, a.dst, n)
    b = gg.EdgeStream(b.src, b.dst, n)
    with ReptStream(n, 8, 8, 1, expected_edges=len(a) + len(b), max_batch=1 << 15) as r:
        _count(r, a, 1 << 15)
        r.reset_async(seed=99)
        proc, local, g, loc = _count(r, b, 1 << 13)
    ref = O.rept_stream(b.src, b.dst, n, 8, 8, 99, pair_counters=False)
    assert_counts_equal(proc, local, ref.tau_proc, ref.local1, "reset_async")
