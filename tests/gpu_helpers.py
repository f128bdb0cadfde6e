"""Shared helpers of the GPU parity tests: run a stream through the C-ABI and fetch its outputs."""
from __future__ import annotations

import numpy as np


def device_edges(stream):
    import torch
    src = torch.from_numpy(stream.src.view(np.int32)).cuda()
    dst = torch.from_numpy(stream.dst.view(np.int32)).cuda()
    return src, dst


def gpu_run(stream, m, c, seed, batch=None, expected_edges=0, flags=0, max_batch=None):
    """Ingest ``stream`` in batches of ``batch`` edges (whole stream if None) through the C-ABI.
    Returns (tau^(i) uint64[c], local uint64[n], tau_hat, tau_hat_v float64[n], stats)."""
    from paper_1811_09136_gb300.rept import ReptStream
    T = len(stream)
    batch = batch or max(T, 1)
    with ReptStream(stream.n_nodes, m, c, seed, expected_edges=expected_edges,
                    max_batch=max_batch or batch, flags=flags) as r:
        src, dst = device_edges(stream)
        for off in range(0, T, batch):
            r.ingest(src[off:off + batch], dst[off:off + batch])
        proc, local = r.counts()
        g, loc = r.estimates()
        stats = r.stats()
        return proc, local.cpu().numpy().view(np.uint64), g, loc.cpu().numpy(), stats


def assert_counts_equal(proc, local, ref_proc, ref_local, what=""):
    assert np.array_equal(proc, np.asarray(ref_proc, dtype=np.uint64)), f"tau^(i) differ {what}"
    if not np.array_equal(local, np.asarray(ref_local, dtype=np.uint64)):
        bad = np.nonzero(local != ref_local)[0]
        raise AssertionError(f"local counts differ at {bad.size} nodes {what}, e.g. node {bad[0]}: "
                             f"{local[bad[0]]} vs {ref_local[bad[0]]}")


def assert_estimates_close(g, loc, ref_g, ref_loc, rtol=1e-12):
    """FP64 estimates within 1e-12 relative (both sides form (double)sum * factor)."""
    assert abs(g - ref_g) <= rtol * max(abs(ref_g), 1e-300), (g, ref_g)
    ref_loc = np.asarray(ref_loc)
    np.testing.assert_allclose(loc, ref_loc, rtol=rtol, atol=0.0)
