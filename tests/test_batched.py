"""The batched path: many streams through one rept_group give every stream exactly the counts of
the plain single-stream path and of the oracle.  Plus host-side checks of the stream mix."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1811_09136_gb300 import batched


def test_mix_is_deterministic_and_in_range():
    a = batched.mix_specs(256, seed=1000)
    b = batched.mix_specs(256, seed=1000)
    assert [(x.kind, x.n_nodes, x.m) for x in a] == [(x.kind, x.n_nodes, x.m) for x in b]
    assert all(1e4 <= x.n_nodes <= 2e6 for x in a)
    assert all(10 <= x.edges_per_node <= 40 for x in a)
    assert all(2.1 <= x.gamma <= 2.5 for x in a)
    assert {x.m for x in a} == {10, 20, 100}
    kinds = sum(x.kind == "rmat" for x in a)
    assert 90 < kinds < 166                      # both graph families, about half each
    logn = np.log([x.n_nodes for x in a])
    assert abs(logn.mean() - 0.5 * (math.log(1e4) + math.log(2e6))) < 0.5  # log-uniform centre


def test_waves_respect_the_budget():
    from paper_1811_09136_gb300.graphgen import EdgeStream
    streams = [EdgeStream(np.zeros(n, np.uint32), np.zeros(n, np.uint32), 1000) for n in (10, 5000, 20, 70000, 3)]
    budget = batched._state_bytes(1000, 70000, 64) + 8 * 70000 + 10
    waves = list(batched._waves(streams, 64, budget))
    assert sorted(i for w in waves for i in w) == list(range(5))
    for w in waves:
        used = sum(batched._state_bytes(1000, len(streams[i]), min(64, len(streams[i]))) + 8 * len(streams[i])
                   for i in w)
        assert used <= budget or len(w) == 1


def _mix(k=7, seed=31):
    specs = batched.mix_specs(k, seed=seed, n_min=800, n_max=12_000, epn=(4.0, 12.0))
    streams = batched.generate_all(specs, processes=1)
    params = [(sp.m, sp.m, sp.hash_seed) for sp in specs]
    return streams, params


@pytest.mark.gpu
@pytest.mark.parametrize("graph,presize,batch,persistent", [(True, True, 1 << 12, False), (False, True, 777, False),
                                                            (True, False, 1 << 10, False), (False, True, 1 << 11, True),
                                                            (True, True, 999, True), (True, False, 1 << 10, True)])
def test_batched_equals_plain_and_oracle(graph, presize, batch, persistent):
    """Launch per step, with and without graphs, pools presized or grown, and one persistent launch per
    round (REPT_GROUP_PERSISTENT; with pools that may grow a round falls back to the launch per step)."""
    streams, params = _mix()
    res_b, _ = batched.run_batched(streams, params, batch=batch, graph=graph, presize=presize,
                                   local_estimates=True, persistent=persistent)
    res_p, _ = batched.run_plain(streams, params, batch=batch, local_estimates=True)
    for s, (m, c, seed), rb, rp in zip(streams, params, res_b, res_p):
        ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, seed, pair_counters=False)
        ref_g, ref_loc = O.estimates(m, c, ref, s.n_nodes)
        for r in (rb, rp):
            assert np.array_equal(r.proc, ref.tau_proc)
            assert np.array_equal(r.local, ref.local1)
            assert abs(r.tau_hat - ref_g) <= 1e-12 * max(abs(ref_g), 1.0)
            np.testing.assert_allclose(r.local_hat, ref_loc, rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_batched_small_memory_budget_runs_in_waves():
    streams, params = _mix(5, seed=44)
    budget = max(batched._state_bytes(s.n_nodes, len(s), 1 << 11) + 8 * len(s) for s in streams) + 1
    assert len(list(batched._waves(streams, 1 << 11, budget))) > 1
    res_b, _ = batched.run_batched(streams, params, batch=1 << 11, budget=budget)
    for s, (m, c, seed), rb in zip(streams, params, res_b):
        ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, seed, pair_counters=False)
        assert np.array_equal(rb.proc, ref.tau_proc) and np.array_equal(rb.local, ref.local1)


@pytest.mark.gpu
def test_ingest_multi_equals_the_oracle():
    """rept_ingest_multi (the library's own group): several streams fed batch by batch, streams
    finishing at different rounds (empty batches), more streams than the first call brought (the
    group is made again, larger), and the oracle's counts for each."""
    import torch
    from paper_1811_09136_gb300 import rept
    streams, params = _mix(k=70, seed=37)
    dev = [(torch.from_numpy(s.src.view(np.int32)).cuda(), torch.from_numpy(s.dst.view(np.int32)).cuda())
           for s in streams]
    handles = [rept.ReptStream(s.n_nodes, m, c, seed, max_batch=1500) for s, (m, c, seed) in zip(streams, params)]
    try:
        # first call with 3 streams, then all 70 (more than the 64 the group was sized for)
        rept.ingest_multi(handles[:3], [d[0][:1500] for d in dev[:3]], [d[1][:1500] for d in dev[:3]])
        fed = [1500] * 3 + [0] * (len(streams) - 3)
        while any(f < len(s) for f, s in zip(fed, streams)):
            a = [d[0][f:f + 1500] for d, f in zip(dev, fed)]
            b = [d[1][f:f + 1500] for d, f in zip(dev, fed)]
            rept.ingest_multi(handles, a, b)
            fed = [min(len(s), f + 1500) for f, s in zip(fed, streams)]
        for h, s, (m, c, seed) in zip(handles, streams, params):
            proc, local = h.counts()
            ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, seed, pair_counters=False)
            assert np.array_equal(proc, ref.tau_proc)
            assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1)
    finally:
        for h in handles:
            h.close()


def test_autotune_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    """Host logic of the autotuner with a fake timing: the fastest (batch, tile) wins, the choice is
    written to the cache, and a second call reads it back without timing anything."""
    calls = []

    def fake_run(streams, params, batch, tile_max, **kw):
        calls.append((batch, tile_max))
        return None, abs(batch - (1 << 18)) / 1e6 + (0.5 if tile_max == 16 else 0.1)

    monkeypatch.setattr(batched, "run_batched", fake_run)
    monkeypatch.setattr(batched, "_device_key", lambda: "fake-gpu")
    monkeypatch.setattr(batched, "_CACHE", str(tmp_path / "autotune.json"))
    b, tm, timings = batched.autotune([], [], key="t", repeat=1)
    assert (b, tm) == (1 << 18, 32) and len(timings) == 6 and len(calls) == 6
    b2, tm2, t2 = batched.autotune([], [], key="t", repeat=1)
    assert (b2, tm2) == (b, tm) and t2 == timings and len(calls) == 6   # served from the cache
    (tmp_path / "autotune.json").write_text("{not json")
    b3, _, _ = batched.autotune([], [], key="t", repeat=1)            # a damaged cache is re-measured
    assert b3 == 1 << 18 and len(calls) == 12


@pytest.mark.gpu
def test_batched_midsize_stream_runs_the_hub_classes_and_matches_the_oracle():
    """A mix with one mid-size power-law stream (2 x 10^5 nodes, 2.4 x 10^6 edges) beside small ones:
    its smaller endpoints reach hundreds of entries, so the warp classes (33-256 entries and more)
    run inside the group's intersection kernel; every stream's counts equal the oracle's static
    enumeration and the plain path's."""
    from paper_1811_09136_gb300 import graphgen as gg
    from paper_1811_09136_gb300 import rept
    import torch
    big = gg.chung_lu(200_000, 2.1, 2_400_000, cap=20_000.0, graph_seed=61, order_seed=62)
    small, sparams = _mix(k=3, seed=29)
    streams = [big] + small
    params = [(20, 20, 4242)] + sparams
    # the big stream really has edges of both warp classes
    with rept.ReptStream(big.n_nodes, 20, 20, 4242, max_batch=1 << 18, flags=rept.FLAG_WORK_COUNTERS) as r:
        src = torch.from_numpy(big.src.view(np.int32)).cuda()
        dst = torch.from_numpy(big.dst.view(np.int32)).cuda()
        for off in range(0, len(big), 1 << 18):
            r.ingest(src[off:off + (1 << 18)], dst[off:off + (1 << 18)])
        st = r.stats()
    assert st["class_items"][4] > 0 and st["class_items"][5] > 0, st["class_items"]
    res_b, _ = batched.run_batched(streams, params, batch=1 << 18, graph=True)
    res_p, _ = batched.run_plain(streams, params, batch=1 << 18)
    for s, (m, c, seed), rb, rp in zip(streams, params, res_b, res_p):
        ref = O.semitriangles(s.src, s.dst, s.n_nodes, m, c, seed)
        ref_g, _ = O.estimates(m, c, O.Counts(ref.tau_proc, ref.local1, ref.local2), s.n_nodes)
        for r in (rb, rp):
            assert np.array_equal(r.proc, ref.tau_proc)
            assert np.array_equal(r.local, ref.local1)
            assert abs(r.tau_hat - ref_g) <= 1e-12 * max(abs(ref_g), 1.0)


@pytest.mark.gpu
def test_persistent_wait_that_runs_out_reports_timeout_and_leaves_the_device_usable():
    """The test hook REPT_GROUP_TEST_TIMEOUT makes the persistent kernel's first grid-wide wait expect
    one block more than the grid holds, so every block's wait runs out after 0.1 s: the kernel records
    the timeout and returns (no block waits without a limit), each stream reports REPT_E_TIMEOUT with
    nothing applied, and after rept_reset the same handles count the oracle's values."""
    import torch
    from paper_1811_09136_gb300 import rept
    streams, params = _mix(k=3, seed=71)
    dev = [(torch.from_numpy(s.src.view(np.int32)).cuda(), torch.from_numpy(s.dst.view(np.int32)).cuda())
           for s in streams]
    handles = [rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=len(s), max_batch=len(s))
               for s, (m, c, seed) in zip(streams, params)]
    try:
        bad = batched.ReptGroup(len(handles), graph=False, persistent=True, test_timeout=True)
        bad.ingest(handles, [d[0] for d in dev], [d[1] for d in dev])
        for h in handles:
            proc, _, rc = h.counts(allow_error=True)
            assert rc == -6, rc                        # REPT_E_TIMEOUT
            assert int(proc.sum()) == 0                # the round was not applied
        bad.close()
        torch.cuda.synchronize()                       # the context is still usable
        good = batched.ReptGroup(len(handles), graph=False, persistent=True)
        for h in handles:
            h.reset()
        good.ingest(handles, [d[0] for d in dev], [d[1] for d in dev])
        for h, s, (m, c, seed) in zip(handles, streams, params):
            proc, local = h.counts()
            ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, seed, pair_counters=False)
            assert np.array_equal(proc, ref.tau_proc)
            assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1)
        good.close()
    finally:
        for h in handles:
            h.close()


def test_timeout_hook_needs_the_persistent_flag():
    """REPT_GROUP_TEST_TIMEOUT alone is refused before any device work (no GPU needed)."""
    import ctypes
    from paper_1811_09136_gb300 import rept
    lib = rept.load()
    lib.rept_group_create.restype = ctypes.c_int
    lib.rept_group_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.rept_group_create(4, batched.GROUP_TEST_TIMEOUT, ctypes.byref(h)) == -1
