"""Run in a child process with REPT_LIBRARY naming the bounds-checked debug build: parity cases
through every kernel path (tile and warp classes, block moves, Algorithm 2, MASCOT, the batched
group, the allocation-free call).  A failed index check makes the next synchronising call raise
(REPT_E_INTERNAL), so a clean exit means every checked access was in bounds and the counts are the
oracle's.  Prints "debug-bounds ok" at the end."""
import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle as O  # noqa: E402
from paper_1811_09136_gb300 import batched, rept  # noqa: E402
from paper_1811_09136_gb300 import graphgen as gg  # noqa: E402
from gpu_helpers import assert_counts_equal, device_edges, gpu_run  # noqa: E402


def main():
    lib = rept.load()
    assert os.path.basename(rept.library_path()) == "librept_debug.so", rept.library_path()
    # small graphs, every batch split (tile classes, table growth from 4 slots)
    for n, q, gs in [(23, 0.4, 2), (40, 0.3, 3)]:
        s = gg.gnp(n, q, graph_seed=gs, order_seed=gs + 10)
        for (m, c) in [(3, 2), (2, 4), (3, 7)]:
            ref = O.rept_stream(s.src, s.dst, n, m, c, 5)
            for batch in (1, 7, len(s)):
                proc, local, _, _, _ = gpu_run(s, m, c, 5, batch=batch)
                assert_counts_equal(proc, local, ref.tau_proc, ref.local1 + ref.local2, f"{n} {m} {c} {batch}")
    # a power-law stream: warp classes, block moves of every size, pool growth, colours kept
    s = gg.cached("powerlaw_20k")
    for (m, c, batch) in [(10, 10, 1 << 15), (1, 1, 50_000), (4, 10, 1 << 16)]:
        ref = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 1, pair_counters=(c > m and c % m != 0))
        proc, local, _, _, _ = gpu_run(s, m, c, 1, batch=batch)
        assert_counts_equal(proc, local, ref.tau_proc, ref.local1 + ref.local2, f"powerlaw {m} {c}")
    # MASCOT
    ref = O.mascot_stream(s.src, s.dst, s.n_nodes, 4, 10, 3)
    proc, local, _, _, _ = gpu_run(s, 4, 10, 3, batch=1 << 16, flags=rept.FLAG_MASCOT)
    assert_counts_equal(proc, local, ref.tau_proc, ref.local1, "mascot")
    # the batched group
    specs = batched.mix_specs(5, seed=77, n_min=800, n_max=8000, epn=(4.0, 10.0))
    streams = batched.generate_all(specs, processes=1)
    params = [(sp.m, sp.m, sp.hash_seed) for sp in specs]
    res, _ = batched.run_batched(streams, params, batch=1 << 11, graph=False, presize=False)
    for st, (m, c, seed), r in zip(streams, params, res):
        ref = O.rept_stream(st.src, st.dst, st.n_nodes, m, c, seed, pair_counters=False)
        assert np.array_equal(r.proc, ref.tau_proc) and np.array_equal(r.local, ref.local1)
    # the allocation-free entry point
    import torch
    fn = lib.rept_count_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    st = gg.chung_lu(5000, 2.2, 40_000, graph_seed=9, order_seed=9)
    src, dst = device_edges(st)
    proc = torch.empty(10, dtype=torch.int64, device="cuda")
    local = torch.empty(st.n_nodes, dtype=torch.int64, device="cuda")
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = fn(src.data_ptr(), dst.data_ptr(), len(st), st.n_nodes, 10, 10, 4, proc.data_ptr(), local.data_ptr(),
            g.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0, rc
    ref = O.rept_stream(st.src, st.dst, st.n_nodes, 10, 10, 4, pair_counters=False)
    ref_g, _ = O.estimates(10, 10, ref, st.n_nodes)
    assert np.array_equal(proc.cpu().numpy().view(np.uint64), ref.tau_proc)
    assert np.array_equal(local.cpu().numpy().view(np.uint64), ref.local1)
    assert abs(float(g.item()) - ref_g) <= 1e-12 * abs(ref_g), (float(g.item()), ref_g)
    print("debug-bounds ok")


if __name__ == "__main__":
    main()
