"""rept_count_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: their device memory is owned by another
allocator, or they cannot afford the device-wide synchronisation that freeing
memory implies.  rept_count_noalloc serves them by keeping all of its scratch in
a fixed device array inside the library.  This test calls it through the C ABI
twice in a row, the first call on the current stream and the second on a stream
of its own (the calls do not overlap: each waits for its stream before it
returns), and checks each result against the
regular handle-based entry points (rept_create / rept_ingest_batch /
rept_counts / rept_estimates): the integer counts must be identical and the
global estimate within 1e-12 relative, the tolerance of the other GPU tests.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1811_09136_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

REPT_E_SCRATCH = -8


def _lib():
    from paper_1811_09136_gb300 import rept
    lib = rept.load()
    fn = lib.rept_count_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return fn


def _noalloc(fn, s, m, c, seed, stream=None):
    import torch
    stream = stream or torch.cuda.current_stream()
    src = torch.from_numpy(s.src.view(np.int32)).cuda()
    dst = torch.from_numpy(s.dst.view(np.int32)).cuda()
    proc = torch.empty(c, dtype=torch.int64, device="cuda")
    local = torch.empty(s.n_nodes, dtype=torch.int64, device="cuda")
    glob = torch.empty(1, dtype=torch.float64, device="cuda")
    # poison the outputs: the call must overwrite them
    proc.fill_(-1)
    local.fill_(-1)
    # the inputs and poisoned outputs were written on the current stream
    stream.wait_stream(torch.cuda.current_stream())
    rc = fn(src.data_ptr(), dst.data_ptr(), len(s), s.n_nodes, m, c, seed, proc.data_ptr(), local.data_ptr(),
            glob.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.current_stream().wait_stream(stream)
    return rc, proc.cpu().numpy().view(np.uint64), local.cpu().numpy().view(np.uint64), float(glob.item())


def _regular(s, m, c, seed):
    from paper_1811_09136_gb300.rept import ReptStream
    import torch
    src = torch.from_numpy(s.src.view(np.int32)).cuda()
    dst = torch.from_numpy(s.dst.view(np.int32)).cuda()
    with ReptStream(s.n_nodes, m, c, seed, max_batch=len(s)) as r:
        r.ingest(src, dst)
        proc, local = r.counts()
        g, _ = r.estimates(local=False)
    return proc, local.cpu().numpy().view(np.uint64), g


def test_noalloc_matches_regular_entry_points_on_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    fn = _lib()
    first = gg.chung_lu(20_000, 2.3, 200_000, graph_seed=42, order_seed=7)
    second = gg.chung_lu(50_000, 2.1, 120_000, cap=2_000.0, graph_seed=3, order_seed=4)
    for s, (m, c, seed), stream in ((first, (10, 10, 1), None), (second, (4, 8, 99), torch.cuda.Stream())):
        rc, proc, local, g = _noalloc(fn, s, m, c, seed, stream)
        assert rc == 0, rc
        ref_proc, ref_local, ref_g = _regular(s, m, c, seed)
        assert np.array_equal(proc, ref_proc)
        assert np.array_equal(local, ref_local)
        assert abs(g - ref_g) <= 1e-12 * abs(ref_g)
        assert int(proc.sum()) > 0


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    fn = _lib()
    n, E = 1 << 22, 1 << 20  # 20 n + 216 E + 200 KiB > 64 MiB
    src = torch.zeros(E, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(src.data_ptr(), src.data_ptr(), E, n, 10, 10, 1, out.data_ptr(), out.data_ptr(), None,
              stream) == REPT_E_SCRATCH
