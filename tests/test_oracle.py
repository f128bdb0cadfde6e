"""The CPU oracle against facts fixed by the paper and by mathematics (no GPU)."""
import pytest

import oracle as O
import oracle_pins as P
from paper_1811_09136_gb300 import graphgen as gg


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()


def test_pcg32_published():
    """The input generators' PCG32 stream matches the PCG reference demo output."""
    want = P.read_golden_hex("pcg32_demo_42_54.txt")
    assert [int(x) for x in gg.pcg32_stream(42, 54, len(want))] == want


def test_generators_contract():
    """Every generator yields distinct undirected edges, no self-loops, ids below n."""
    import numpy as np
    for s in (gg.chung_lu(5000, 2.1, 30_000, cap=400.0), gg.rmat(12, 8), gg.gnp(40, 0.2)):
        assert (s.src < s.n_nodes).all() and (s.dst < s.n_nodes).all()
        assert not (s.src == s.dst).any()
        key = np.minimum(s.src, s.dst).astype(np.uint64) << np.uint64(32) | np.maximum(s.src, s.dst)
        assert np.unique(key).size == key.size
    a, b = gg.chung_lu(5000, 2.1, 30_000), gg.chung_lu(5000, 2.1, 30_000)
    assert a.sha256() == b.sha256()


def test_parallel_design_equals_the_sequential_oracle_and_the_definition():
    """The one-thread-per-processor oracle (the paper's multi-core design, used as a timing
    baseline) gives the sequential oracle's counts and the static enumeration's, c <= m, c = c1 m
    and c mod m != 0, with more and fewer threads than processors."""
    import numpy as np
    import oracle as O
    from paper_1811_09136_gb300 import graphgen as gg
    s = gg.chung_lu(1500, 2.2, 9000, graph_seed=5, order_seed=6)
    for (m, c, threads) in [(5, 3, 2), (4, 8, 3), (3, 7, 16)]:
        a = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 11, pair_counters=False)
        b = O.rept_stream_parallel(s.src, s.dst, s.n_nodes, m, c, 11, threads)
        e = O.semitriangles(s.src, s.dst, s.n_nodes, m, c, 11)
        assert np.array_equal(a.tau_proc, b.tau_proc) and np.array_equal(b.tau_proc, e.tau_proc)
        assert np.array_equal(a.local1, b.local1) and np.array_equal(a.local2, b.local2)
        assert np.array_equal(b.local1, e.local1) and np.array_equal(b.local2, e.local2)


def test_oracle_clean_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    """Every oracle routine on random small graphs, built with -fsanitize=address,undefined (abort
    on the first report): no memory error, no undefined behaviour, and the routines agree."""
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "oracle_sanitize")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=gnu11", "-fopenmp", "-fsanitize=address,undefined",
                           "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
                           os.path.join(here, "native", "oracle_sanitize.c"), O._SRC, "-o", exe])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0", UBSAN_OPTIONS="print_stacktrace=1")
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stdout + out.stderr[-4000:]
    assert "oracle sanitize failures: 0" in out.stdout
