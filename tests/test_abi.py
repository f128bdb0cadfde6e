"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every declared entry point."""
import ctypes
import os
import re

from paper_1811_09136_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(rept_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"rept_create", "rept_ingest_batch", "rept_estimates", "rept_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_launch_counter_without_gpu():
    lib = ctypes.CDLL(_build.build())
    lib.rept_strerror.restype = ctypes.c_char_p
    assert lib.rept_strerror(-2) == b"edge endpoint >= n_nodes"
    lib.rept_kernel_launches.restype = ctypes.c_uint64
    assert lib.rept_kernel_launches() == 0


def test_create_rejects_bad_config_before_touching_the_device():
    from paper_1811_09136_gb300.rept import Config
    lib = ctypes.CDLL(_build.build())
    h = ctypes.c_void_p()
    for cfg in (Config(0, 1, 1, 10, 0, 0, 0), Config(4, 0, 1, 10, 0, 0, 0), Config(4, 4, 1, 0, 0, 0, 0),
                Config(3, 5000, 1, 10, 0, 0, 0), Config(4, 4, 1, 10, 0, 0, 0, 12, 0), Config(4, 4, 1, 10, 0, 0, 0, 0, 1),
                Config(4, 4, 1, 10, 0, 0, 0, 0, 0, 0, 1), Config(4, 4, 1, 10, 0, 0, 0, 0, 0, 0, 0, 1),
                Config(4, 4, 1, 10, 0, 0, 0, 0, 2, 9), Config(4, 4, 1, 10, 0, 0, 0, 0, 3, 3),
                Config(3, 7, 1, 10, 0, 0, 0, 0, 0, 3)):
        assert lib.rept_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1


def test_estimates_from_counts_on_the_host():
    """rept_estimates_from_counts forms the global estimate on the host (no device work without
    local counts): (m^2/c) * sum for c <= m and MASCOT, (m/c1) * sum for c = c1 m; Algorithm 2's
    case is refused."""
    from paper_1811_09136_gb300 import rept
    lib = rept.load()
    g = ctypes.c_double()
    for m, c, flags, want in ((10, 10, 0, 10.0), (10, 4, 0, 25.0), (20, 100, 0, 4.0), (5, 8, rept.FLAG_MASCOT, 25 / 8)):
        proc = (ctypes.c_uint64 * c)(*[3 * i + 1 for i in range(c)])
        assert lib.rept_estimates_from_counts(m, c, flags, proc, None, 0, ctypes.byref(g), None, None) == 0
        assert g.value == float(sum(3 * i + 1 for i in range(c))) * want
    proc = (ctypes.c_uint64 * 7)()
    assert lib.rept_estimates_from_counts(3, 7, 0, proc, None, 0, ctypes.byref(g), None, None) == -1
    assert lib.rept_estimates_from_counts(0, 7, 0, proc, None, 0, ctypes.byref(g), None, None) == -1
