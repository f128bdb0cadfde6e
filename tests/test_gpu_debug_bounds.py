"""The bounds-checked debug build (REPT_DEBUG_BOUNDS), a stand-in for a memory checker: every pool,
queue and node index that the kernels use is checked, and a failed check is recorded and reported
instead of touching memory.  The parity cases of tests/debug_bounds_run.py run through it in a
child process (REPT_LIBRARY selects the library) and must finish with the oracle's counts and no
failed check."""
import os
import subprocess
import sys

import pytest

from paper_1811_09136_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_compiles_every_check(tmp_path):
    """The checks compile (no GPU needed)."""
    out = str(tmp_path / "librept_debug_check.so")
    cmd = [_build._nvcc(), "-DREPT_DEBUG_BOUNDS", *_build.NVCC_FLAGS, "-I", _build.INCLUDE, "-I", _build.CSRC,
           "-shared", "-o", out, os.path.join(_build.CSRC, "rept_api.cu")]
    subprocess.check_call(cmd)
    assert os.path.getsize(out) > 0


@pytest.mark.gpu
def test_parity_under_bounds_checks():
    path = _build.build(debug_bounds=True)
    env = dict(os.environ, REPT_LIBRARY=path)
    out = subprocess.run([sys.executable, os.path.join(HERE, "debug_bounds_run.py")], env=env,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0 and "debug-bounds ok" in out.stdout, out.stdout[-3000:] + out.stderr[-3000:]
    assert "index check" not in out.stderr, out.stderr[-3000:]
