"""The division-free modulo behind the colour hash equals % for every tested 64-bit value (host build)."""
import os
import subprocess

from paper_1811_09136_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fast_mod_matches_percent(tmp_path):
    exe = str(tmp_path / "fastmod_check")
    subprocess.check_call([_build._nvcc(), "-O2", "-std=c++17", "-I", _build.CSRC, "-I", _build.INCLUDE, "-o", exe,
                           os.path.join(HERE, "native", "fastmod_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches: 0" in out.stdout
