"""bench.py's reference arm runs the CPU oracle only, so its JSON contract is checked here without a
GPU: one line on rank 0 with the metric, the timing keys, impl = reference, an e2e object with no
host-device bytes and a cpu_baseline describing the run; under torchrun with two ranks, rank 0
alone prints and both exit 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _last_json(out: str) -> dict:
    lines = [l for l in out.strip().splitlines() if l.startswith("{")]
    assert lines, out
    return json.loads(lines[-1])


def _check(d: dict, steps: int, warmup: int):
    assert d["impl"] == "reference" and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == steps and d["warmup"] == warmup and d["ms_per_step"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["config"]["workload"].startswith("powerlaw_20k")


def test_reference_arm_one_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "powerlaw_20k",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    _check(_last_json(out.stdout), 2, 1)


def test_reference_arm_two_ranks_rank0_prints():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "powerlaw_20k", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    _check(json.loads(lines[0]), 1, 1)


def test_oracle_comparison_of_timed_counts():
    """bench.compare_with_oracle: identical counts pass; one changed tau^(i), one changed local
    count, an estimate off by more than 1e-12 relative, or another input each fail."""
    import hashlib
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_1811_09136_gb300 import graphgen as gg
    s = gg.gnp(30, 0.3, 5, 6)
    proc = np.array([3, 0, 7], dtype=np.uint64)
    local = np.arange(30, dtype=np.uint64)
    dig = {"k": {"input_sha256": s.sha256(), "tau_proc": ["3", "0", "7"],
                 "local_sha256": hashlib.sha256(local.astype("<u8").tobytes()).hexdigest(),
                 "tau_hat": (1234.5).hex()}}
    assert bench.compare_with_oracle(dig, "k", s, proc, local, 1234.5)["identical"]
    assert not bench.compare_with_oracle(dig, "k", s, proc + np.uint64(1), local, 1234.5)["identical"]
    bad = local.copy()
    bad[7] += np.uint64(1)
    assert not bench.compare_with_oracle(dig, "k", s, proc, bad, 1234.5)["identical"]
    assert not bench.compare_with_oracle(dig, "k", s, proc, local, 1234.5 * (1 + 1e-11))["identical"]
    assert bench.compare_with_oracle(dig, "k", s, proc, local, 1234.5 * (1 + 1e-13))["identical"]
    assert not bench.compare_with_oracle(dig, "k", gg.gnp(30, 0.3, 5, 7), proc, local, 1234.5)["checked"]
    assert not bench.compare_with_oracle(dig, "other", s, proc, local, 1234.5)["checked"]
