#!/usr/bin/env python3
"""Benchmark: stream edges/s of the REPT counting path at bit-exact counts on one GB300.

The default run prints ONE JSON line that covers the metric's terms:

  value        R-MAT graph, (a,b,c,d) = (0.57,0.19,0.19,0.05), scale 20 (1,048,576 nodes),
               16 * 2^20 draws deduplicated (15,700,820 distinct edges), seeded random stream
               order; p = 0.01 (m = 100), c = 100 processors, hash seed 1, ingested in batches of
               2^20 edges.  One step = reset the stream state, ingest the whole stream batch by
               batch, compute the global and local estimates (every row of the hot path).  Inputs
               resident in HBM when the timed region starts; the edges (126 MB) plus the device
               state (about 2 GB) exceed the 129 MB L2, so no flush is needed between steps.
  other_c      the same stream at c = 30
  powerlaw_4m  Chung-Lu, 2^22 nodes, exponent 2.1, degree cap 50,000, 64 * 2^20 edges; m = 20,
               c = 100 in five hash groups
  batched      256 independent streams (R-MAT / Chung-Lu, 1e4..2e6 nodes, 10-40 edges per node,
               p in {0.1, 0.05, 0.01}, c = m) through the batched path against a loop of the plain
               single-stream path, at the autotuned chunk and at chunks of 2^16 and 2^18 edges
  exact        every timed count compared with the oracle's counts (tests/golden/count_digests.json,
               written by tests/golden/make_count_digests.py from the oracle alone)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload headline|rmat_s20|powerlaw_20k|powerlaw_4m|batched|serve] [--quick]

`--workload rmat_s20|powerlaw_20k|powerlaw_4m` runs that single stream alone, `batched` the mix
alone, `serve` a Poisson request trace with continuous batching (p50/p99 latency).  Under torchrun
(N > 1) every rank counts its own replica of the streams with its own hash seed (the plain path has
no cross-stream exchange: replicas only) and `value` is the total over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "stream edges/sec at bit-exact counts, batched vs plain, % of HBM peak, 1 GB300"
BATCH = 1 << 20
SEED = 1
DIGESTS = os.path.join(ROOT, "tests", "golden", "count_digests.json")
MIX_SEED = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "rmat_s20", "powerlaw_20k", "powerlaw_4m", "batched", "serve"])
    ap.add_argument("--streams", type=int, default=256, help="batched: number of streams")
    ap.add_argument("--requests", type=int, default=1000, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--quick", action="store_true", help="skip the CPU baselines and the end-to-end legs")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split the headline stream's processors among the ranks (colour "
                         "sharding, strong scaling, one uint64 all-reduce per step) instead of replicas")
    return ap.parse_args()


# --------------------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(local_rank: int) -> str:
    import torch
    try:
        u = torch.cuda.get_device_properties(local_rank).uuid
        return "GPU-" + str(u)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local_rank]
        return str(local_rank)


def peaks():
    """(HBM GB/s, its source) from the measured peaks file, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d:
                return float(d[k]), "of measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "of fallback"


# Integer-issue peak of the GPU: 152 SMs x 4 schedulers, each issuing one warp instruction (32
# thread operations) per cycle; scaled by the SM clock sampled during the timed region.
SMS, SMSP_PER_SM, LANES = 152, 4, 32
# Thread operations the intersection needs per unit of work (the algorithmic count, not what the
# compiler emits): per scanned list entry with a stored colour, the colour filter of the larger
# endpoint's edge -- the ordered key (min, max: 2), the seed xor (2), SplitMix64 (64-bit add 2, three
# 64-bit xor-shifts 3 x 4, two 64-bit multiplies by constants 2 x 3: 20), the high word of the
# divisibility test (64-bit subtract 2, multiply 3, funnel shift 1, compare 1: 7) -- plus the entry's
# id mask, colour extraction and age test (3): 34; per scanned entry without stored colours, the
# age test and mask (2); per probe, the home-bucket hash and the 4-key compare (8); per counted
# wedge, the colours of both edges (2 x 31) and the three local updates (3): 65.
OPS_ENTRY_COLOURED, OPS_ENTRY_PLAIN, OPS_PROBE, OPS_WEDGE = 34, 2, 8, 65


# --------------------------------------------------------------------------- oracle digests
def load_digests() -> dict:
    try:
        with open(DIGESTS) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def digest_key(name, m, c, seed):
    return f"{name}|m={m}|c={c}|seed={seed}"


def compare_with_oracle(digests, key, stream, proc, local, tau_hat) -> dict:
    """The timed counts against the oracle's (bit for bit) and the estimate within 1e-12."""
    d = digests.get(key)
    if d is None:
        return {"checked": False, "why": f"no oracle digest for {key}"}
    if d["input_sha256"] != stream.sha256():
        return {"checked": False, "why": "input differs from the one the digest was made for"}
    local = np.ascontiguousarray(local, dtype=np.uint64)
    same_proc = [str(int(x)) for x in proc] == d["tau_proc"]
    same_local = hashlib.sha256(local.astype("<u8").tobytes()).hexdigest() == d["local_sha256"]
    ref = float.fromhex(d["tau_hat"])
    close = abs(tau_hat - ref) <= 1e-12 * max(abs(ref), 1.0)
    return {"checked": True, "identical": bool(same_proc and same_local and close), "tau_proc": same_proc,
            "local": same_local, "tau_hat_within_1e-12": close}


# --------------------------------------------------------------------------- workloads
WORKLOADS = {
    # name: (m, c, description)
    "rmat_s20": (100, 100, "R-MAT scale 20, ef 16"),
    "powerlaw_20k": (10, 10, "Chung-Lu 20,000 nodes, exponent 2.3, 200,000 edges"),
    "powerlaw_4m": (20, 100, "Chung-Lu 2^22 nodes, exponent 2.1, degree cap 50,000, 64 * 2^20 edges"),
}


def workload(name):
    from paper_1811_09136_gb300 import graphgen
    return graphgen.cached(name)


def cpu_sample_rate(s, m, c, budget_s=15.0):
    """The oracle (sequential CPU REPT) on a prefix of the same stream, sized to ~budget_s seconds."""
    import oracle
    n_edges = 1 << 14
    while True:
        t = time.perf_counter()
        oracle.rept_stream(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, m, c, SEED, pair_counters=False)
        spent = time.perf_counter() - t
        if spent > budget_s / 4 or n_edges >= len(s):
            break
        n_edges = min(len(s), n_edges * 4)
    return n_edges, spent


def kernel_source_sha16() -> str:
    """Digest of the kernel sources: a recorded ncu traffic figure is reported only for the kernels
    it was captured from."""
    h = hashlib.sha256()
    for f in ("rept_kernels.cuh", "rept_common.cuh"):
        with open(os.path.join(ROOT, "paper_1811_09136_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) per k_intersect launch from an ncu capture, keyed by (workload, c, digest
# of the kernel sources at capture time).  A figure whose digest no longer matches the sources is not
# reported (traffic null).
K3_TRAFFIC: dict = {("rmat_s20", 100, "6093804f85a48125"): 864792474.0}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank, pg):
    """The CPU oracle, as it stands, on the host cores: a bounded prefix of the stream per step."""
    if rank != 0:
        return 0
    name = args.workload if args.workload in WORKLOADS else "rmat_s20"
    s = workload(name)
    m, c, desc = WORKLOADS[name]
    import oracle
    # a step of about 2 s at most, so that --steps K --warmup W stays within a few minutes
    n_edges, _ = cpu_sample_rate(s, m, c, budget_s=2.0)
    for _ in range(args.warmup):
        oracle.rept_stream(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, m, c, SEED, pair_counters=False)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.rept_stream(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, m, c, SEED, pair_counters=False)
    el = time.perf_counter() - t
    v = args.steps * n_edges / el
    sample = f"first {n_edges} edges of the stream per step (sequential REPT, {c} processors)"
    line = {"metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{name}: {desc}, {len(s)} edges, m={m}, c={c}, seed={SEED}, "
                                   f"batches of {BATCH}", "sample": sample},
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- single-stream leg
def time_steps(r, src, dst, T, steps, stream):
    """`steps` full passes (reset, all batches, estimates) bracketed by CUDA events on `stream`."""
    import torch

    def step():
        r.reset()
        for off in range(0, T, BATCH):
            r.ingest(src[off:off + BATCH], dst[off:off + BATCH])
        return r.estimates(local=True)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g = None
    for _ in range(steps):
        g, _ = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), g, step


def single_leg(name, m, c, seed, steps, warmup, dev, pg, digests, clock_mhz_hint=None, e2e=False, world=1):
    """One stream: timed steps, per-kernel event times, the oracle comparison, and the intersection
    kernel's algorithmic bytes and thread operations (from an untimed pass with work counters)."""
    import torch
    from paper_1811_09136_gb300 import rept

    s = workload(name)
    T = len(s)
    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(s.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(s.dst.view(np.int32)).to(dev)
    r = rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=T, max_batch=BATCH, flags=rept.FLAG_PROFILE)
    _, _, step = time_steps(r, src, dst, T, 0, stream)
    for _ in range(warmup):
        step()
    r.kernel_times(clear=True)
    barrier(pg)
    torch.cuda.synchronize(dev)
    launches0 = rept.kernel_launches()
    ms, g, _ = time_steps(r, src, dst, T, steps, stream)
    barrier(pg)
    launches = rept.kernel_launches() - launches0
    kt = r.kernel_times(clear=True)
    ms_max = max_over_ranks(pg, ms, dev)
    proc, local_t = r.counts()
    local = local_t.cpu().numpy().view(np.uint64)
    exact = compare_with_oracle(digests, digest_key(name, m, c, seed), s, proc, local, g)

    # work counters of the intersection (one extra, untimed pass)
    with rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=T, max_batch=BATCH,
                         flags=rept.FLAG_WORK_COUNTERS) as rw:
        for off in range(0, T, BATCH):
            rw.ingest(src[off:off + BATCH], dst[off:off + BATCH])
        proc_w, _ = rw.counts()
        st = rw.stats()
    assert np.array_equal(proc_w, proc), "work-counter pass disagrees with the timed pass"
    coloured = (c + m - 1) // m == 1 and 2 <= m <= 256 and s.n_nodes <= (1 << 24)
    edges = T - st["self_loops"]
    k3_bytes = 24 * edges + 8 * st["small_entries"] + 8 * st["probes"] + 16 * st["counted"]
    k3_ops = ((OPS_ENTRY_COLOURED if coloured else OPS_ENTRY_PLAIN) * st["small_entries"] +
              OPS_PROBE * st["probes"] + OPS_WEDGE * st["counted"])
    k3_ms, k3_n = kt["intersect"]
    k3_s = k3_ms / steps * 1e-3
    hbm, hbm_src = peaks()
    achieved = k3_bytes / k3_s / 1e9
    ws_bytes = 8 * T + 8 * st["pool_used"] + 28 * s.n_nodes
    out = {
        "edges": T, "value": world * steps * T / (ms_max * 1e-3), "unit": "edges/s", "steps": steps,
        "warmup": warmup, "ms_per_step": ms_max / steps, "tau_hat": g, "semi_triangles": int(proc.sum()),
        "exact": exact, "gpu_launches": launches,
        "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items()},
        "work": {k: st[k] for k in ("small_entries", "probes", "wedges", "counted", "stored_edges",
                                    "class_items", "class_probes", "class_cycles")},
        "l2": (f"inputs and state larger than L2, no flush: {ws_bytes / 1e9:.2f} GB touched per step (edges, "
               f"node blocks written as they are handed out, per-node arrays cleared at every step's start)"
               if ws_bytes > (129 << 20) else "working set fits in L2 (no flush)"),
        "k3": {"bytes": k3_bytes, "ops": k3_ops, "seconds": k3_s, "launches": k3_n // max(steps, 1),
               "coloured": coloured},
        "hbm_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "peak_source": hbm_src},
    }
    tr = K3_TRAFFIC.get((name, c, kernel_source_sha16()))
    out["hbm_roofline"]["traffic"] = tr
    if e2e:
        h_src = torch.from_numpy(s.src.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_dst = torch.from_numpy(s.dst.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_loc = torch.empty(s.n_nodes, dtype=torch.float64).pin_memory().numpy()

        def step_host():
            r.reset()
            r.ingest_host(h_src, h_dst, batch=BATCH)
            return r.estimates_host(out=h_loc)

        step_host()
        barrier(pg)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for _ in range(steps):
            step_host()
        torch.cuda.synchronize(dev)
        el = max_over_ranks(pg, time.perf_counter() - t, dev)
        out["e2e"] = {"value": world * steps * T / el, "unit": "edges/s", "h2d_bytes_per_step": 8 * T,
                      "d2h_bytes_per_step": 8 + 8 * s.n_nodes}
    r.close()
    return out


def issue_roofline(k3, sm_mhz):
    mhz = sm_mhz or 2070.0
    peak = SMS * SMSP_PER_SM * LANES * mhz * 1e6 / 1e12  # T thread-ops/s
    achieved = k3["ops"] / k3["seconds"] / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "peak_source": f"152 SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz (sampled SM clock)"}


# --------------------------------------------------------------------------- batched leg
def batched_leg(args, world, rank, pg, digests, e2e=False, chunks=(1 << 16, 1 << 18)):
    """256 independent streams: the batched path (one launch per step for all streams, CUDA graphs)
    against a loop of the plain single-stream path, at identical counts; both compared with the
    oracle.  Chunk size and tile width are autotuned on a 16-stream sample of the mix."""
    from paper_1811_09136_gb300 import batched

    seed = MIX_SEED + 7919 * rank
    specs = batched.mix_specs(args.streams, seed=seed)
    t = time.perf_counter()
    streams = batched.generate_all(specs)
    gen_s = time.perf_counter() - t
    params = [(sp.m, sp.m, sp.hash_seed) for sp in specs]
    E = sum(len(x) for x in streams)
    sample = sorted(range(len(streams)), key=lambda i: len(streams[i]))[::max(1, len(streams) // 16)][:16]
    b, tm, timings = batched.autotune([streams[i] for i in sample], [params[i] for i in sample],
                                      key=f"mix{args.streams}")
    res_b, t_b = batched.run_batched(streams, params, batch=b, tile_max=tm)
    res_q, t_q = batched.run_batched(streams, params, batch=b, tile_max=tm, persistent=True)
    res_p, t_p = batched.run_plain(streams, params, batch=b, tile_max=tm)
    assert all(np.array_equal(x.proc, y.proc) and np.array_equal(x.local, y.local) for x, y in zip(res_b, res_q))
    same = all(np.array_equal(x.proc, y.proc) and np.array_equal(x.local, y.local) for x, y in zip(res_b, res_p))
    assert same, "batched and plain counts differ"
    checks = [compare_with_oracle(digests, digest_key(f"mix{MIX_SEED}#{sp.index}", sp.m, sp.m, sp.hash_seed),
                                  st, r.proc, r.local, r.tau_hat)
              for sp, st, r in zip(specs, streams, res_b)]
    checked = [c for c in checks if c["checked"]]
    exact = {"streams": len(checks), "checked": len(checked),
             "identical": bool(checked) and all(c["identical"] for c in checked)}
    t_b = max_over_ranks(pg, t_b)
    t_q = max_over_ranks(pg, t_q)
    t_p = max_over_ranks(pg, t_p)
    out = {"streams": args.streams, "edges": E, "value": world * E / t_b, "unit": "edges/s", "seconds": t_b,
           "batch": b, "tile_max": tm, "autotune_s": timings, "generation_s": gen_s,
           "persistent": {"value": world * E / t_q, "unit": "edges/s", "seconds": t_q,
                          "what": "one cooperative launch per round runs every step for every stream"},
           "plain_loop": {"value": world * E / t_p, "unit": "edges/s", "seconds": t_p},
           "batched_over_plain": t_p / t_b, "identical_counts": same, "exact": exact, "by_chunk": {}}
    for ch in chunks:
        rb, tb = batched.run_batched(streams, params, batch=ch, tile_max=tm)
        rq, tq = batched.run_batched(streams, params, batch=ch, tile_max=tm, persistent=True)
        rp, tp = batched.run_plain(streams, params, batch=ch, tile_max=tm)
        ok = all(np.array_equal(x.proc, y.proc) and np.array_equal(x.local, y.local) and
                 np.array_equal(x.proc, z.proc) and np.array_equal(x.local, q.local)
                 for x, y, z, q in zip(rb, rp, res_b, rq))
        assert ok, f"counts differ at chunk {ch}"
        tb, tq, tp = max_over_ranks(pg, tb), max_over_ranks(pg, tq), max_over_ranks(pg, tp)
        out["by_chunk"][str(ch)] = {"batched": world * E / tb, "persistent": world * E / tq,
                                    "plain_loop": world * E / tp, "batched_over_plain": tp / tb,
                                    "persistent_over_plain": tp / tq, "identical_counts": ok}
    if e2e:
        rb, te = batched.run_batched(streams, params, batch=b, tile_max=tm, host_io=True)
        assert all(np.array_equal(x.proc, y.proc) for x, y in zip(rb, res_b))
        te = max_over_ranks(pg, te)
        out["e2e"] = {"value": world * E / te, "unit": "edges/s", "h2d_bytes_per_step": 8 * E,
                      "d2h_bytes_per_step": sum(8 + 8 * sp.m + 4 for sp in specs)}
    return out, streams, params


def batched_cpu_baseline(streams, params, budget_s=10.0):
    """The oracle on the first 2^16 edges of up to 16 streams of the mix, one host core."""
    import oracle
    done, spent, used = 0, 0.0, 0
    for s, (m, c, seed) in zip(streams[::max(1, len(streams) // 16)], params[::max(1, len(streams) // 16)]):
        n = min(len(s), 1 << 16)
        t = time.perf_counter()
        oracle.rept_stream(s.src[:n], s.dst[:n], s.n_nodes, m, c, seed, pair_counters=False)
        spent += time.perf_counter() - t
        done += n
        used += 1
        if spent > budget_s:
            break
    return {"value": done / spent, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"first {min(1 << 16, 10**12)} edges of {used} streams of the mix (sequential REPT)"}


# --------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local, pg):
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    digests = load_digests()
    seed = SEED + rank  # an independent replica (own hash seed) per rank
    clocks = ClockSampler(gpu_uuid(local)).start()
    head = single_leg("rmat_s20", 100, 100, seed, args.steps, args.warmup, dev, pg, digests,
                      e2e=not args.quick, world=world)
    clk = clocks.stop()
    c30 = single_leg("rmat_s20", 100, 30, seed, 3, 1, dev, pg, digests, world=world)
    p4m = single_leg("powerlaw_4m", 20, 100, seed, 3, 1, dev, pg, digests, world=world)
    bat, streams, params = batched_leg(args, world, rank, pg, digests, e2e=not args.quick)

    cpu = cpu_parallel = None
    if rank == 0 and world == 1 and not args.quick:
        s = workload("rmat_s20")
        n_edges, el = cpu_sample_rate(s, 100, 100)
        cpu = {"value": n_edges / el, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_edges} edges of the R-MAT scale-20 stream (sequential REPT, 100 processors); "
                         f"early edges meet smaller sets, so this overstates the oracle's full-stream rate",
               "nproc": os.cpu_count()}
        import oracle
        threads = max(1, min(100, os.cpu_count() or 1))
        t0 = time.perf_counter()
        oracle.rept_stream_parallel(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, 100, 100, SEED, threads)
        el_p = time.perf_counter() - t0
        cpu_parallel = {"value": n_edges / el_p, "unit": "edges/s", "threads": threads, "nproc": os.cpu_count(),
                        "kind": "paper multi-core design (one thread per processor, each with its own pass)",
                        "sample": f"first {n_edges} edges of the same stream"}
        bat["cpu_baseline"] = batched_cpu_baseline(streams, params)

    if rank == 0:
        hbm = head["hbm_roofline"]
        alu = issue_roofline(head["k3"], clk.get("sm_mhz"))
        roof = dict(alu)
        roof.update({"kernel": "k_intersect", "traffic": hbm["traffic"],
                     "algorithmic_ops_per_step": head["k3"]["ops"],
                     "kernel_ms_per_step": head["k3"]["seconds"] * 1e3,
                     "launches_per_step": head["k3"]["launches"],
                     "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "peak_source")},
                     "algorithmic_bytes_per_step": head["k3"]["bytes"]})
        for leg in (c30, p4m):
            leg["hbm_roofline"]["issue"] = issue_roofline(leg["k3"], clk.get("sm_mhz"))
        all_exact = all(x["exact"].get("identical", False) for x in (head, c30, p4m)) and bat["exact"]["identical"]
        line = {
            "metric": METRIC, "value": head["value"], "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": f"rmat_s20: R-MAT scale 20, ef 16, {head['edges']} edges, m=100, c=100, "
                                   f"seed={SEED}, batches of {BATCH}",
                       "parallelism": "replicas" if world > 1 else "single", "l2": head["l2"],
                       "tau_hat": head["tau_hat"], "semi_triangles": head["semi_triangles"]},
            "identical_to_oracle": all_exact,
            "exact": head["exact"],
            "roofline": roof,
            "kernel_ms_per_step": head["kernel_ms_per_step"],
            "work": head["work"],
            "clocks": clk, "e2e": head.get("e2e"), "gpu_launches": head["gpu_launches"],
            "cpu_baseline": cpu, "cpu_parallel": cpu_parallel,
            "other_c": {k: c30[k] for k in ("value", "ms_per_step", "tau_hat", "exact", "kernel_ms_per_step")},
            "powerlaw_4m": {k: p4m[k] for k in ("edges", "value", "ms_per_step", "steps", "tau_hat", "exact",
                                                "kernel_ms_per_step", "work", "hbm_roofline")},
            "batched": bat,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_single_only(args, world, rank, local, pg):
    """--workload rmat_s20|powerlaw_20k|powerlaw_4m: that stream alone."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, c, desc = WORKLOADS[args.workload]
    clocks = ClockSampler(gpu_uuid(local)).start()
    leg = single_leg(args.workload, m, c, SEED + rank, args.steps, args.warmup, dev, pg, load_digests(),
                     e2e=not args.quick, world=world)
    clk = clocks.stop()
    if rank == 0:
        roof = issue_roofline(leg["k3"], clk.get("sm_mhz"))
        roof.update({"kernel": "k_intersect", "hbm": leg["hbm_roofline"]})
        line = {"metric": METRIC, "value": leg["value"], "unit": "edges/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {desc}, {leg['edges']} edges, m={m}, c={c}, "
                                       f"seed={SEED}, batches of {BATCH}", "l2": leg["l2"]},
                "identical_to_oracle": leg["exact"].get("identical", False), "exact": leg["exact"],
                "roofline": roof, "kernel_ms_per_step": leg["kernel_ms_per_step"], "work": leg["work"],
                "clocks": clk, "e2e": leg.get("e2e"), "gpu_launches": leg["gpu_launches"]}
        print(json.dumps(line), flush=True)
    return 0


def run_batched_only(args, world, rank, local, pg):
    import torch
    torch.cuda.set_device(local)
    bat, streams, params = batched_leg(args, world, rank, pg, load_digests(), e2e=not args.quick)
    if rank == 0:
        line = {"metric": METRIC, "value": bat["value"], "unit": "edges/s", "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": 1e3 * bat["seconds"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": f"batched: {args.streams} streams (R-MAT / Chung-Lu, n log-uniform in "
                                       f"[1e4, 2e6], 10-40 edges per node, p in {{0.1, 0.05, 0.01}}, c = m), "
                                       f"{bat['edges']} edges"},
                "identical_to_oracle": bat["exact"]["identical"], "batched": bat, "e2e": bat.get("e2e")}
        print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, world, rank, local, pg):
    """--shard: the R-MAT scale-20 stream (m = c = 100) counted once by all ranks together, each rank
    keeping its own processors (whole colour ranges) and ingesting the whole stream; a step ends with
    the all-reduce of the counts and the estimates from the sums.  Total work is fixed (strong
    scaling)."""
    import torch
    from paper_1811_09136_gb300 import shard

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = workload("rmat_s20")
    T = len(s)
    src = torch.from_numpy(s.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(s.dst.view(np.int32)).to(dev)
    ss = shard.ShardedStream(s.n_nodes, 100, 100, SEED, world, rank, pg, expected_edges=T, max_batch=BATCH)

    def step():
        ss.reset()
        for off in range(0, T, BATCH):
            ss.ingest(src[off:off + BATCH], dst[off:off + BATCH])
        return ss.estimates(local=True)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(gpu_uuid(local)).start()
    barrier(pg)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g, _ = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(pg)
    clk = clocks.stop()
    ms = max_over_ranks(pg, ev0.elapsed_time(ev1), dev)
    proc, loc = ss.counts()
    exact = compare_with_oracle(load_digests(), digest_key("rmat_s20", 100, 100, SEED), s, proc,
                                loc.cpu().numpy().view(np.uint64), g)
    if rank == 0:
        line = {"metric": METRIC, "value": args.steps * T / (ms * 1e-3), "unit": "edges/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32/u64",
                "data": "synthetic",
                "config": {"workload": f"rmat_s20: R-MAT scale 20, ef 16, {T} edges, m=100, c=100, seed={SEED}, "
                                       f"batches of {BATCH}", "parallelism": f"colour shards x{world}",
                           "shard": list(ss.range)},
                "identical_to_oracle": exact.get("identical", False), "exact": exact, "clocks": clk}
        print(json.dumps(line), flush=True)
    ss.close()
    return 0


def run_serving(args, world, rank, local, pg):
    """A Poisson request trace served with continuous batching: aggregate edges/s and latency."""
    import torch
    from paper_1811_09136_gb300 import serve

    torch.cuda.set_device(local)
    t = time.perf_counter()
    reqs = serve.build_trace(n_requests=args.requests, rate=args.rate, seed=5 + rank)
    gen_s = time.perf_counter() - t
    rep = serve.serve(reqs)
    sm = rep.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": sm["edges_per_s"] * world, "unit": "edges/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 * sm["makespan_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": f"serve: {args.requests} requests, Poisson arrivals at {args.rate}/s, "
                                       f"streams from the batched mix plus an R-MAT scale-24 ef-16 stream "
                                       f"(p=0.01, c=100) every 50th request, chunks of 2^16-2^20",
                           "generation_s": gen_s},
                "serving": sm}
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.gpus != world and world > 1:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    if args.impl == "reference":
        rc = run_reference(args, world, rank, pg)
    elif args.workload == "batched":
        rc = run_batched_only(args, world, rank, local, pg)
    elif args.workload == "serve":
        rc = run_serving(args, world, rank, local, pg)
    elif args.shard:
        rc = run_sharded(args, world, rank, local, pg)
    elif args.workload == "headline":
        rc = run_ours(args, world, rank, local, pg)
    else:
        rc = run_single_only(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
