#!/usr/bin/env python3
"""Benchmark: stream edges/s of the REPT counting path at bit-exact counts on one GB300.

Workload (default): R-MAT graph, (a,b,c,d) = (0.57,0.19,0.19,0.05), scale 20
(1,048,576 nodes), 16 * 2^20 draws deduplicated (15,700,820 distinct edges),
seeded random stream order; p = 0.01 (m = 100), c = 100 processors, hash
seed 1, ingested in batches of 2^20 edges.  One step = reset the stream
state, ingest the whole stream batch by batch, compute the global and local
estimates (every row of the hot path).  Inputs already resident in HBM when
the timed region starts; the edge list (126 MB) plus the device state
(~0.9 GB) exceed the 129 MB L2, so no explicit flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--c 100]
                  [--workload rmat_s20|powerlaw_20k|powerlaw_4m|batched|serve]

The other workloads: powerlaw_20k (Chung-Lu, 20,000 nodes, m = c = 10) and powerlaw_4m (Chung-Lu,
2^22 nodes, 64 * 2^20 edges, m = 20, c = 100 in five hash groups) in the same single-stream form;
batched (256 independent streams, the batched path against a loop of the plain path); serve (a
Poisson request trace with continuous batching, p50/p99 latency).

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank counts its
own replica of the stream with its own hash seed (the plain path has no
cross-stream exchange: replicas only) and `value` is the total over ranks.
"""
from __future__ import annotations

import argparse
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
M = 100
SEED = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--c", type=int, default=100, help="processors (the workload runs at c=30 and c=100)")
    ap.add_argument("--workload", default="rmat_s20",
                    choices=["rmat_s20", "powerlaw_20k", "powerlaw_4m", "batched", "serve"],
                    help="rmat_s20 (default, the headline), powerlaw_20k, powerlaw_4m, batched (256 streams, "
                         "batched vs a loop of the plain path), serve (Poisson request trace)")
    ap.add_argument("--streams", type=int, default=256, help="batched: number of streams")
    ap.add_argument("--requests", type=int, default=1000, help="serve: number of requests")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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


def hbm_peak():
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


# --------------------------------------------------------------------------- workload
WORKLOADS = {
    # name: (m, c, description)
    "rmat_s20": (100, None, "R-MAT scale 20, ef 16"),
    "powerlaw_20k": (10, 10, "Chung-Lu 20,000 nodes, exponent 2.3, 200,000 edges"),
    "powerlaw_4m": (20, 100, "Chung-Lu 2^22 nodes, exponent 2.1, degree cap 50,000, 64 * 2^20 edges"),
}


def workload(name="rmat_s20"):
    from paper_1811_09136_gb300 import graphgen
    return graphgen.cached(name)


def cpu_sample_rate(s, m, c, budget_s=15.0):
    """The oracle (sequential CPU REPT) on a prefix of the same stream, sized to ~budget_s seconds."""
    import oracle
    n_edges = 1 << 14
    spent = 0.0
    while True:
        t = time.perf_counter()
        oracle.rept_stream(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, m, c, SEED, pair_counters=False)
        spent = time.perf_counter() - t
        if spent > budget_s / 4 or n_edges >= len(s):
            break
        n_edges = min(len(s), n_edges * 4)
    return n_edges, spent


# DRAM bytes (read + write) per k_intersect launch, the mean over the 15 launches of one step from an
# ncu capture of the current kernel (profiles/k_intersect_rmat_s20_c100.md); absent for workloads not
# captured.  Must be removed when the kernel changes.
K3_TRAFFIC = {("rmat_s20", 100): 786.7e6}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank, pg):
    """The CPU oracle, as it stands, on the host cores: a bounded prefix of the stream per step."""
    if rank != 0:
        return 0
    name = args.workload if args.workload in WORKLOADS else "rmat_s20"
    s = workload(name)
    m, c, desc = WORKLOADS[name]
    c = args.c if c is None else c
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


# --------------------------------------------------------------------------- our arm
def single_stream_setup(args, rank):
    name = args.workload
    s = workload(name)
    m, c, desc = WORKLOADS[name]
    c = args.c if c is None else c
    return s, m, c, SEED + rank, desc  # independent replica (own hash seed) per rank


def time_single_stream(r, src, dst, T, steps, stream):
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


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1811_09136_gb300 import rept

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, m, c, seed, desc = single_stream_setup(args, rank)
    T = len(s)
    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(s.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(s.dst.view(np.int32)).to(dev)
    r = rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=T, max_batch=BATCH, flags=rept.FLAG_PROFILE)

    _, _, step = time_single_stream(r, src, dst, T, 0, stream)
    for _ in range(args.warmup):
        step()
    r.kernel_times(clear=True)
    clocks = ClockSampler(gpu_uuid(local))
    barrier(pg)
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = rept.kernel_launches()
    ms, g, _ = time_single_stream(r, src, dst, T, args.steps, stream)
    barrier(pg)
    launches = rept.kernel_launches() - launches0
    clk = clocks.stop()
    kt = r.kernel_times(clear=True)
    ms_max = max_over_ranks(pg, ms, dev)
    proc, _ = r.counts()

    # ---- algorithmic bytes of the intersection kernel (one extra, untimed pass with work counters)
    with rept.ReptStream(s.n_nodes, m, c, seed, expected_edges=T, max_batch=BATCH,
                         flags=rept.FLAG_WORK_COUNTERS) as rw:
        for off in range(0, T, BATCH):
            rw.ingest(src[off:off + BATCH], dst[off:off + BATCH])
        proc_w, _ = rw.counts()
        st = rw.stats()
    assert np.array_equal(proc_w, proc), "work-counter pass disagrees with the timed pass"
    # per list entry scanned: 8 B {neighbour (with its colour in the top bits), stream index}
    per_entry = 8
    k3_bytes = 24 * (T - st["self_loops"]) + per_entry * st["small_entries"] + 8 * st["probes"] + 16 * st["counted"]
    # bytes a step touches: its edges, the node blocks it fills (8-byte slots plus colour bytes) and
    # the per-node arrays (meta, local, add)
    ws_bytes = 8 * T + per_entry * st["pool_used"] + 20 * s.n_nodes
    k3_ms, k3_n = kt["intersect"]
    k3_ms_step = k3_ms / args.steps
    peak, peak_src = hbm_peak()
    achieved = k3_bytes / (k3_ms_step * 1e-3) / 1e9

    # ---- the same stream at c = 30 (the workload is quoted at c = 30 and c = 100)
    other_c = None
    if args.workload == "rmat_s20" and c != 30:
        with rept.ReptStream(s.n_nodes, m, 30, seed, expected_edges=T, max_batch=BATCH) as r30:
            _, _, step30 = time_single_stream(r30, src, dst, T, 0, stream)
            step30()
            ms30, g30, _ = time_single_stream(r30, src, dst, T, 3, stream)
        other_c = {"c": 30, "edges_per_s": 3 * T / (ms30 * 1e-3), "ms_per_step": ms30 / 3, "tau_hat": g30}

    # ---- end to end through the C-ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
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
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize(dev)
        el = max_over_ranks(pg, time.perf_counter() - t, dev)
        e2e = {"value": world * args.steps * T / el, "unit": "edges/s", "h2d_bytes_per_step": 8 * T,
               "d2h_bytes_per_step": 8 + 8 * s.n_nodes}

    cpu = cpu_parallel = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_edges, el = cpu_sample_rate(s, m, c)
        cpu = {"value": n_edges / el, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"first {n_edges} edges of the same stream (sequential REPT, {c} processors); "
                         f"early edges meet smaller sets, so this overstates the oracle's full-stream rate",
               "nproc": os.cpu_count()}
        # the paper's multi-core design on the same sample: one thread per processor
        import oracle
        threads = max(1, min(c, os.cpu_count() or 1))
        t0 = time.perf_counter()
        oracle.rept_stream_parallel(s.src[:n_edges], s.dst[:n_edges], s.n_nodes, m, c, SEED, threads)
        el_p = time.perf_counter() - t0
        cpu_parallel = {"value": n_edges / el_p, "unit": "edges/s", "threads": threads, "nproc": os.cpu_count(),
                        "kind": "paper multi-core design (one thread per processor, each with its own pass)",
                        "sample": f"first {n_edges} edges of the same stream"}

    if rank == 0:
        value = world * args.steps * T / (ms_max * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}, {T} edges, m={m}, c={c}, seed={SEED}, "
                                   f"batches of {BATCH}",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": (f"inputs and state larger than L2, no flush: {ws_bytes / 1e9:.2f} GB touched per "
                              f"step (edges, node blocks in use, per-node arrays; every step also resets them)"
                              if ws_bytes > (129 << 20) else "working set fits in L2 (no flush)"),
                       "tau_hat": g, "semi_triangles": int(proc.sum()), "other_c": other_c},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": K3_TRAFFIC.get((args.workload, c)),
                         "kernel": "k_intersect",
                         "limiter": "integer issue where colours are kept (ncu: 76 % issue active, ALU pipe "
                                    "66 %, DRAM 9 %); algorithmic bytes understate the kernel's load",
                         "peak_source": peak_src, "algorithmic_bytes_per_step": k3_bytes,
                         "kernel_ms_per_step": k3_ms_step, "launches_per_step": k3_n // args.steps},
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
            "work": {k: st[k] for k in ("small_entries", "small_slots", "probes", "probe_slots", "wedges",
                                        "counted", "stored_edges", "class_items", "class_probes",
                                        "class_cycles")},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "cpu_baseline": cpu,
            "cpu_parallel": cpu_parallel,
        }
        print(json.dumps(line), flush=True)
    r.close()
    return 0


def run_batched_mix(args, world, rank, local, pg):
    """256 independent streams: the batched path (one launch per step for all streams, CUDA graphs)
    against a loop of the plain single-stream path, at identical counts.  Batch size and tile width
    are autotuned on a 16-stream sample of the mix."""
    import torch
    from paper_1811_09136_gb300 import batched

    torch.cuda.set_device(local)
    specs = batched.mix_specs(args.streams, seed=1000 + 7919 * rank)
    t = time.perf_counter()
    streams = batched.generate_all(specs)
    gen_s = time.perf_counter() - t
    params = [(sp.m, sp.m, sp.hash_seed) for sp in specs]
    E = sum(len(x) for x in streams)
    sample = sorted(range(len(streams)), key=lambda i: len(streams[i]))[::max(1, len(streams) // 16)][:16]
    b, tm, timings = batched.autotune([streams[i] for i in sample], [params[i] for i in sample],
                                      key=f"mix{args.streams}")
    res_b, t_b = batched.run_batched(streams, params, batch=b, tile_max=tm)
    res_p, t_p = batched.run_plain(streams, params, batch=b, tile_max=tm)
    same = all(np.array_equal(x.proc, y.proc) and np.array_equal(x.local, y.local) for x, y in zip(res_b, res_p))
    assert same, "batched and plain counts differ"
    t_b = max_over_ranks(pg, t_b)
    t_p = max_over_ranks(pg, t_p)
    if rank == 0:
        line = {"metric": METRIC, "value": world * E / t_b, "unit": "edges/s", "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": 1e3 * t_b, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": f"batched: {args.streams} streams (R-MAT / Chung-Lu, n log-uniform in "
                                       f"[1e4, 2e6], 10-40 edges per node, p in {{0.1, 0.05, 0.01}}, c = m), "
                                       f"{E} edges", "batch": b, "tile_max": tm, "autotune_s": timings,
                           "generation_s": gen_s},
                "plain_loop": {"value": world * E / t_p, "unit": "edges/s", "ms": 1e3 * t_p},
                "batched_over_plain": t_p / t_b, "identical_counts": same}
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args, world, rank, local, pg):
    """A Poisson request trace served with continuous batching: aggregate edges/s and latency."""
    import torch
    from paper_1811_09136_gb300 import serve

    torch.cuda.set_device(local)
    t = time.perf_counter()
    reqs = serve.build_trace(n_requests=args.requests, seed=5 + rank)
    gen_s = time.perf_counter() - t
    rep = serve.serve(reqs)
    sm = rep.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": sm["edges_per_s"] * world, "unit": "edges/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 * sm["makespan_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": f"serve: {args.requests} requests, Poisson arrivals at 200/s, streams "
                                       f"from the batched mix plus an R-MAT scale-24 ef-16 stream (p=0.01, "
                                       f"c=100) every 50th request, chunks of 2^16-2^20",
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
        rc = run_batched_mix(args, world, rank, local, pg)
    elif args.workload == "serve":
        rc = run_serving(args, world, rank, local, pg)
    else:
        rc = run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
