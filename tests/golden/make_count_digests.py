"""Write tests/golden/count_digests.json: the oracle's counts for the full-size workloads.

For every workload (a seeded synthetic stream and its m, c, hash seed) this runs the oracle's static
semi-triangle enumeration (oracle.semitriangles: a triangle counts for processor i when its two
earliest edges on the stream both carry processor i's colour, Section III) and the oracle's
estimators (oracle.estimates: Section III-A, III-B.1), and stores

  input_sha256   the stream's digest (node count, src, dst), so that a changed generator is caught
  tau_proc       every tau^(i), as decimal strings (uint64)
  local_sha256   SHA-256 of the uint64 array sum_i tau_v^(i) (little-endian, n_nodes entries)
  local_sum      its sum (3 * sum_i tau^(i) by Algorithm 1's updates)
  tau_hat        the global estimate, as float.hex

Only the oracle and the input generators are called here; nothing comes from the CUDA path.  The
bench compares its timed counts with these entries.

  python tests/golden/make_count_digests.py [--only rmat_s20 ...] [--mix N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1811_09136_gb300 import graphgen as gg  # noqa: E402

OUT = os.path.join(HERE, "count_digests.json")

# (workload, m, c, hash seed)
SINGLE = [("powerlaw_20k", 10, 10, 1), ("rmat_s20", 100, 100, 1), ("rmat_s20", 100, 30, 1),
          ("powerlaw_4m", 20, 100, 1)]


def key_of(name: str, m: int, c: int, seed: int) -> str:
    return f"{name}|m={m}|c={c}|seed={seed}"


def digest(stream, m: int, c: int, seed: int) -> dict:
    e = O.semitriangles(stream.src, stream.dst, stream.n_nodes, m, c, seed)
    local = (e.local1 + e.local2).astype(np.uint64)
    g, _ = O.estimates(m, c, O.Counts(e.tau_proc, e.local1, e.local2), stream.n_nodes)
    return {"input_sha256": stream.sha256(), "n_edges": len(stream), "n_nodes": stream.n_nodes,
            "tau_proc": [str(int(x)) for x in e.tau_proc],
            "local_sha256": hashlib.sha256(local.astype("<u8").tobytes()).hexdigest(),
            "local_sum": str(int(local.sum())), "tau_hat": float(g).hex(), "triangles": int(e.triangles)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None, help="single-stream workload names to (re)compute")
    ap.add_argument("--mix", type=int, default=0, help="also the first N streams of the batched mix (seed 1000)")
    args = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    for name, m, c, seed in SINGLE:
        if args.only is not None and name not in args.only:
            continue
        t = time.time()
        out[key_of(name, m, c, seed)] = digest(gg.cached(name), m, c, seed)
        print(f"{name} m={m} c={c}: {time.time() - t:.1f} s", flush=True)
        _write(out)
    if args.mix:
        from paper_1811_09136_gb300 import batched
        specs = batched.mix_specs(args.mix, seed=1000)
        for sp in specs:
            k = key_of(f"mix1000#{sp.index}", sp.m, sp.m, sp.hash_seed)
            if k in out:
                continue
            t = time.time()
            out[k] = digest(sp.generate(), sp.m, sp.m, sp.hash_seed)
            print(f"mix #{sp.index} ({sp.kind}, n={sp.n_nodes}, E={out[k]['n_edges']}): {time.time() - t:.1f} s",
                  flush=True)
            _write(out)


def _write(out):
    tmp = OUT + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    os.replace(tmp, OUT)


if __name__ == "__main__":
    main()
