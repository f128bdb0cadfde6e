"""Accuracy sweeps: REPT against parallel MASCOT at the same sampling probability.

For a fixed graph and stream order, each method is run over R hash seeds for every processor
count c; the normalised root mean square error of the global estimate,
NRMSE = sqrt(mean((tau_hat - tau)^2)) / tau, is reported per (method, c) — the measure of the
paper's accuracy figures (Section V, global-count NRMSE against c at p = 0.01 and p = 0.1).
tau itself comes from the same kernels with m = c = 1, where every edge is kept and the count is
exact.

Closed forms for the variances, when the graph's eta is supplied:
  REPT, c <= m          (tau (m^2 - c) + 2 eta (m - c)) / c           (Theorem 3)
  REPT, c = c1 m        tau (m - 1) / c1                              (Section III-B.1)
  REPT, c > m, c2 != 0  about 1 / (1/V1 + 1/V2), the inverse-variance combination of the
                        full groups' V1 = tau (m - 1) / c1 and the partial group's
                        V2 = (tau (m^2 - c2) + 2 eta (m - c2)) / c2    (Algorithm 2)
  parallel MASCOT       (tau (m^2 - 1) + 2 eta (m - 1)) / c           (Section III-C)

Run as ``python -m paper_1811_09136_gb300.accuracy --graph powerlaw_20k --m 10 --c 2 4 8 16 32``.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import graphgen, rept


def theory_variance(method: str, tau: float, eta: float, m: int, c: int) -> float:
    """The closed-form variance of the global estimate (see the module docstring)."""
    if method == "mascot":
        return (tau * (m * m - 1) + 2 * eta * (m - 1)) / c
    if c <= m:
        return (tau * (m * m - c) + 2 * eta * (m - c)) / c
    c1, c2 = c // m, c % m
    v1 = tau * (m - 1) / c1
    if c2 == 0:
        return v1
    v2 = (tau * (m * m - c2) + 2 * eta * (m - c2)) / c2
    return 1.0 / (1.0 / v1 + 1.0 / v2)


def spread_seeds(R: int, salt: int = 0) -> list[int]:
    """R hash seeds spread over the 64-bit space (SplitMix64 of a counter).  Seeds that differ only in
    their low bits would make key ^ seed collide across seeds and correlate the runs."""
    out, x = [], (0x5EED0000 + salt) & ((1 << 64) - 1)
    for _ in range(R):
        x = (x + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & ((1 << 64) - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & ((1 << 64) - 1)
        out.append((z ^ (z >> 31)) >> 1)
    return out


def _device_stream(s: graphgen.EdgeStream):
    import torch
    return (torch.from_numpy(s.src.view(np.int32)).cuda(), torch.from_numpy(s.dst.view(np.int32)).cuda())


def exact_triangles(s: graphgen.EdgeStream, src=None, dst=None) -> int:
    """tau from the GPU path with m = c = 1 (every edge kept, tau^(0) = tau)."""
    if src is None:
        src, dst = _device_stream(s)
    with rept.ReptStream(s.n_nodes, 1, 1, 1, expected_edges=len(s), max_batch=len(s)) as h:
        h.ingest(src, dst)
        proc, _ = h.counts()
    return int(proc[0])


def estimates_over_seeds(s: graphgen.EdgeStream, m: int, c: int, seeds, mascot: bool, src=None, dst=None,
                         batch: int = 1 << 20) -> np.ndarray:
    """Global estimates of one method for every hash seed, one handle reset between seeds."""
    if src is None:
        src, dst = _device_stream(s)
    flags = rept.FLAG_MASCOT if mascot else 0
    out = np.empty(len(seeds), dtype=np.float64)
    batch = min(batch, max(1, len(s)))
    with rept.ReptStream(s.n_nodes, m, c, seeds[0], expected_edges=len(s), max_batch=batch, flags=flags) as h:
        for r, seed in enumerate(seeds):
            if r:
                h.reset_async(seed=seed)
            for off in range(0, len(s), batch):
                h.ingest(src[off:off + batch], dst[off:off + batch])
            out[r], _ = h.estimates(local=False)
    return out


def sweep(s: graphgen.EdgeStream, m: int, cs, R: int, eta: float | None = None, salt: int = 0,
          methods=("rept", "mascot"), log=None) -> dict:
    """NRMSE of REPT and parallel MASCOT for every c in ``cs`` over R hash seeds (the same seeds for
    both methods).  With ``eta`` the closed-form NRMSE is reported beside each measured one."""
    src, dst = _device_stream(s)
    tau = exact_triangles(s, src, dst)
    seeds = spread_seeds(R, salt)
    rows = []
    for c in cs:
        for method in methods:
            t0 = time.perf_counter()
            est = estimates_over_seeds(s, m, c, seeds, method == "mascot", src, dst)
            secs = time.perf_counter() - t0
            err = est - tau
            row = {"method": method, "m": m, "p": 1.0 / m, "c": c, "R": R,
                   "nrmse": float(math.sqrt(np.mean(err * err)) / tau) if tau else float("nan"),
                   "bias": float(np.mean(err) / tau) if tau else float("nan"),
                   "seconds": secs}
            if eta is not None and tau:
                row["nrmse_theory"] = math.sqrt(theory_variance(method, tau, eta, m, c)) / tau
            rows.append(row)
            if log:
                log(row)
    return {"edges": len(s), "n_nodes": s.n_nodes, "tau": tau, "eta": eta, "rows": rows}


def markdown(result: dict) -> str:
    """The sweep as a table: one row per c, REPT and MASCOT side by side."""
    by = {}
    for r in result["rows"]:
        by.setdefault(r["c"], {})[r["method"]] = r
    theory = result["eta"] is not None
    head = "| c | REPT NRMSE | MASCOT NRMSE | MASCOT / REPT |" + (" REPT theory | MASCOT theory |" if theory else "")
    lines = [head, "|" + "---|" * (6 if theory else 4)]
    for c in sorted(by):
        a, b = by[c].get("rept"), by[c].get("mascot")
        cells = [str(c), f"{a['nrmse']:.4f}" if a else "", f"{b['nrmse']:.4f}" if b else "",
                 f"{b['nrmse'] / a['nrmse']:.2f}" if a and b and a["nrmse"] > 0 else ""]
        if theory:
            cells += [f"{a['nrmse_theory']:.4f}" if a else "", f"{b['nrmse_theory']:.4f}" if b else ""]
        lines.append("| " + " | ".join(cells) + " |")
    return "\n".join(lines)


def _graph(name: str) -> graphgen.EdgeStream:
    if name == "powerlaw_200k":
        # Chung-Lu, 200,000 nodes, exponent 2.1, 2,000,000 distinct edges: the p = 0.01 sweep graph
        return graphgen.chung_lu(200_000, 2.1, 2_000_000, graph_seed=42, order_seed=7)
    return graphgen.cached(name)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--graph", default="powerlaw_20k", help="powerlaw_20k, powerlaw_200k, rmat_s20, powerlaw_4m")
    ap.add_argument("--m", type=int, default=10, help="1/p")
    ap.add_argument("--c", type=int, nargs="+", default=[2, 4, 8, 16, 32])
    ap.add_argument("--runs", type=int, default=100, help="hash seeds per (method, c)")
    ap.add_argument("--eta", type=float, default=None, help="the graph's eta, for the closed-form columns")
    ap.add_argument("--json", default=None, help="also write the result here")
    a = ap.parse_args(argv)
    rept.load()
    res = sweep(_graph(a.graph), a.m, a.c, a.runs, a.eta, log=lambda r: print(json.dumps(r), flush=True))
    res["graph"] = a.graph
    print(markdown(res))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
