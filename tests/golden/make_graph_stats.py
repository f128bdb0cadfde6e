"""Write sweep_graph_stats.txt: tau and eta of the accuracy-sweep graphs, from the oracle's static
enumeration only (eta = sum over edges g of C(a_g, 2), a_g = triangles through g with g not their
last edge; Table I's eta).  Run from the repository root: python tests/golden/make_graph_stats.py"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle as O  # noqa: E402
from paper_1811_09136_gb300 import graphgen as gg  # noqa: E402

GRAPHS = {
    "powerlaw_20k": lambda: gg.cached("powerlaw_20k"),
    "powerlaw_200k": lambda: gg.chung_lu(200_000, 2.1, 2_000_000, graph_seed=42, order_seed=7),
}

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep_graph_stats.txt")
    with open(out, "w") as f:
        f.write("# graph edges tau eta  (oracle static enumeration; written by make_graph_stats.py)\n")
        for name, make in GRAPHS.items():
            s = make()
            e = O.semitriangles(s.src, s.dst, s.n_nodes, 1, 1, 1)
            f.write(f"{name} {len(s)} {e.triangles} {e.eta}\n")
    print(open(out).read())
