"""Pins for the CPU oracle: facts fixed by the paper or by mathematics, not by the oracle itself.

Each ``pin_*`` function raises AssertionError when the oracle library ``lib``
disagrees with something the paper or mathematics fixes.  ``test_oracle.py``
runs them on the real oracle; ``test_oracle_mutants.py`` runs them on copies
of the oracle with a planted mistake and expects at least one to fail.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

import oracle as O
from paper_1811_09136_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def read_golden_hex(name: str) -> list[int]:
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(int(line, 16))
    return out


# --------------------------------------------------------------------------
# independent brute force of the semi-triangle definition (Section III: a
# triangle is a semi-triangle of processor i when its first two edges on the
# stream are both stored by i; processor i = k*m + j keeps group-k colour j)
# --------------------------------------------------------------------------
def _py_splitmix64(x: int) -> int:
    z = (x + GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def py_colour(u: int, v: int, seed: int, k: int, m: int) -> int:
    lo, hi = min(u, v), max(u, v)
    return _py_splitmix64(((lo << 32) | hi) ^ ((seed + k * GAMMA) & MASK64)) % m


def brute_force(src, dst, n, m, c, seed, mascot=False):
    """tau^(i) and tau_v^(i) by checking every node triple (n must be small).  With ``mascot``,
    sampler i keeps the edges of hash group i with colour 0 (parallel MASCOT, Section III-C)."""
    when = {}
    for t, (a, b) in enumerate(zip(src.tolist(), dst.tolist())):
        if a != b:
            when[(min(a, b), max(a, b))] = t
    tau = np.zeros(c, dtype=np.uint64)
    loc = np.zeros((c, n), dtype=np.uint64)
    groups = c if mascot else (c + m - 1) // m
    for a, b, d in itertools.combinations(range(n), 3):
        es = [(a, b), (a, d), (b, d)]
        if not all(e in when for e in es):
            continue
        first_two = sorted(es, key=lambda e: when[e])[:2]
        for k in range(groups):
            j1 = py_colour(*first_two[0], seed, k, m)
            j2 = py_colour(*first_two[1], seed, k, m)
            i = k if mascot else k * m + j1
            if j1 == j2 and i < c and (j1 == 0 or not mascot):
                tau[i] += 1
                for x in (a, b, d):
                    loc[i, x] += 1
    return tau, loc


SMALL_CASES = [(2, 1), (2, 2), (3, 2), (4, 4), (5, 3), (2, 4), (3, 6), (3, 7), (4, 9), (1, 1), (1, 3)]


# --------------------------------------------------------------------------
# pins
# --------------------------------------------------------------------------
def pin_splitmix64_published(lib=None):
    """Outputs 1..5 of SplitMix64 from state 0, as published."""
    want = read_golden_hex("splitmix64_state0.txt")
    got = [O.splitmix64((k * GAMMA) & MASK64, lib=lib) for k in range(len(want))]
    assert got == want, (got, want)


def pin_colour_uniform(lib=None):
    """Section III-A asks h to be uniform on {1..m}: chi-square over 40,000 keys, m = 10 and 7,
    plus agreement of two groups' colours at the rate 1/m that independence gives."""
    rng = np.random.default_rng(123)
    us = rng.integers(0, 1 << 31, size=40_000)
    vs = rng.integers(0, 1 << 31, size=40_000)
    for m in (10, 7):
        cols = np.array([O.colour(int(u), int(v), 1, 0, m, lib=lib) for u, v in zip(us[:20_000], vs[:20_000])])
        counts = np.bincount(cols, minlength=m)
        exp = cols.size / m
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        assert chi2 < 40.0, (m, chi2)          # df <= 9: p ~ 5e-6
    m = 4
    same = sum(O.colour(int(u), int(v), 9, 0, m, lib=lib) == O.colour(int(u), int(v), 9, 1, m, lib=lib)
               for u, v in zip(us[:8000], vs[:8000]))
    assert abs(same / 8000 - 1 / m) < 0.03, same


def pin_brute_force(lib=None):
    """Streaming oracle and static enumeration equal the brute-force definition, per processor and node."""
    for gi, (n, q) in enumerate([(9, 0.7), (14, 0.5), (22, 0.35)]):
        s = gg.gnp(n, q, graph_seed=11 + gi, order_seed=5 + gi)
        for (m, c) in SMALL_CASES:
            for seed in (1, 77):
                tau, loc = brute_force(s.src, s.dst, n, m, c, seed)
                a = O.rept_stream(s.src, s.dst, n, m, c, seed, per_proc_local=True, lib=lib)
                b = O.semitriangles(s.src, s.dst, n, m, c, seed, per_proc_local=True, lib=lib)
                assert np.array_equal(a.tau_proc, tau), (n, m, c, seed, a.tau_proc, tau)
                assert np.array_equal(a.tau_local_proc, loc), (n, m, c, seed)
                assert np.array_equal(b.tau_proc, tau), (n, m, c, seed)
                assert np.array_equal(b.tau_local_proc, loc), (n, m, c, seed)


def pin_complete_graph(lib=None):
    """m = 1 keeps every edge in one processor, so it counts every triangle:
    K_n has C(n,3) triangles and C(n-1,2) through each node."""
    for n in (3, 4, 5, 11, 30):
        s = gg.complete(n, order_seed=n)
        a = O.rept_stream(s.src, s.dst, n, 1, 1, 1, lib=lib)
        assert int(a.tau_proc[0]) == math.comb(n, 3)
        assert np.all(a.local1 == math.comb(n - 1, 2))
        g, loc = O.estimates(1, 1, a, n, lib=lib)
        assert g == float(math.comb(n, 3))
        e = O.semitriangles(s.src, s.dst, n, 1, 1, 1, lib=lib)
        assert e.triangles == math.comb(n, 3) and int(e.tau_proc[0]) == math.comb(n, 3)


def pin_local_sum_invariant(lib=None):
    """Each closed wedge adds |N_uv| to tau^(i) and 3|N_uv| to the local counts (Algorithm 1):
    sum_v tau_v^(i) = 3 tau^(i) for every processor."""
    s = gg.chung_lu(3000, 2.2, 20_000, graph_seed=3, order_seed=4)
    for (m, c) in [(5, 5), (6, 4), (3, 7), (2, 6)]:
        a = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 9, per_proc_local=True, lib=lib)
        assert np.array_equal(a.tau_local_proc.sum(axis=1), 3 * a.tau_proc), (m, c)
        assert int(a.local1.sum() + a.local2.sum()) == 3 * int(a.tau_proc.sum())


def pin_count_before_insert(lib=None):
    """Algorithm 1 counts with the sets as they stand and inserts afterwards: the arriving edge's
    own colour never matters, and a triangle is counted only when its last edge arrives."""
    # triangle 0-1-2: edges (0,1), (1,2) then (0,2); with m = 1 exactly one semi-triangle
    src = np.array([0, 1, 0], dtype=np.uint32)
    dst = np.array([1, 2, 2], dtype=np.uint32)
    for T, want in ((2, 0), (3, 1)):
        a = O.rept_stream(src[:T], dst[:T], 3, 1, 1, 1, lib=lib)
        assert int(a.tau_proc[0]) == want
    # search seeds where the first two edges share colour j but the last has another: counted;
    # and where the first two differ but the last matches one of them: not counted.
    m = 3
    found_a = found_b = False
    for seed in range(1, 400):
        c01, c12, c02 = (py_colour(0, 1, seed, 0, m), py_colour(1, 2, seed, 0, m), py_colour(0, 2, seed, 0, m))
        a = O.rept_stream(src, dst, 3, m, m, seed, lib=lib)
        if c01 == c12 != c02:
            found_a = True
            assert int(a.tau_proc[c01]) == 1 and int(a.tau_proc.sum()) == 1, seed
        if c01 != c12 and c02 in (c01, c12):
            found_b = True
            assert int(a.tau_proc.sum()) == 0, seed
    assert found_a and found_b


def pin_self_loops(lib=None):
    """Self-loops are skipped: same counts as without them, and counted as skipped."""
    s = gg.gnp(25, 0.4, 2, 3)
    src = np.concatenate([s.src, np.array([4, 7, 7], dtype=np.uint32)])
    dst = np.concatenate([s.dst, np.array([4, 7, 7], dtype=np.uint32)])
    perm = np.random.default_rng(0).permutation(src.size)
    # place the loops in the middle of the stream without disturbing the edges' relative order
    keep = np.sort(perm[: s.src.size])
    order = np.full(src.size, -1)
    order[keep] = np.arange(s.src.size)
    loops = [i for i in range(src.size) if order[i] < 0]
    for li, pos in enumerate(loops):
        order[pos] = s.src.size + li
    src2, dst2 = src[order], dst[order]
    a = O.rept_stream(s.src, s.dst, 25, 3, 3, 5, lib=lib)
    b = O.rept_stream(src2, dst2, 25, 3, 3, 5, lib=lib)
    assert np.array_equal(a.tau_proc, b.tau_proc) and np.array_equal(a.local1, b.local1)
    assert b.skipped == 3


def pin_networkx_triangles(lib=None):
    """m = 1: the single processor's counts equal the graph's triangle counts (networkx)."""
    import pytest
    nx = pytest.importorskip("networkx")
    s = gg.chung_lu(2000, 2.3, 12_000, graph_seed=8, order_seed=9)
    G = nx.Graph()
    G.add_nodes_from(range(s.n_nodes))
    G.add_edges_from(zip(s.src.tolist(), s.dst.tolist()))
    tri = nx.triangles(G)
    a = O.rept_stream(s.src, s.dst, s.n_nodes, 1, 1, 3, lib=lib)
    assert int(a.tau_proc[0]) == sum(tri.values()) // 3
    assert all(int(a.local1[v]) == tri[v] for v in range(s.n_nodes))


def pin_eta_exact_at_m1(lib=None):
    """With m = 1 one processor stores every edge, so eta^(0) must be the exact eta of Table I
    (pairs of triangles sharing an edge that is last in neither), computed independently here."""
    s = gg.gnp(18, 0.5, 21, 22)
    when = {(min(a, b), max(a, b)): t for t, (a, b) in enumerate(zip(s.src.tolist(), s.dst.tolist()))}
    tris = [t for t in itertools.combinations(range(18), 3)
            if all((min(x, y), max(x, y)) in when for x, y in itertools.combinations(t, 2))]
    def non_last(t):
        es = sorted(((min(x, y), max(x, y)) for x, y in itertools.combinations(t, 2)), key=lambda e: when[e])
        return set(es[:2])
    eta, eta_v = 0, np.zeros(18, dtype=np.int64)
    for t1, t2 in itertools.combinations(tris, 2):
        shared = set(itertools.combinations(sorted(set(t1) & set(t2)), 2))
        if len(shared) == 1:
            g = shared.pop()
            if g in non_last(t1) and g in non_last(t2):
                eta += 1
                for v in set(t1) & set(t2):
                    eta_v[v] += 1
    a = O.rept_stream(s.src, s.dst, 18, 1, 1, 4, lib=lib)
    assert int(a.eta_proc[0]) == eta, (int(a.eta_proc[0]), eta)
    assert np.array_equal(a.eta_local.astype(np.int64), eta_v)
    e = O.semitriangles(s.src, s.dst, 18, 1, 1, 4, lib=lib)
    assert e.eta == eta and np.array_equal(e.eta_local.astype(np.int64), eta_v)


def pin_batch_split_and_static(lib=None):
    """The static enumeration of the definition equals the streaming run on a 20,000-node
    power-law stream for several (m, c), including both c > m cases."""
    s = gg.powerlaw_20k()
    for (m, c) in [(10, 10), (10, 3), (4, 8), (4, 9)]:
        a = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, 1, pair_counters=False, lib=lib)
        b = O.semitriangles(s.src, s.dst, s.n_nodes, m, c, 1, lib=lib)
        assert np.array_equal(a.tau_proc, b.tau_proc), (m, c)
        assert np.array_equal(a.local1, b.local1) and np.array_equal(a.local2, b.local2), (m, c)


def _spread_seeds(R, salt):
    """R hash seeds spread over the 64-bit space.  Seeds that differ only in low bits make
    key ^ seed collide across seeds and edges (key1 ^ s1 == key2 ^ s2), which correlates the
    runs; independent draws stand in for independently chosen hash functions."""
    rng = np.random.default_rng(10_000 + salt)
    return [int(x) for x in rng.integers(0, 1 << 63, size=R, dtype=np.int64)]


def _stat_run(s, m, c, seeds, node, lib):
    g_est, l_est = [], []
    for seed in seeds:
        a = O.rept_stream(s.src, s.dst, s.n_nodes, m, c, seed, lib=lib)
        g, loc = O.estimates(m, c, a, s.n_nodes, lib=lib)
        g_est.append(g)
        l_est.append(loc[node])
    return np.array(g_est), np.array(l_est)


def pin_theorem3_statistics(lib=None):
    """Theorem 3 (and its c = m and c mod m = 0 cases): over 400 hash seeds the estimates are
    unbiased and their variance is (tau(m^2-c) + 2 eta(m-c)) / c, resp. tau(m-1)/c1.
    Bands: mean within 4.5 standard errors; variance ratio within [0.7, 1.45]."""
    s = gg.gnp(30, 0.5, 31, 32)
    e = O.semitriangles(s.src, s.dst, 30, 1, 1, 1, lib=lib)
    tau, eta = e.triangles, e.eta
    node = int(np.argmax(e.tri_local))
    tau_v, eta_v = int(e.tri_local[node]), int(e.eta_local[node])
    seeds = _spread_seeds(400, 1)
    for (m, c) in [(2, 1), (4, 2), (3, 3), (3, 6)]:
        if c <= m:
            var = (tau * (m * m - c) + 2 * eta * (m - c)) / c
            var_v = (tau_v * (m * m - c) + 2 * eta_v * (m - c)) / c
        else:
            c1 = c // m
            var, var_v = tau * (m - 1) / c1, tau_v * (m - 1) / c1
        g, l = _stat_run(s, m, c, seeds, node, lib)
        R = len(seeds)
        assert abs(g.mean() - tau) < 4.5 * math.sqrt(var / R), (m, c, g.mean(), tau, var)
        assert 0.7 < g.var(ddof=1) / var < 1.45, (m, c, g.var(ddof=1), var)
        assert abs(l.mean() - tau_v) < 4.5 * math.sqrt(var_v / R), (m, c, l.mean(), tau_v)
        assert 0.7 < l.var(ddof=1) / var_v < 1.45, (m, c, l.var(ddof=1), var_v)


def pin_partial_group_statistics(lib=None):
    """c > m with c mod m != 0 (Algorithm 2): both group estimates are unbiased, and the
    inverse-variance combination stays within 4.5 standard errors of tau with a variance no
    larger than the full groups' tau(m-1)/c1 (it adds an independent estimate)."""
    s = gg.gnp(30, 0.5, 31, 32)
    e = O.semitriangles(s.src, s.dst, 30, 1, 1, 1, lib=lib)
    tau, eta = e.triangles, e.eta
    m, c = 3, 7
    c1, c2 = c // m, c % m
    ests, t1s, t2s, eta_hats = [], [], [], []
    for seed in _spread_seeds(400, 2):
        a = O.rept_stream(s.src, s.dst, 30, m, c, seed, lib=lib)
        g, _ = O.estimates(m, c, a, 30, lib=lib)
        ests.append(g)
        t1s.append(float(a.tau_proc[: c1 * m].sum()) * m / c1)
        t2s.append(float(a.tau_proc[c1 * m:].sum()) * m * m / c2)
        eta_hats.append(float(a.eta_proc.sum()) * m ** 3 / c)
    ests, t1s, t2s, eta_hats = map(np.array, (ests, t1s, t2s, eta_hats))
    var1 = tau * (m - 1) / c1
    var2 = (tau * (m * m - c2) + 2 * eta * (m - c2)) / c2
    R = ests.size
    assert abs(t1s.mean() - tau) < 4.5 * math.sqrt(var1 / R)
    assert abs(t2s.mean() - tau) < 4.5 * math.sqrt(var2 / R)
    assert abs(ests.mean() - tau) < 4.5 * math.sqrt(var1 / R)
    assert ests.var(ddof=1) < 1.2 * var1
    # eta_hat = sum_i m^3 eta^(i) / c is unbiased for eta (Section III-B.2)
    assert abs(eta_hats.mean() - eta) < 4.5 * eta_hats.std(ddof=1) / math.sqrt(R) + 1e-9


def pin_partial_group_local_statistics(lib=None):
    """c > m with c mod m != 0 (Algorithm 2), per node: over 400 spread hash seeds, on the three
    nodes with the most triangles,
      - the full groups' local estimate (m / c1) * local1[v] and the partial group's
        (m^2 / c2) * local2[v] are unbiased for tau_v (Section III-B.2),
      - the combined local estimate is unbiased and its variance is at most 1.2 * tau_v (m-1) / c1
        (the full groups' variance; the combination only adds an independent estimate), and
      - the eta_v estimate that the combination used is unbiased for the exact eta_v.
    The last one is read back from the combination itself: with a1, a2 the two group estimates and
    est their combination (w2 a1 + w1 a2) / (w1 + w2), the weight ratio is r = w1 / w2 =
    (a1 - est) / (est - a2); w1 = a1 (m-1) / c1 gives w2 = w1 / r, and Section III-B.2's
    w2 = (a1 (m^2 - c2) + 2 eta_hat_v (m - c2)) / c2 gives eta_hat_v.  Seeds where a1 = 0 or the
    two estimates coincide carry no information and are skipped."""
    s = gg.gnp(30, 0.5, 31, 32)
    e = O.semitriangles(s.src, s.dst, 30, 1, 1, 1, lib=lib)
    nodes = [int(x) for x in np.argsort(-e.tri_local.astype(np.int64), kind="stable")[:3]]
    for (m, c) in [(3, 7), (4, 9)]:
        c1, c2 = c // m, c % m
        a1s, a2s, ests, eta_hats = [], [], [], []
        for seed in _spread_seeds(400, 4):
            a = O.rept_stream(s.src, s.dst, 30, m, c, seed, lib=lib)
            _, loc = O.estimates(m, c, a, 30, lib=lib)
            a1 = a.local1[nodes].astype(np.float64) * m / c1
            a2 = a.local2[nodes].astype(np.float64) * m * m / c2
            a1s.append(a1)
            a2s.append(a2)
            ests.append(loc[nodes])
            row = np.full(len(nodes), np.nan)
            for j in range(len(nodes)):
                if a1[j] > 0 and abs(a1[j] - a2[j]) > 1e-9 * a1[j] and abs(loc[nodes[j]] - a2[j]) > 1e-9 * a1[j]:
                    r = (a1[j] - loc[nodes[j]]) / (loc[nodes[j]] - a2[j])
                    w2 = a1[j] * (m - 1) / c1 / r
                    row[j] = (w2 * c2 - a1[j] * (m * m - c2)) / (2 * (m - c2))
            eta_hats.append(row)
        a1s, a2s, ests, eta_hats = map(np.array, (a1s, a2s, ests, eta_hats))
        R = a1s.shape[0]
        for j, v in enumerate(nodes):
            tv, ev = int(e.tri_local[v]), int(e.eta_local[v])
            var1 = tv * (m - 1) / c1
            var2 = (tv * (m * m - c2) + 2 * ev * (m - c2)) / c2
            assert abs(a1s[:, j].mean() - tv) < 4.5 * math.sqrt(var1 / R), (m, c, v, a1s[:, j].mean(), tv)
            assert abs(a2s[:, j].mean() - tv) < 4.5 * math.sqrt(var2 / R), (m, c, v, a2s[:, j].mean(), tv)
            assert abs(ests[:, j].mean() - tv) < 4.5 * math.sqrt(var1 / R), (m, c, v, ests[:, j].mean(), tv)
            assert ests[:, j].var(ddof=1) < 1.2 * var1, (m, c, v, ests[:, j].var(ddof=1), var1)
            eh = eta_hats[:, j][~np.isnan(eta_hats[:, j])]
            assert eh.size > R // 2, (m, c, v, eh.size)
            assert abs(eh.mean() - ev) < 4.5 * eh.std(ddof=1) / math.sqrt(eh.size) + 1e-9, (m, c, v, eh.mean(), ev)


def pin_mascot_brute_force(lib=None):
    """Parallel MASCOT (Section III-C): sampler i stores an edge iff hash group i colours it 0, and
    counts a triangle iff its two earliest edges are both stored.  The streaming and static oracles
    equal the brute force of that definition, per sampler and node."""
    for gi, (n, q) in enumerate([(10, 0.7), (18, 0.45)]):
        s = gg.gnp(n, q, graph_seed=21 + gi, order_seed=8 + gi)
        for (m, c) in [(1, 2), (2, 1), (2, 3), (3, 5), (4, 2)]:
            for seed in (3, 1234567):
                tau, loc = brute_force(s.src, s.dst, n, m, c, seed, mascot=True)
                a = O.mascot_stream(s.src, s.dst, n, m, c, seed, per_proc_local=True, lib=lib)
                t2, l2, tl2 = O.mascot_semitriangles(s.src, s.dst, n, m, c, seed, per_proc_local=True, lib=lib)
                assert np.array_equal(a.tau_proc, tau), (n, m, c, seed, a.tau_proc, tau)
                assert np.array_equal(a.tau_local_proc, loc), (n, m, c, seed)
                assert np.array_equal(a.local1, loc.sum(axis=0)), (n, m, c, seed)
                assert np.array_equal(t2, tau) and np.array_equal(tl2, loc), (n, m, c, seed)


def pin_mascot_complete_graph(lib=None):
    """m = 1 (p = 1): every sampler keeps every edge, so each counts all C(n,3) triangles of K_n and
    the averaged estimate is exact."""
    for n in (4, 9, 20):
        s = gg.complete(n, order_seed=n + 1)
        a = O.mascot_stream(s.src, s.dst, n, 1, 3, 5, lib=lib)
        assert np.all(a.tau_proc == math.comb(n, 3))
        assert np.all(a.local1 == 3 * math.comb(n - 1, 2))
        g, loc = O.mascot_estimates(1, 3, a, n, lib=lib)
        assert g == float(math.comb(n, 3)) and np.all(loc == float(math.comb(n - 1, 2)))


def pin_mascot_statistics(lib=None):
    """Section III-C: averaging c independent MASCOT samplers with p = 1/m is unbiased with variance
    (tau(m^2-1) + 2 eta(m-1)) / c, which exceeds REPT's (tau(m^2-c) + 2 eta(m-c)) / c for
    1 < c <= m.  400 spread hash seeds; same bands as the Theorem 3 pin."""
    s = gg.gnp(30, 0.5, 31, 32)
    e = O.semitriangles(s.src, s.dst, 30, 1, 1, 1, lib=lib)
    tau, eta = e.triangles, e.eta
    node = int(np.argmax(e.tri_local))
    tau_v, eta_v = int(e.tri_local[node]), int(e.eta_local[node])
    seeds = _spread_seeds(400, 3)
    R = len(seeds)
    for (m, c) in [(2, 1), (3, 3), (2, 4)]:
        var = (tau * (m * m - 1) + 2 * eta * (m - 1)) / c
        var_v = (tau_v * (m * m - 1) + 2 * eta_v * (m - 1)) / c
        g, l = [], []
        for seed in seeds:
            a = O.mascot_stream(s.src, s.dst, 30, m, c, seed, lib=lib)
            gg_, loc = O.mascot_estimates(m, c, a, 30, lib=lib)
            g.append(gg_)
            l.append(loc[node])
        g, l = np.array(g), np.array(l)
        assert abs(g.mean() - tau) < 4.5 * math.sqrt(var / R), (m, c, g.mean(), tau, var)
        assert 0.7 < g.var(ddof=1) / var < 1.45, (m, c, g.var(ddof=1), var)
        assert abs(l.mean() - tau_v) < 4.5 * math.sqrt(var_v / R), (m, c, l.mean(), tau_v)
        assert 0.7 < l.var(ddof=1) / var_v < 1.45, (m, c, l.var(ddof=1), var_v)
        if 1 < c <= m:
            assert var > (tau * (m * m - c) + 2 * eta * (m - c)) / c


ALL_PINS = [pin_splitmix64_published, pin_colour_uniform, pin_brute_force, pin_complete_graph,
            pin_local_sum_invariant, pin_count_before_insert, pin_self_loops, pin_networkx_triangles,
            pin_eta_exact_at_m1, pin_batch_split_and_static, pin_theorem3_statistics,
            pin_partial_group_statistics, pin_partial_group_local_statistics, pin_mascot_brute_force, pin_mascot_complete_graph,
            pin_mascot_statistics]
