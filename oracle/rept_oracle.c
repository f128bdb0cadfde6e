/*
 * REPT oracle: a plain, slow, sequential CPU statement of what the method
 * computes (Wang et al., "REPT: A Streaming Algorithm of Approximating Global
 * and Local Triangle Counts in Parallel").
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg use it.  It shares no code with the CUDA path: the
 * hash, the per-processor sets, the counters and the estimators are all
 * written here again from the paper.
 *
 * Contents
 *   orc_splitmix64 / orc_colour    the edge-partition hash h_k (Section III-A,
 *                                  III-B; the concrete function is SplitMix64
 *                                  of the ordered endpoint pair xor a
 *                                  per-group seed, mod m)
 *   orc_rept_stream                Algorithm 1 run per processor, with the
 *                                  grouping of Section III-B for c > m and the
 *                                  triangle-pair counters of Algorithm 2
 *   orc_estimates                  the estimators of Section III-A (c <= m),
 *                                  III-B.1 (c > m, c mod m = 0) and Algorithm 2
 *                                  (c > m, c mod m != 0)
 *   orc_mascot_stream,             parallel MASCOT (Section I, III-C): c
 *   orc_mascot_estimates,          independent p = 1/m samplers, sampler i
 *   orc_mascot_semitriangles       keeping h_i colour 0, estimates averaged
 *   orc_rept_stream_parallel       the same counts the paper's multi-core way:
 *                                  one thread per processor (a timing baseline)
 *   orc_semitriangles              the definition of a semi-triangle written
 *                                  out as a static triangle enumeration: a
 *                                  triangle counts for processor i iff its two
 *                                  earliest edges on the stream both belong to
 *                                  E^(i) (Section III, definition of Delta^(i))
 *
 * Processors are 0-based: processor i belongs to group k = i / m and keeps
 * the edges whose group-k colour equals j = i % m (Algorithm 2's index split,
 * read 0-based).  Group k uses seed s_k = seed + k * 0x9E3779B97F4A7C15
 * (mod 2^64).  Self-loops are skipped (not stored, not counted).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ hash */

/* One output step of SplitMix64 (Steele, Lea, Flood 2014) taken from state x. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* h_k(u, v): colour in {0..m-1} of the undirected edge {u, v} in hash group k. */
uint32_t orc_colour(uint32_t u, uint32_t v, uint64_t seed, uint32_t k, uint32_t m) {
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    uint64_t key = (lo << 32) | hi;
    uint64_t s_k = seed + (uint64_t)k * 0x9E3779B97F4A7C15ULL;
    return (uint32_t)(orc_splitmix64(key ^ s_k) % (uint64_t)m);
}

/* ------------------------------------------------- small containers (plain) */

typedef struct { uint32_t* a; uint32_t n, cap; } vec32;

static int vec_push(vec32* v, uint32_t x) {
    if (v->n == v->cap) {
        uint32_t nc = v->cap ? 2 * v->cap : 4;
        uint32_t* na = (uint32_t*)realloc(v->a, (size_t)nc * sizeof(uint32_t));
        if (!na) return -1;
        v->a = na; v->cap = nc;
    }
    v->a[v->n++] = x;
    return 0;
}

/* open-addressing map uint64 key -> uint64 value; key ~0 is reserved */
typedef struct { uint64_t* key; uint64_t* val; uint64_t mask, n; } umap;
#define UM_EMPTY 0xFFFFFFFFFFFFFFFFULL

static uint64_t um_mix(uint64_t k) {   /* Murmur3 64-bit finaliser: slot choice only */
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33; return k;
}

static int um_init(umap* m, uint64_t cap) {
    uint64_t c = 16;
    while (c < cap) c <<= 1;
    m->key = (uint64_t*)malloc(c * sizeof(uint64_t));
    m->val = (uint64_t*)malloc(c * sizeof(uint64_t));
    if (!m->key || !m->val) return -1;
    memset(m->key, 0xFF, c * sizeof(uint64_t));
    m->mask = c - 1; m->n = 0;
    return 0;
}

static void um_free(umap* m) { free(m->key); free(m->val); m->key = m->val = NULL; }

static uint64_t* um_find(const umap* m, uint64_t k) {
    uint64_t h = um_mix(k) & m->mask;
    while (m->key[h] != UM_EMPTY) {
        if (m->key[h] == k) return &m->val[h];
        h = (h + 1) & m->mask;
    }
    return NULL;
}

static int um_grow(umap* m);

/* returns pointer to the value for k, inserting (k, init) if absent */
static uint64_t* um_get(umap* m, uint64_t k, uint64_t init) {
    if (2 * (m->n + 1) > m->mask + 1 && um_grow(m)) return NULL;
    uint64_t h = um_mix(k) & m->mask;
    while (m->key[h] != UM_EMPTY) {
        if (m->key[h] == k) return &m->val[h];
        h = (h + 1) & m->mask;
    }
    m->key[h] = k; m->val[h] = init; m->n++;
    return &m->val[h];
}

static int um_grow(umap* m) {
    umap g;
    if (um_init(&g, 2 * (m->mask + 1))) return -1;
    for (uint64_t i = 0; i <= m->mask; ++i)
        if (m->key[i] != UM_EMPTY) *um_get(&g, m->key[i], m->val[i]) = m->val[i];
    um_free(m);
    *m = g;
    return 0;
}

static uint64_t edge_key(uint32_t u, uint32_t v) {
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    return (lo << 32) | hi;
}

/* ------------------------------------------------------ streaming oracle */

/*
 * Sequential REPT.  For every edge (u, v) of the stream and every processor
 * i: first UpdateTriangleCNT / UpdateTrianglePairCNT(i, (u, v)) on the sets
 * as they stand, then insert (u, v) into E^(i) iff h_k(u, v) == j
 * (Algorithm 1; Algorithm 2 for the pair counters).
 *
 * Outputs (all caller-allocated, zero-filled here):
 *   tau_proc[c]         tau^(i)
 *   eta_proc[c]         eta^(i)                                (may be NULL)
 *   local1[n]           sum of tau_v^(i) over processors i < c1*m, or over all
 *                       processors when c <= m                (may be NULL)
 *   local2[n]           sum of tau_v^(i) over the last, partial group when
 *                       c > m and c mod m != 0                (may be NULL)
 *   eta_local[n]        sum over all processors of eta_v^(i)  (may be NULL)
 *   tau_local_proc[c*n] tau_v^(i), processor-major           (may be NULL)
 *   skipped             self-loops seen                       (may be NULL)
 * Returns 0, or -1 on bad arguments / out of memory, -2 on an id >= n.
 */
/* The processor-to-sampler map: REPT's processor i = k*m + j keeps group-k
 * colour j; a parallel-MASCOT sampler i (Section III-C) keeps the edges whose
 * own hash h_i colours them 0, i.e. an independent p = 1/m sample. */
static void proc_map(int mascot, uint32_t i, uint32_t m, uint32_t* k, uint32_t* j) {
    *k = mascot ? i : i / m;
    *j = mascot ? 0 : i % m;
}

static int sample_stream(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                         uint32_t m, uint32_t c, uint64_t seed, int mascot, uint32_t i_lo, uint32_t i_hi,
                         uint64_t* tau_proc, uint64_t* eta_proc,
                         uint64_t* local1, uint64_t* local2, uint64_t* eta_local,
                         uint64_t* tau_local_proc, uint64_t* skipped) {
    if (m == 0 || c == 0 || n == 0 || !tau_proc) return -1;
    uint32_t c1 = c / m;                 /* number of full groups (0 when c < m) */
    uint32_t full = (mascot || c <= m) ? c : c1 * m;   /* processors feeding local1 */
    memset(tau_proc, 0, c * sizeof(uint64_t));
    if (eta_proc) memset(eta_proc, 0, c * sizeof(uint64_t));
    if (local1) memset(local1, 0, (size_t)n * sizeof(uint64_t));
    if (local2) memset(local2, 0, (size_t)n * sizeof(uint64_t));
    if (eta_local) memset(eta_local, 0, (size_t)n * sizeof(uint64_t));
    if (tau_local_proc) memset(tau_local_proc, 0, (size_t)c * n * sizeof(uint64_t));
    if (skipped) *skipped = 0;

    /* Per processor: N_x^(i) as a growable array, found through a map keyed
     * by (i, x); E^(i) as a map from edge key to the triangle counter
     * tau_(u,v)^(i) of Algorithm 2. */
    umap adj_index;                      /* (i << 32 | x) -> index into lists */
    umap* edges = (umap*)calloc(c, sizeof(umap));
    vec32* lists = NULL;
    uint64_t n_lists = 0, cap_lists = 0;
    vec32 common = {0, 0, 0};
    int rc = 0;
    if (!edges || um_init(&adj_index, 1024)) { free(edges); return -1; }
    for (uint32_t i = i_lo; i < i_hi; ++i)
        if (um_init(&edges[i], 64)) { rc = -1; goto done; }

    for (uint64_t t = 0; t < T; ++t) {
        uint32_t u = src[t], v = dst[t];
        if (u >= n || v >= n) { rc = -2; goto done; }
        if (u == v) { if (skipped) ++*skipped; continue; }
        for (uint32_t i = i_lo; i < i_hi; ++i) {
            uint32_t k, j;
            proc_map(mascot, i, m, &k, &j);
            /* ---- UpdateTriangleCNT(i, (u, v)): N_{u,v}^(i) = N_u^(i) cap N_v^(i) */
            uint64_t* pu = um_find(&adj_index, ((uint64_t)i << 32) | u);
            uint64_t* pv = um_find(&adj_index, ((uint64_t)i << 32) | v);
            common.n = 0;
            if (pu && pv) {
                vec32* a = &lists[*pu];
                vec32* b = &lists[*pv];
                uint32_t other = v;                  /* probe the larger set */
                if (a->n > b->n) { vec32* t2 = a; a = b; b = t2; other = u; }
                for (uint32_t q = 0; q < a->n; ++q) {
                    uint32_t w = a->a[q];
                    if (um_find(&edges[i], edge_key(other, w)))
                        if (vec_push(&common, w)) { rc = -1; goto done; }
                }
            }
            uint64_t nuv = common.n;
            tau_proc[i] += nuv;
            uint64_t* l_sum = (i < full) ? local1 : local2;
            if (l_sum) { l_sum[u] += nuv; l_sum[v] += nuv; }
            if (tau_local_proc) {
                tau_local_proc[(uint64_t)i * n + u] += nuv;
                tau_local_proc[(uint64_t)i * n + v] += nuv;
            }
            for (uint64_t q = 0; q < nuv; ++q) {
                uint32_t w = common.a[q];
                if (l_sum) l_sum[w] += 1;
                if (tau_local_proc) tau_local_proc[(uint64_t)i * n + w] += 1;
                /* Algorithm 2: triangle-pair counters */
                uint64_t* tuw = um_find(&edges[i], edge_key(u, w));
                uint64_t* tvw = um_find(&edges[i], edge_key(v, w));
                if (eta_proc) eta_proc[i] += *tuw + *tvw;
                if (eta_local) {
                    eta_local[w] += *tuw + *tvw;
                    eta_local[u] += *tuw;
                    eta_local[v] += *tvw;
                }
                *tuw += 1;
                *tvw += 1;
            }
            /* ---- insert after counting.  The new edge's pair counter starts at
             * 0, not at |N_uv^(i)| as Algorithm 2 prints it: a triangle whose
             * last edge is g must not pair through g (Table I's eta, and the
             * proof of Theorem 3, count only shared edges that are last in
             * neither triangle), and only the zero start gives
             * E[eta^(i)] = eta / m^3 as Section III-B.2 states. */
            if (orc_colour(u, v, seed, k, m) == j) {
                uint64_t* cnt = um_get(&edges[i], edge_key(u, v), 0);
                if (!cnt) { rc = -1; goto done; }
                uint32_t ends[2] = {u, v}, nb[2] = {v, u};
                for (int s = 0; s < 2; ++s) {
                    uint64_t* li = um_get(&adj_index, ((uint64_t)i << 32) | ends[s], n_lists);
                    if (!li) { rc = -1; goto done; }
                    if (*li == n_lists) {
                        if (n_lists == cap_lists) {
                            uint64_t nc = cap_lists ? 2 * cap_lists : 1024;
                            vec32* nl = (vec32*)realloc(lists, nc * sizeof(vec32));
                            if (!nl) { rc = -1; goto done; }
                            lists = nl; cap_lists = nc;
                        }
                        lists[n_lists].a = NULL; lists[n_lists].n = lists[n_lists].cap = 0;
                        ++n_lists;
                    }
                    if (vec_push(&lists[*li], nb[s])) { rc = -1; goto done; }
                }
            }
        }
    }
done:
    for (uint64_t q = 0; q < n_lists; ++q) free(lists[q].a);
    free(lists);
    free(common.a);
    for (uint32_t i = i_lo; i < i_hi; ++i) um_free(&edges[i]);
    free(edges);
    um_free(&adj_index);
    return rc;
}

int orc_rept_stream(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                    uint32_t m, uint32_t c, uint64_t seed,
                    uint64_t* tau_proc, uint64_t* eta_proc,
                    uint64_t* local1, uint64_t* local2, uint64_t* eta_local,
                    uint64_t* tau_local_proc, uint64_t* skipped) {
    return sample_stream(src, dst, T, n, m, c, seed, 0, 0, c, tau_proc, eta_proc, local1, local2, eta_local,
                         tau_local_proc, skipped);
}

/*
 * The paper's multi-core design (Section IV): the processors are independent, so each runs
 * Algorithm 1 over the whole stream with its own sets, one OpenMP thread per processor at a time
 * (`threads` threads).  Same tau_proc, local1 and local2 as orc_rept_stream; used to time a
 * multi-core CPU baseline.
 */
int orc_rept_stream_parallel(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                             uint32_t m, uint32_t c, uint64_t seed, uint64_t* tau_proc,
                             uint64_t* local1, uint64_t* local2, int threads) {
    if (m == 0 || c == 0 || n == 0 || !tau_proc || !local1 || !local2 || threads < 1) return -1;
    memset(tau_proc, 0, c * sizeof(uint64_t));
    memset(local1, 0, (size_t)n * sizeof(uint64_t));
    memset(local2, 0, (size_t)n * sizeof(uint64_t));
    int rc = 0;
    #pragma omp parallel num_threads(threads)
    {
        uint64_t* tp = (uint64_t*)calloc(c, sizeof(uint64_t));
        uint64_t* l1 = (uint64_t*)calloc(n, sizeof(uint64_t));
        uint64_t* l2 = (uint64_t*)calloc(n, sizeof(uint64_t));
        uint64_t* a1 = (uint64_t*)calloc(n, sizeof(uint64_t));
        uint64_t* a2 = (uint64_t*)calloc(n, sizeof(uint64_t));
        int mine = (tp && l1 && l2 && a1 && a2) ? 0 : -1;
        #pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < (int64_t)c; ++i) {
            if (mine) continue;
            mine = sample_stream(src, dst, T, n, m, c, seed, 0, (uint32_t)i, (uint32_t)i + 1, tp, NULL, l1, l2,
                                 NULL, NULL, NULL);
            if (mine) continue;
            tau_proc[i] = tp[i];
            for (uint32_t v = 0; v < n; ++v) { a1[v] += l1[v]; a2[v] += l2[v]; }
        }
        #pragma omp critical
        {
            if (mine) rc = mine;
            else
                for (uint32_t v = 0; v < n; ++v) { local1[v] += a1[v]; local2[v] += a2[v]; }
        }
        free(tp); free(l1); free(l2); free(a1); free(a2);
    }
    return rc;
}

/*
 * Parallel MASCOT (Section I, Section III-C): c independent edge samplers with
 * p = 1/m, sampler i storing (u, v) iff h_i(u, v) == 0 (hash group i, colour 0),
 * each counting like one processor of Algorithm 1.  Outputs as for
 * orc_rept_stream; every sampler feeds local1 and local2 stays zero.
 */
int orc_mascot_stream(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                      uint32_t m, uint32_t c, uint64_t seed,
                      uint64_t* tau_proc, uint64_t* local1, uint64_t* tau_local_proc, uint64_t* skipped) {
    return sample_stream(src, dst, T, n, m, c, seed, 1, 0, c, tau_proc, NULL, local1, NULL, NULL, tau_local_proc,
                         skipped);
}

/* ------------------------------------------------------------- estimators */

/*
 * FP64 estimates from the integer counters.
 *   c <= m              : tau_hat = (m^2 / c) * sum_i tau^(i)            (Section III-A)
 *   c > m, c mod m == 0 : tau_hat = (m / c1) * sum_{i < c1 m} tau^(i)    (Section III-B.1)
 *   c > m, c mod m != 0 : inverse-variance combination of the two group
 *                         estimates with plug-in variances (Algorithm 2);
 *                         when both weights vanish the first estimate is used.
 * Local estimates use local1 / local2 / eta_local the same way (est_local may
 * be NULL).  Each scale factor is formed in double first and multiplied by the
 * exactly converted integer sum.
 */
void orc_estimates(uint32_t m, uint32_t c, const uint64_t* tau_proc, const uint64_t* eta_proc,
                   const uint64_t* local1, const uint64_t* local2, const uint64_t* eta_local,
                   uint32_t n, double* est_global, double* est_local) {
    double md = (double)m;
    uint32_t c1 = c / m, c2 = c % m;
    if (c <= m) {
        double f = md * md / (double)c;
        uint64_t s = 0;
        for (uint32_t i = 0; i < c; ++i) s += tau_proc[i];
        *est_global = (double)s * f;
        if (est_local)
            for (uint32_t v = 0; v < n; ++v) est_local[v] = (double)local1[v] * f;
        return;
    }
    double f1 = md / (double)c1;
    uint64_t s1 = 0;
    for (uint32_t i = 0; i < c1 * m; ++i) s1 += tau_proc[i];
    if (c2 == 0) {
        *est_global = (double)s1 * f1;
        if (est_local)
            for (uint32_t v = 0; v < n; ++v) est_local[v] = (double)local1[v] * f1;
        return;
    }
    double f2 = md * md / (double)c2;
    uint64_t s2 = 0, se = 0;
    for (uint32_t i = c1 * m; i < c; ++i) s2 += tau_proc[i];
    for (uint32_t i = 0; i < c; ++i) se += eta_proc[i];
    double t1 = (double)s1 * f1, t2 = (double)s2 * f2;
    double eta_hat = (double)se * (md * md * md / (double)c);
    double w1 = t1 * (md - 1.0) / (double)c1;
    double w2 = (t1 * (md * md - (double)c2) + 2.0 * eta_hat * (md - (double)c2)) / (double)c2;
    *est_global = (w1 + w2 > 0.0) ? (w2 * t1 + w1 * t2) / (w1 + w2) : t1;
    if (est_local) {
        for (uint32_t v = 0; v < n; ++v) {
            double a1 = (double)local1[v] * f1, a2 = (double)local2[v] * f2;
            double eh = (double)eta_local[v] * (md * md * md / (double)c);
            double v1 = a1 * (md - 1.0) / (double)c1;
            double v2 = (a1 * (md * md - (double)c2) + 2.0 * eh * (md - (double)c2)) / (double)c2;
            est_local[v] = (v1 + v2 > 0.0) ? (v2 * a1 + v1 * a2) / (v1 + v2) : a1;
        }
    }
}

/*
 * Parallel MASCOT's estimates (Section I, Section III-C): the mean over the c
 * samplers of the single-sampler estimate p^-2 tau^(i) = m^2 tau^(i), i.e.
 * (m^2 / c) * sum_i tau^(i); the local estimates likewise from local1.
 */
void orc_mascot_estimates(uint32_t m, uint32_t c, const uint64_t* tau_proc, const uint64_t* local1,
                          uint32_t n, double* est_global, double* est_local) {
    double md = (double)m;
    double inv_p2 = md * md;             /* one sampler's estimate is p^-2 tau^(i) */
    double mean_f = inv_p2 / (double)c;  /* ... averaged over the c samplers */
    uint64_t s = 0;
    for (uint32_t i = 0; i < c; ++i) s += tau_proc[i];
    *est_global = (double)s * mean_f;
    if (est_local)
        for (uint32_t v = 0; v < n; ++v) est_local[v] = (double)local1[v] * mean_f;
}

/* ------------------------------------------- static semi-triangle definition */

typedef struct { uint32_t nbr, eidx; } fent;

#define ATOMIC_INC(p) __atomic_fetch_add((p), 1ull, __ATOMIC_RELAXED)

static int fent_cmp(const void* a, const void* b) {
    uint32_t x = ((const fent*)a)->nbr, y = ((const fent*)b)->nbr;
    return (x > y) - (x < y);
}

/*
 * Enumerate every triangle of G once (degree-ordered forward algorithm,
 * Schank & Wagner 2005) and classify it by the definition of a
 * semi-triangle: with e1 < e2 the stream indices of its two earliest edges,
 * processor i = k*m + j (i < c) counts it iff h_k(e1) == h_k(e2) == j.
 * Also accumulates exact graph statistics used by the variance tests:
 *   tri_total   tau (all triangles), tri_local[n] tau_v,
 *   eta_total   eta = sum over edges g of C(a_g, 2), a_g = triangles that
 *               contain g with g not their last edge (two triangles share at
 *               most one edge, so every counted pair shares exactly g),
 *   eta_loc[n]  eta_v = the same sum over the edges g incident to v.
 * Any output pointer may be NULL.  Self-loops and repeated edges must not be
 * present (returns -3 if a repeated edge is found).
 */
static int enumerate_semitriangles(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                                   uint32_t m, uint32_t c, uint64_t seed, int mascot,
                                   uint64_t* tau_proc, uint64_t* local1, uint64_t* local2,
                                   uint64_t* tau_local_proc,
                                   uint64_t* tri_total, uint64_t* tri_local,
                                   uint64_t* eta_total, uint64_t* eta_loc) {
    if (n == 0 || (m == 0 && tau_proc) ) return -1;
    uint32_t c1 = m ? c / m : 0;
    uint32_t full = (mascot || c <= m) ? c : c1 * m;
    /* hash groups to classify under: one per MASCOT sampler, ceil(c/m) for REPT */
    uint32_t groups = !m ? 0 : mascot ? c : (c + m - 1) / m;
    if (tau_proc) memset(tau_proc, 0, c * sizeof(uint64_t));
    if (local1) memset(local1, 0, (size_t)n * sizeof(uint64_t));
    if (local2) memset(local2, 0, (size_t)n * sizeof(uint64_t));
    if (tau_local_proc) memset(tau_local_proc, 0, (size_t)c * n * sizeof(uint64_t));
    if (tri_total) *tri_total = 0;
    if (tri_local) memset(tri_local, 0, (size_t)n * sizeof(uint64_t));
    if (eta_total) *eta_total = 0;
    if (eta_loc) memset(eta_loc, 0, (size_t)n * sizeof(uint64_t));

    uint64_t* deg = (uint64_t*)calloc(n, sizeof(uint64_t));
    uint64_t* off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* a_g = (uint32_t*)calloc(T ? T : 1, sizeof(uint32_t));
    if (!deg || !off || !a_g) { free(deg); free(off); free(a_g); return -1; }
    for (uint64_t t = 0; t < T; ++t) {
        if (src[t] >= n || dst[t] >= n) { free(deg); free(off); free(a_g); return -2; }
        if (src[t] == dst[t]) continue;
        deg[src[t]]++; deg[dst[t]]++;
    }
    /* orientation: x -> y iff (deg x, x) < (deg y, y) */
    #define BEFORE(x, y) (deg[x] < deg[y] || (deg[x] == deg[y] && (x) < (y)))
    for (uint64_t t = 0; t < T; ++t) {
        uint32_t u = src[t], v = dst[t];
        if (u == v) continue;
        off[(BEFORE(u, v) ? u : v) + 1]++;
    }
    for (uint32_t x = 0; x < n; ++x) off[x + 1] += off[x];
    fent* fw = (fent*)malloc((off[n] ? off[n] : 1) * sizeof(fent));
    uint64_t* fill = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    if (!fw || !fill) { free(deg); free(off); free(a_g); free(fw); free(fill); return -1; }
    memcpy(fill, off, (size_t)n * sizeof(uint64_t));
    for (uint64_t t = 0; t < T; ++t) {
        uint32_t u = src[t], v = dst[t];
        if (u == v) continue;
        uint32_t x = BEFORE(u, v) ? u : v, y = (x == u) ? v : u;
        fw[fill[x]].nbr = y; fw[fill[x]].eidx = (uint32_t)t; fill[x]++;
    }
    free(fill);
    int rc = 0;
    for (uint32_t x = 0; x < n; ++x) {
        qsort(fw + off[x], off[x + 1] - off[x], sizeof(fent), fent_cmp);
        for (uint64_t q = off[x] + 1; q < off[x + 1]; ++q)
            if (fw[q].nbr == fw[q - 1].nbr) rc = -3;
    }
    if (rc) goto out;

    /* The enumeration is split over threads by node x (OpenMP when compiled with it); counters are
     * shared and updated atomically, so the totals do not depend on the split. */
    uint64_t tri_count = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(+ : tri_count)
    for (uint32_t x = 0; x < n; ++x) {
        for (uint64_t p = off[x]; p < off[x + 1]; ++p) {
            uint32_t y = fw[p].nbr;
            uint32_t e_xy = fw[p].eidx;
            /* merge N+(x) and N+(y), both sorted by node id */
            uint64_t a = off[x], ae = off[x + 1], b = off[y], be = off[y + 1];
            while (a < ae && b < be) {
                if (fw[a].nbr < fw[b].nbr) { ++a; continue; }
                if (fw[a].nbr > fw[b].nbr) { ++b; continue; }
                uint32_t z = fw[a].nbr, e_xz = fw[a].eidx, e_yz = fw[b].eidx;
                ++a; ++b;
                /* triangle {x, y, z} with edge indices e_xy, e_xz, e_yz */
                uint32_t e[3] = {e_xy, e_xz, e_yz};
                uint32_t ends[3][2] = {{x, y}, {x, z}, {y, z}};
                int last = 0;
                for (int q = 1; q < 3; ++q) if (e[q] > e[last]) last = q;
                int f1 = (last + 1) % 3, f2 = (last + 2) % 3;   /* the two earliest edges */
                ++tri_count;
                if (tri_local) { ATOMIC_INC(&tri_local[x]); ATOMIC_INC(&tri_local[y]); ATOMIC_INC(&tri_local[z]); }
                __atomic_fetch_add(&a_g[e[f1]], 1u, __ATOMIC_RELAXED);
                __atomic_fetch_add(&a_g[e[f2]], 1u, __ATOMIC_RELAXED);
                for (uint32_t k = 0; k < groups; ++k) {
                    uint32_t j1 = orc_colour(ends[f1][0], ends[f1][1], seed, k, m);
                    uint32_t j2 = orc_colour(ends[f2][0], ends[f2][1], seed, k, m);
                    uint32_t i = mascot ? k : k * m + j1;
                    if (j1 != j2 || i >= c || (mascot && j1 != 0)) continue;
                    if (tau_proc) ATOMIC_INC(&tau_proc[i]);
                    uint64_t* l_sum = (i < full) ? local1 : local2;
                    if (l_sum) { ATOMIC_INC(&l_sum[x]); ATOMIC_INC(&l_sum[y]); ATOMIC_INC(&l_sum[z]); }
                    if (tau_local_proc) {
                        ATOMIC_INC(&tau_local_proc[(uint64_t)i * n + x]);
                        ATOMIC_INC(&tau_local_proc[(uint64_t)i * n + y]);
                        ATOMIC_INC(&tau_local_proc[(uint64_t)i * n + z]);
                    }
                }
            }
        }
    }
    if (tri_total) *tri_total = tri_count;
    if (eta_total || eta_loc) {
        for (uint64_t t = 0; t < T; ++t) {
            uint64_t pairs = (uint64_t)a_g[t] * (a_g[t] - (a_g[t] ? 1 : 0)) / 2;
            if (eta_total) *eta_total += pairs;
            if (eta_loc && src[t] != dst[t]) { eta_loc[src[t]] += pairs; eta_loc[dst[t]] += pairs; }
        }
    }
    #undef BEFORE
out:
    free(deg); free(off); free(a_g); free(fw);
    return rc;
}

int orc_semitriangles(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                      uint32_t m, uint32_t c, uint64_t seed,
                      uint64_t* tau_proc, uint64_t* local1, uint64_t* local2,
                      uint64_t* tau_local_proc,
                      uint64_t* tri_total, uint64_t* tri_local,
                      uint64_t* eta_total, uint64_t* eta_loc) {
    return enumerate_semitriangles(src, dst, T, n, m, c, seed, 0, tau_proc, local1, local2, tau_local_proc,
                                   tri_total, tri_local, eta_total, eta_loc);
}

/* The same enumeration classified for parallel MASCOT: sampler i counts a
 * triangle iff its two earliest edges both have h_i colour 0. */
int orc_mascot_semitriangles(const uint32_t* src, const uint32_t* dst, uint64_t T, uint32_t n,
                             uint32_t m, uint32_t c, uint64_t seed,
                             uint64_t* tau_proc, uint64_t* local1, uint64_t* tau_local_proc) {
    return enumerate_semitriangles(src, dst, T, n, m, c, seed, 1, tau_proc, local1, NULL, tau_local_proc,
                                   NULL, NULL, NULL, NULL);
}
