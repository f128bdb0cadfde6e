/*
 * Seeded synthetic edge-stream generators (Chung-Lu power-law and R-MAT).
 *
 * These stand in for the real graphs of the evaluation (Section IV-A,
 * Table II), which are not available here: heavy-tailed degree
 * distributions, undirected simple graphs, streamed in a uniformly random
 * order.  This file holds no arithmetic of the counting method itself; both
 * the CPU oracle and the CUDA path consume the arrays it writes.
 *
 * Randomness: PCG32 (O'Neill 2014, "PCG: A Family of Simple Fast
 * Space-Efficient Statistically Good Algorithms for Random Number
 * Generation"), XSH-RR output, one independent stream per purpose.  Integer
 * and double arithmetic only, no platform intrinsics: the output is the same
 * on x86_64 and aarch64.
 *
 * Output contract of every generator: `src[i], dst[i]` for i < returned
 * count, node ids in [0, n), no self-loops, no duplicate undirected edges,
 * each edge randomly oriented, the edge list in a seeded uniform random
 * order (Fisher-Yates), node ids scrambled by a seeded random permutation so
 * that degree does not follow id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t state, inc; } pcg32;

static uint32_t pcg32_next(pcg32* r) {
    uint64_t old = r->state;
    r->state = old * 6364136223846793005ULL + r->inc;
    uint32_t xs = (uint32_t)(((old >> 18u) ^ old) >> 27u);
    uint32_t rot = (uint32_t)(old >> 59u);
    return (xs >> rot) | (xs << ((32u - rot) & 31u));
}

static void pcg32_seed(pcg32* r, uint64_t initstate, uint64_t initseq) {
    r->state = 0u;
    r->inc = (initseq << 1u) | 1u;
    pcg32_next(r);
    r->state += initstate;
    pcg32_next(r);
}

/* uniform double in [0,1) with 53 random bits */
static double pcg32_double(pcg32* r) {
    uint64_t a = pcg32_next(r) >> 5, b = pcg32_next(r) >> 6;
    return (double)(a * 67108864ULL + b) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, bound) for bound < 2^32 (Lemire's nearly-divisionless method) */
static uint32_t pcg32_bounded(pcg32* r, uint32_t bound) {
    uint64_t m = (uint64_t)pcg32_next(r) * bound;
    uint32_t l = (uint32_t)m;
    if (l < bound) {
        uint32_t t = (uint32_t)(-bound) % bound;
        while (l < t) { m = (uint64_t)pcg32_next(r) * bound; l = (uint32_t)m; }
    }
    return (uint32_t)(m >> 32);
}

/* uniform 64-bit index in [0, bound) for bound up to 2^63 (rejection on a mask) */
static uint64_t pcg32_bounded64(pcg32* r, uint64_t bound) {
    if (bound <= 0xFFFFFFFFULL) return pcg32_bounded(r, (uint32_t)bound);
    uint64_t mask = bound - 1;
    mask |= mask >> 1; mask |= mask >> 2; mask |= mask >> 4;
    mask |= mask >> 8; mask |= mask >> 16; mask |= mask >> 32;
    for (;;) {
        uint64_t x = (((uint64_t)pcg32_next(r) << 32) | pcg32_next(r)) & mask;
        if (x < bound) return x;
    }
}

/* ---- open-addressing set of undirected edge keys (min<<32 | max) ---- */
typedef struct { uint64_t* slot; uint64_t mask; uint64_t n; } keyset;
#define KS_EMPTY 0xFFFFFFFFFFFFFFFFULL

static int keyset_init(keyset* s, uint64_t expect) {
    uint64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    s->slot = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!s->slot) return -1;
    memset(s->slot, 0xFF, cap * sizeof(uint64_t));
    s->mask = cap - 1; s->n = 0;
    return 0;
}

static uint64_t mix_key(uint64_t k) {  /* Murmur3 64-bit finaliser, for slot choice only */
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33; return k;
}

/* returns 1 if inserted, 0 if already present */
static int keyset_add(keyset* s, uint64_t key) {
    uint64_t h = mix_key(key) & s->mask;
    for (;;) {
        if (s->slot[h] == KS_EMPTY) { s->slot[h] = key; s->n++; return 1; }
        if (s->slot[h] == key) return 0;
        h = (h + 1) & s->mask;
    }
}

/* shuffle the edge list, orient each edge at random, relabel nodes */
static void finish_stream(uint64_t* keys, uint64_t ne, uint32_t n, uint64_t graph_seed,
                          uint64_t order_seed, uint32_t* src, uint32_t* dst, int relabel) {
    pcg32 ro; pcg32_seed(&ro, order_seed, 0x5EED0DE5ULL);
    for (uint64_t i = ne; i > 1; --i) {                 /* Fisher-Yates */
        uint64_t j = pcg32_bounded64(&ro, i);
        uint64_t t = keys[i - 1]; keys[i - 1] = keys[j]; keys[j] = t;
    }
    uint32_t* perm = NULL;
    if (relabel) {
        perm = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
        for (uint32_t i = 0; i < n; ++i) perm[i] = i;
        pcg32 rp; pcg32_seed(&rp, graph_seed, 0x9E12D0ULL);
        for (uint32_t i = n; i > 1; --i) {
            uint32_t j = pcg32_bounded(&rp, i);
            uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
        }
    }
    for (uint64_t i = 0; i < ne; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        if (perm) { a = perm[a]; b = perm[b]; }
        if (pcg32_next(&ro) & 1u) { uint32_t t = a; a = b; b = t; }
        src[i] = a; dst[i] = b;
    }
    free(perm);
}

/*
 * Chung-Lu graph: node i gets weight w_i proportional to (i+1)^(-1/(gamma-1)),
 * scaled so that the weights sum to 2*n_edges and (if cap > 0) clipped at
 * `cap` with the remainder re-scaled (a few fixed-point passes).  Endpoint
 * pairs are drawn i.i.d. with probability proportional to w (inverse CDF),
 * self-loops and repeats discarded, until `n_edges` distinct undirected edges
 * exist (or `max_draws` draws were made).  Returns the number of edges.
 */
int64_t gg_chung_lu(uint32_t n, double gamma, double cap, uint64_t n_edges, uint64_t max_draws,
                    uint64_t graph_seed, uint64_t order_seed, uint32_t* src, uint32_t* dst) {
    if (n < 2 || gamma <= 1.0 || n_edges == 0) return -1;
    double* cdf = (double*)malloc((size_t)n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    if (!cdf || !w) { free(cdf); free(w); return -2; }
    double expo = -1.0 / (gamma - 1.0), sum = 0.0;
    for (uint32_t i = 0; i < n; ++i) { w[i] = pow((double)i + 1.0, expo); sum += w[i]; }
    double target = 2.0 * (double)n_edges;
    for (uint32_t i = 0; i < n; ++i) w[i] *= target / sum;
    if (cap > 0) {
        for (int pass = 0; pass < 50; ++pass) {
            double capped = 0.0, free_sum = 0.0;
            for (uint32_t i = 0; i < n; ++i) {
                if (w[i] >= cap) { w[i] = cap; capped += cap; } else free_sum += w[i];
            }
            if (free_sum <= 0.0) break;
            double scale = (target - capped) / free_sum;
            if (scale <= 1.0 + 1e-12) break;
            for (uint32_t i = 0; i < n; ++i) if (w[i] < cap) w[i] *= scale;
        }
        for (uint32_t i = 0; i < n; ++i) if (w[i] > cap) w[i] = cap;
    }
    double acc = 0.0;
    for (uint32_t i = 0; i < n; ++i) { acc += w[i]; cdf[i] = acc; }
    free(w);
    keyset ks;
    if (keyset_init(&ks, n_edges)) { free(cdf); return -2; }
    uint64_t* keys = (uint64_t*)malloc(n_edges * sizeof(uint64_t));
    if (!keys) { free(cdf); free(ks.slot); return -2; }
    pcg32 rg; pcg32_seed(&rg, graph_seed, 0xC1C1ULL);
    uint64_t ne = 0, draws = 0;
    while (ne < n_edges && draws < max_draws) {
        uint32_t e[2];
        for (int s = 0; s < 2; ++s) {
            double x = pcg32_double(&rg) * acc;
            uint32_t lo = 0, hi = n - 1;              /* first index with cdf > x */
            while (lo < hi) { uint32_t mid = lo + (hi - lo) / 2; if (cdf[mid] > x) hi = mid; else lo = mid + 1; }
            e[s] = lo;
        }
        ++draws;
        if (e[0] == e[1]) continue;
        uint32_t a = e[0] < e[1] ? e[0] : e[1], b = e[0] < e[1] ? e[1] : e[0];
        uint64_t key = ((uint64_t)a << 32) | b;
        if (keyset_add(&ks, key)) keys[ne++] = key;
    }
    free(cdf); free(ks.slot);
    finish_stream(keys, ne, n, graph_seed, order_seed, src, dst, 1);
    free(keys);
    return (int64_t)ne;
}

/*
 * R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004): `n_draws` edges, each
 * placed by `scale` recursive choices of a quadrant with probabilities
 * (a, b, c, 1-a-b-c); self-loops and repeated undirected pairs dropped.
 * Returns the number of distinct edges (<= n_draws).
 */
int64_t gg_rmat(uint32_t scale, uint64_t n_draws, double a, double b, double c,
                uint64_t graph_seed, uint64_t order_seed, uint32_t* src, uint32_t* dst) {
    if (scale == 0 || scale > 31 || n_draws == 0) return -1;
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)(a * two32), tab = (uint64_t)((a + b) * two32),
             tabc = (uint64_t)((a + b + c) * two32);
    keyset ks;
    if (keyset_init(&ks, n_draws)) return -2;
    uint64_t* keys = (uint64_t*)malloc(n_draws * sizeof(uint64_t));
    if (!keys) { free(ks.slot); return -2; }
    pcg32 rg; pcg32_seed(&rg, graph_seed, 0x2A7ULL);
    uint64_t ne = 0;
    for (uint64_t d = 0; d < n_draws; ++d) {
        uint32_t x = 0, y = 0;
        for (uint32_t l = 0; l < scale; ++l) {
            uint64_t r = pcg32_next(&rg);
            uint32_t bx = r >= tab, by = (r >= ta && r < tab) || r >= tabc;
            x = (x << 1) | bx; y = (y << 1) | by;
        }
        if (x == y) continue;
        uint32_t lo = x < y ? x : y, hi = x < y ? y : x;
        uint64_t key = ((uint64_t)lo << 32) | hi;
        if (keyset_add(&ks, key)) keys[ne++] = key;
    }
    free(ks.slot);
    finish_stream(keys, ne, 1u << scale, graph_seed, order_seed, src, dst, 1);
    free(keys);
    return (int64_t)ne;
}

/*
 * Erdos-Renyi G(n, q) on small n for tests: every pair independently with
 * probability q, then shuffled (no relabelling).  Returns the edge count;
 * `cap_edges` bounds the output.
 */
int64_t gg_gnp(uint32_t n, double q, uint64_t graph_seed, uint64_t order_seed,
               uint32_t* src, uint32_t* dst, uint64_t cap_edges) {
    pcg32 rg; pcg32_seed(&rg, graph_seed, 0x6E9ULL);
    uint64_t total = (uint64_t)n * (n - 1) / 2;
    uint64_t* keys = (uint64_t*)malloc((total ? total : 1) * sizeof(uint64_t));
    if (!keys) return -2;
    uint64_t ne = 0;
    for (uint32_t i = 0; i < n; ++i)
        for (uint32_t j = i + 1; j < n; ++j)
            if (pcg32_double(&rg) < q) keys[ne++] = ((uint64_t)i << 32) | j;
    if (ne > cap_edges) { free(keys); return -3; }
    finish_stream(keys, ne, n, graph_seed, order_seed, src, dst, 0);
    free(keys);
    return (int64_t)ne;
}

/* seeded uniform shuffle of an existing edge list (used to re-order a stream) */
void gg_shuffle(uint32_t* src, uint32_t* dst, uint64_t ne, uint64_t order_seed) {
    pcg32 ro; pcg32_seed(&ro, order_seed, 0x5EED0DE5ULL);
    for (uint64_t i = ne; i > 1; --i) {
        uint64_t j = pcg32_bounded64(&ro, i);
        uint32_t t = src[i - 1]; src[i - 1] = src[j]; src[j] = t;
        t = dst[i - 1]; dst[i - 1] = dst[j]; dst[j] = t;
    }
}

/* PCG32 sample stream, exposed so tests can check it against published output */
void gg_pcg32_fill(uint64_t initstate, uint64_t initseq, uint32_t* out, uint64_t n) {
    pcg32 r; pcg32_seed(&r, initstate, initseq);
    for (uint64_t i = 0; i < n; ++i) out[i] = pcg32_next(&r);
}
