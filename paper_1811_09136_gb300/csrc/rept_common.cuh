// Device-side data layout and helpers of the REPT streaming counter.
//
// HBM layout of one stream (one rept_state):
//   meta[n_nodes]   uint4 {off, cnt, add, 0}: node x's block starts at slot
//                   4*off of the pool and holds cnt entries; its size is a
//                   function of cnt alone (table_lg below), so a node's block
//                   is re-allocated exactly when cnt crosses a power-of-two
//                   boundary.  add counts the current batch's new entries of x
//                   (zero between batches); it shares x's 16-byte record so
//                   that the insert's position counter and the block's place
//                   sit in one 32-byte sector.  k_classify counts into the
//                   compact array cnt_add[n_nodes] first; k_plan moves the
//                   counts into the records.
//   pool[]          8-byte slots: per node, an open-addressing (linear probing,
//                   4-key buckets) table of 2^lg neighbour ids and their stream
//                   indices (2^lg slots in all; for streams with stored colours
//                   each 32-byte bucket holds its 4 ids and then their 4
//                   indices, so that an insert or a probe hit touches one
//                   sector; streams that probe every candidate keep all ids
//                   first and the indices after them, ids packed densely), then
//                   the same entries as a packed list of {nbr, eidx} pairs
//                   (and, for streams with colour words, one word per entry).
//                   An entry (w, t) of x is the stored edge {x, w} that
//                   arrived at stream index t.  Empty keys are all-ones.  The
//                   tables of all processors share one union adjacency: an
//                   edge is stored once if any processor keeps it, and which
//                   processors keep it is recomputed from the hash when needed
//                   (Section III-A: processor i keeps colour i).
//   local[n_nodes]  uint64 sum over processors of tau_v^(i)
//   proc[c]         uint64 tau^(i)
// Per-batch scratch: touched[] (nodes with add > 0), grow_rel[] (their new
// table's offset relative to this batch's allocation), the work records, and
// the control block.
#pragma once

#include <cstdint>
#include <cstdio>

#include "rept.h"

namespace rept {

constexpr uint32_t kEmptyId = 0xFFFFFFFFu;
constexpr unsigned long long kEmptySlot = 0xFFFFFFFFFFFFFFFFull;
constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment
constexpr uint32_t kIdBits = 24;                             // node-id bits of a list entry with a colour
constexpr uint32_t kIdMask = (1u << kIdBits) - 1u;
constexpr uint32_t kNoGrow = 0xFFFFFFFFu;
constexpr uint32_t kMaxProcessors = 4096;  // per-block tau^(i) histogram lives in shared memory
// Number of k_intersect work classes (see bin_of_cnt).
constexpr int kBins = 6;
// Within a class, work items are ordered by a hash of the larger endpoint (kKeyBits bits), so that
// the edges probing the same large table run back to back and find it in L2.
constexpr int kKeyBits = 13;
constexpr uint32_t kKeyBuckets = 1u << kKeyBits;
constexpr uint32_t kSortBuckets = kBins * kKeyBuckets;
constexpr uint16_t kNoKey = 0xFFFFu;

// status bits (sticky)
constexpr unsigned kStRange = 1u, kStCapacity = 2u, kStInternal = 4u, kStTimeout = 8u, kStDuplicate = 16u;
constexpr unsigned kStBounds = 32u;  // REPT_DEBUG_BOUNDS builds: an index check failed

// The REPT_E_* code (rept.h) that a sticky status word reports, most specific condition first.  A
// failed index check of the REPT_DEBUG_BOUNDS build is an internal error.
inline int status_to_code(unsigned st) {
    if (st & kStRange) return REPT_E_RANGE;
    if (st & kStCapacity) return REPT_E_CAPACITY;
    if (st & kStTimeout) return REPT_E_TIMEOUT;
    if (st & kStInternal) return REPT_E_INTERNAL;
    if (st & kStDuplicate) return REPT_E_DUPLICATE;
    if (st & kStBounds) return REPT_E_INTERNAL;
    return REPT_OK;
}

// REPT_DEBUG_BOUNDS builds: print the first failed index check ({site, index, bound, failures}, the
// `dbg` words of the control block) to stderr.
inline void report_failed_check(const unsigned long long* dbg) {
    if (dbg[3])
        std::fprintf(stderr, "rept: index check at site %llu failed: index %llu, bound %llu (%llu failures)\n",
                     dbg[0], dbg[1], dbg[2], dbg[3]);
}

// x mod m for 64-bit x and 32-bit m >= 2 without a division: Lemire, Kaser, Kurz, "Faster Remainder
// by Direct Computation" (2019).  With the 128-bit magic M = floor((2^128 - 1) / m) + 1, the low 128
// bits of M * x, multiplied by m, hold x mod m in their top 64 bits; 128 >= 64 + log2(m) bits of magic
// make this exact for every 64-bit x.
struct FastMod {
    uint64_t mh, ml;  // M = mh * 2^64 + ml
    uint64_t qinv;    // m = q * 2^k with q odd: q^-1 mod 2^64
    uint64_t lim;     // floor((2^64 - 1) / m)
    uint32_t m;
    uint32_t k;
};

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

inline FastMod make_fastmod(uint32_t m) {
    FastMod f{0, 0, 0, 0, m, 0};
    if (m >= 2) {
        // divisibility test constants: the odd part's inverse by Newton's iteration (q*q = 1 mod 8
        // gives 3 correct bits; each step doubles them), and the largest quotient
        uint32_t k = 0;
        while (((m >> k) & 1u) == 0u) ++k;
        const uint64_t q = m >> k;
        uint64_t inv = q;
        for (int it = 0; it < 6; ++it) inv *= 2u - q * inv;
        f.qinv = inv;
        f.k = k;
        f.lim = ~0ull / m;
        // floor((2^128 - 1) / m) + 1, by long division of the all-ones 128-bit value
        const uint64_t ones = ~0ull;
        const uint64_t qh = ones / m, rh = ones % m;
        const unsigned __int128 low = ((unsigned __int128)rh << 64) | ones;
        const uint64_t ql = (uint64_t)(low / m);
        f.ml = ql + 1;
        f.mh = qh + (f.ml == 0 ? 1 : 0);
    }
    return f;
}

__host__ __device__ __forceinline__ uint32_t fast_mod(uint64_t x, const FastMod& f) {
    if (f.m < 2) return 0u;
    const uint64_t ll = f.ml * x;                        // low 128 bits of M * x: (lh, ll)
    const uint64_t lh = mulhi64(f.ml, x) + f.mh * x;
    const uint64_t a = lh * (uint64_t)f.m;               // (lh, ll) * m >> 128
    const uint64_t b = mulhi64(ll, (uint64_t)f.m);
    return (uint32_t)(mulhi64(lh, (uint64_t)f.m) + ((a + b) < a ? 1u : 0u));
}

// x mod m == j for j < m, without forming the remainder: x >= j and n = x - j divisible by m.  With
// m = q * 2^k (q odd), n is a multiple of m exactly when (n * q^-1 mod 2^64) rotated right by k is at
// most floor((2^64 - 1) / m) (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, Section 9): one 64-bit multiply instead of a remainder.
// mod_equals_in_range assumes m >= 2 and j < m; mod_equals takes any m and j.
__host__ __device__ __forceinline__ bool mod_equals_in_range(uint64_t x, uint32_t j, const FastMod& f) {
    if (x < j) return false;
    const uint64_t y = (x - j) * f.qinv;
#ifdef __CUDA_ARCH__
    // rotate right by k < 32 (m < 2^32): each half is a funnel shift of the two halves
    const uint32_t lo = (uint32_t)y, hi = (uint32_t)(y >> 32);
    const uint64_t r = ((uint64_t)__funnelshift_r(hi, lo, f.k) << 32) | __funnelshift_r(lo, hi, f.k);
#else
    const uint64_t r = (y >> f.k) | (y << ((64u - f.k) & 63u));
#endif
    return r <= f.lim;
}

// The same test without a branch: every lane forms the product, so lanes of a warp never part ways
// over it (x - j wraps when x < j, and the first factor then makes the result false).
__host__ __device__ __forceinline__ bool mod_equals_nobranch(uint64_t x, uint32_t j, const FastMod& f) {
    const uint64_t y = (x - j) * f.qinv;
#ifdef __CUDA_ARCH__
    const uint32_t lo = (uint32_t)y, hi = (uint32_t)(y >> 32);
    const uint64_t r = ((uint64_t)__funnelshift_r(hi, lo, f.k) << 32) | __funnelshift_r(lo, hi, f.k);
#else
    const uint64_t r = (y >> f.k) | (y << ((64u - f.k) & 63u));
#endif
    return (x >= j) & (r <= f.lim);
}

__host__ __device__ __forceinline__ bool mod_equals(uint64_t x, uint32_t j, const FastMod& f) {
    if (f.m < 2) return j == 0u;
    if (j >= f.m) return false;
    return mod_equals_in_range(x, j, f);
}

struct Ctrl {
    unsigned long long n_touched;   // nodes in touched[] this batch
    unsigned long long need_quads;  // table space requested by this batch, in 4-slot units
    unsigned long long pool_top;    // 4-slot units handed out so far
    unsigned long long self_loops;
    unsigned long long stored;      // stored (kept) edges
    unsigned int status;
    unsigned int pad;
    // work counters of k_intersect<true> (see rept_stats)
    unsigned long long small_entries, small_slots, probes, probe_slots, wedges, counted;
    unsigned long long class_items[6], class_probes[6], class_cycles[6];
    // per-batch work list of k_intersect: class c occupies items[bin_start[c] .. + bin_count[c])
    unsigned long long bin_start[kBins];
    unsigned long long bin_count[kBins];
    unsigned long long bin_next[kBins];
    unsigned long long n_pairs;  // entries of pair_list this batch
    unsigned long long n_big;   // nodes whose table (32..2048 slots) k_rehash_big moves, a warp each
    unsigned long long n_huge;  // nodes whose table (>= 4096 slots) k_rehash_huge moves, a block each
    unsigned long long huge_next;
    unsigned long long dbg[4];  // REPT_DEBUG_BOUNDS builds: first failed check {site, index, bound}, count
};

// What k_intersect needs about one arriving edge t = (s, l), s the endpoint with the smaller table:
// both tables' offsets (in 4-slot units) and sizes, written by k_insert once the batch's tables are
// final, then moved into sorted order by k_sort_scatter.
struct __align__(16) WorkItem {
    uint32_t s, l, off_s, off_l;
    uint32_t t;      // stream index of the edge
    uint32_t lgs;    // log2 table sizes: smaller | larger << 8
    uint32_t cnt_s;  // entries of the smaller endpoint
    uint32_t key;    // work class * kKeyBuckets + hash of l, or kNoKey
};

// Everything a kernel needs to know about one stream's state.
struct StreamDev {
    uint32_t m, c, groups, n_nodes;
    uint64_t seed;
    FastMod fm;         // x mod m
    uint32_t tile_max;  // edges whose smaller endpoint has more entries get a warp (4, 8, 16 or 32)
    uint4* meta;  // per node {block offset in 4-slot units, entries, this batch's new entries, 0}
    uint32_t* cnt_add;  // [n_nodes] new entries per node as k_classify counts them (a compact array, so
                        // that its atomics stay in L2); k_plan moves each touched node's count into its
                        // record and clears it, so it is zero between batches
    uint2* pool;
    unsigned long long pool_quads;
    // How list entries carry their edge's colours (the intersection tests colours before it probes):
    // kColNone: plain entries; kColInEntry: every list entry {w, t} of node x carries h_0(x, w) in
    // the top 8 bits of its first word (w itself in the low kIdBits), for one hash group,
    // 2 <= m <= 256 and n_nodes <= 2^kIdBits; kColWords: a parallel array of 32-bit words beside
    // the list holds h_k(x, w) of every hash group k in bits [k * cbits, (k + 1) * cbits), for REPT
    // with groups * cbits <= 32
    uint32_t colours;
    uint32_t cbits;  // kColWords: bits per group colour, ceil(log2 m)
    uint32_t cmask;  // (1 << cbits) - 1
    unsigned long long* local;
    unsigned long long* proc;
    uint32_t* touched;
    uint32_t* grow_rel;
    struct WorkItem* rec;   // [max_batch] work record of each edge (key kNoKey if it closes no wedge)
    struct WorkItem* srec;  // [max_batch] the records of edges that can close wedges, sorted by key
    uint32_t* hist;         // [kSortBuckets] counts, then cursors, of the counting sort by key
    uint32_t* big;      // [big_cap] touched-list indices of nodes with a large table to move: the
                        // k_rehash_big list from the front, the k_rehash_huge list from the back
    unsigned long long big_cap;
    Ctrl* ctrl;
    // c > m with c mod m != 0 (Algorithm 2): the partial group's local counts and the triangle-pair
    // counters; all NULL otherwise
    uint32_t c1;                    // full groups: processors i < c1 * m feed `local`, the rest `local2`
    uint32_t keep;                  // colours each hash group keeps: m (REPT), 1 (parallel MASCOT)
    uint32_t pstride;               // processors per hash group: m (REPT), 1 (parallel MASCOT)
    // colour sharding: this state keeps processors [pbeg, pbeg + pcount) only (all c by default),
    // which belong to hash groups [kbeg, kend)
    uint32_t pbeg, pcount, kbeg, kend;
    unsigned long long* local2;     // [n_nodes] sum of tau_v^(i) over the partial group
    unsigned long long* eta_proc;   // [c] eta^(i)
    unsigned long long* eta_local;  // [n_nodes] sum over processors of eta_v^(i)
    uint2* edge_ends;               // [pair_cap] endpoints of the stored edge with stream index t
    uint32_t* pair_tau;             // [pair_cap * groups] tau_(e)^(i) of edge e in group k (Algorithm 2)
    uint32_t* pair_evt;             // [pair_cap * groups] this batch's closed wedges through (e, k)
    uint32_t* pair_list;            // [pair_cap * groups] the (e, k) with events this batch: e * groups + k
    unsigned long long pair_cap;    // stream indices covered by the pair arrays
    unsigned long long* local_proc; // [c * n_nodes] tau_v^(i), processor-major (REPT_FLAG_LOCAL_PER_PROCESSOR)
};

// The block a batch kernel's body runs as: its index among the nbx blocks that share one stream's
// work (blockIdx.x and gridDim.x for a launch per stream, or a virtual block of the persistent group
// kernel, which runs every step of the batch path for every stream of a group).
struct Grid {
    uint32_t bx, nbx;
};

// Grid-wide barrier state of the persistent group kernel (one per group, in device memory).  The
// host clears count and timed_out before each launch and sets extra: the arrivals a barrier waits for
// beyond the grid's blocks (0; a test sets 1 so that the wait can only run out).
struct GroupSync {
    unsigned int count;      // blocks arrived at the current barrier
    unsigned int gen;        // barriers completed (advanced by the last block to arrive)
    unsigned int timed_out;  // some block's wait gave up
    unsigned int extra;
};

// One batch of edges appended to a stream.
struct BatchDev {
    const uint32_t* src;
    const uint32_t* dst;
    unsigned long long n;
    unsigned long long t0;  // stream index of src[0], dst[0]
};

// Index checks of the REPT_DEBUG_BOUNDS build (a stand-in for a memory checker): a failed check
// records {site, index, bound} once, counts, raises kStBounds, and the caller skips the access.
// Release builds compile them away.
#ifdef REPT_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_ok(Ctrl* c, unsigned site, unsigned long long idx, unsigned long long bound) {
    if (idx < bound) return true;
    if (atomicAdd(&c->dbg[3], 1ull) == 0ull) {
        c->dbg[0] = site;
        c->dbg[1] = idx;
        c->dbg[2] = bound;
    }
    atomicOr(&c->status, kStBounds);
    return false;
}
#define REPT_CHECK(c, site, idx, bound) dbg_ok((c), (site), (idx), (bound))
#else
#define REPT_CHECK(c, site, idx, bound) true
#endif

// One output step of SplitMix64 from state x (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + kGoldenGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// h_k({a, b}) given the group seed s_k.
__device__ __forceinline__ uint32_t colour_of(uint32_t a, uint32_t b, uint64_t s_k, const FastMod& fm) {
    uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    return fast_mod(splitmix64(((lo << 32) | hi) ^ s_k), fm);
}

__device__ __forceinline__ uint64_t group_seed(uint64_t seed, uint32_t k) { return seed + (uint64_t)k * kGoldenGamma; }

// h_k({a, b}) == j, for m >= 2 and a colour j < m.
__device__ __forceinline__ bool colour_is(uint32_t a, uint32_t b, uint64_t s_k, const FastMod& fm, uint32_t j) {
    uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    return mod_equals_in_range(splitmix64(((lo << 32) | hi) ^ s_k), j, fm);
}

// Do the wedge edges {s, w} and {l, w} have the same colour in the group of seed s_k?  Their hash
// values are congruent modulo m exactly when m divides their (exact, non-negative) difference, which
// the divisibility test decides without a remainder; only then is the colour j itself formed.
__device__ __forceinline__ bool same_colour(uint32_t s, uint32_t l, uint32_t w, uint64_t s_k, const FastMod& fm,
                                            uint32_t& j) {
    const uint64_t ks = ((uint64_t)(s < w ? s : w) << 32) | (s < w ? w : s);
    const uint64_t kl = ((uint64_t)(l < w ? l : w) << 32) | (l < w ? w : l);
    const uint64_t zs = splitmix64(ks ^ s_k), zl = splitmix64(kl ^ s_k);
    if (!mod_equals_nobranch(zs >= zl ? zs - zl : zl - zs, 0u, fm)) return false;
    j = fast_mod(zs, fm);
    return true;
}

// Is edge {u, v} kept by some processor (k*m + h_k(u,v) < c for some group k)?
// The processor that keeps colour j of hash group k, if any: REPT's processor i = k*m + j (i < c);
// parallel MASCOT's sampler i = k keeps colour 0 only (an independent p = 1/m sample per group).
// Only the processors of this state's shard count (pbeg + pcount <= c, so i < c as well).
__device__ __forceinline__ bool processor_of(const StreamDev& d, uint32_t k, uint32_t j, uint32_t& i) {
    i = k * d.pstride + j;
    return j < d.keep && i - d.pbeg < d.pcount;
}

__device__ __forceinline__ bool kept_by_any(const StreamDev& d, uint32_t u, uint32_t v) {
    for (uint32_t k = d.kbeg; k < d.kend; ++k) {
        uint32_t i, j = colour_of(u, v, group_seed(d.seed, k), d.fm);
        if (processor_of(d, k, j, i)) return true;
    }
    return false;
}

constexpr uint32_t kColNone = 0u, kColInEntry = 1u, kColWords = 2u;

// The mask that takes a node id out of the first word of a list entry.
__host__ __device__ __forceinline__ uint32_t id_mask(const StreamDev& d) {
    return d.colours == kColInEntry ? kIdMask : ~0u;
}
__host__ __device__ __forceinline__ bool has_words(const StreamDev& d) { return d.colours == kColWords; }
// The stream's tables are interleaved (key_word) exactly when it stores colours.
__host__ __device__ __forceinline__ bool tables_interleaved(const StreamDev& d) { return d.colours != kColNone; }

// With one hash group, a wedge (s, w), (l, w) can count only for the processor of colour
// js = h_0(s, w), and only if that processor exists and h_0(l, w) = js.  The intersection reads js from
// s's list entry and asks this of the hash alone before it probes l's table for w, so all but about
// 1/m of the probes are skipped.
__device__ __forceinline__ bool wedge_may_count(const StreamDev& d, uint32_t l, uint32_t w, uint32_t js) {
    // every step evaluated and combined with & (no early exit), so the lanes of a warp never part
    // ways over it (measured 4 % faster than the short-circuit form).  With one hash group the
    // processor of colour js is js itself: REPT keeps every colour below m (and js < m), parallel
    // MASCOT's single sampler keeps colour 0 only (pbeg = 0, pcount = 1), so the shard's range test
    // alone decides processor_of here.
    const uint64_t lo = l < w ? l : w, hi = l < w ? w : l;
    const uint64_t z = splitmix64(((lo << 32) | hi) ^ d.seed);
    return (js - d.pbeg < d.pcount) & mod_equals_nobranch(z, js, d.fm);
}

// The scans' form of wedge_may_count: a superset test.  It never rejects an entry whose wedge can
// count, and may pass a few whose wedge cannot; count_wedge decides every queued wedge exactly.
// z mod m = js implies that m divides z - js, i.e. that r = rotr((z - js) q^-1, k) <= floor((2^64 - 1)
// / m); only the high words are compared (a pass rate of about 1/m + 2^-32).  The range test of
// wedge_may_count is left out: every entry of a list carries a kept colour (its edge is stored
// because this state's processor of that colour keeps it), and z < js, which the exact test
// excludes, has probability below 2^-56.
__device__ __forceinline__ bool colour_may_match(const StreamDev& d, uint32_t l, uint32_t w, uint32_t js) {
    const uint64_t lo = l < w ? l : w, hi = l < w ? w : l;
    const uint64_t z = splitmix64(((lo << 32) | hi) ^ d.seed);
    const uint64_t y = (z - js) * d.fm.qinv;
    const uint32_t r_hi = __funnelshift_r((uint32_t)(y >> 32), (uint32_t)y, d.fm.k);
    return r_hi <= (uint32_t)(d.fm.lim >> 32);
}

// With several hash groups (kColWords), a wedge (s, w), (l, w) can count only for a group k whose
// colour js_k = h_k(s, w) names a kept processor and equals h_k(l, w).  The word cw holds every js_k
// (read from s's entry); the groups are tried in order and the first that agrees decides, so an
// entry that counts for no processor costs one hash per group and no probe of l's table.
__device__ __forceinline__ bool words_may_count(const StreamDev& d, uint32_t l, uint32_t w, uint32_t cw) {
    const uint64_t lo = l < w ? l : w, hi = l < w ? w : l;
    const uint64_t key = (lo << 32) | hi;
    uint64_t sk = group_seed(d.seed, d.kbeg);
    for (uint32_t k = d.kbeg; k < d.kend; ++k, sk += kGoldenGamma) {
        const uint32_t js = (cw >> (k * d.cbits)) & d.cmask;
        uint32_t i;
        if (processor_of(d, k, js, i) && mod_equals_in_range(splitmix64(key ^ sk), js, d.fm)) return true;
    }
    return false;
}

// The scans' superset form of words_may_count (as colour_may_match is of wedge_may_count): every
// group of this state is tested, each with the high words of its divisibility test, and the results
// are combined with | (no early exit, so the lanes of a warp stay together).  Groups whose colour
// js_k no processor keeps may pass too; count_wedge decides every queued wedge exactly.
__device__ __forceinline__ bool words_may_match(const StreamDev& d, uint32_t l, uint32_t w, uint32_t cw) {
    const uint64_t lo = l < w ? l : w, hi = l < w ? w : l;
    const uint64_t key = (lo << 32) | hi;
    const uint32_t lim_hi = (uint32_t)(d.fm.lim >> 32);
    uint64_t sk = group_seed(d.seed, d.kbeg);
    bool any = false;
    for (uint32_t k = d.kbeg; k < d.kend; ++k, sk += kGoldenGamma) {
        const uint32_t js = (cw >> (k * d.cbits)) & d.cmask;
        const uint64_t y = (splitmix64(key ^ sk) - js) * d.fm.qinv;
        any |= __funnelshift_r((uint32_t)(y >> 32), (uint32_t)y, d.fm.k) <= lim_hi;
    }
    return any;
}

// log2 of the table capacity for cnt entries: capacity = max(4, nextpow2(2*cnt)); 0 when empty.
__host__ __device__ __forceinline__ uint32_t table_lg(uint32_t cnt) {
    if (cnt == 0) return 0;
    uint32_t x = 2u * cnt - 1u;  // ceil(log2(2*cnt)) = bit length of (2*cnt - 1)
#ifdef __CUDA_ARCH__
    uint32_t lg = 32u - __clz(x);
#else
    uint32_t lg = 32u - (uint32_t)__builtin_clz(x);
#endif
    return lg < 2u ? 2u : lg;
}

// A node's block in the pool: its hash table (2^lg slots, probed by neighbour id) followed by its
// entry list (list_slots(lg) slots, the same entries packed in insertion order, scanned when the
// node is the smaller endpoint) and, with kColWords, the entries' colour words (one uint32 per list
// slot, word_slots(lg) slots).  Every part is a multiple of 4 slots (32 bytes).
__host__ __device__ __forceinline__ uint32_t list_slots(uint32_t lg) { return lg >= 3u ? (1u << (lg - 1u)) : 4u; }
__host__ __device__ __forceinline__ uint32_t word_slots(uint32_t lg) { return lg >= 4u ? (1u << (lg - 2u)) : 4u; }
__host__ __device__ __forceinline__ uint32_t block_quads(uint32_t lg, bool words) {
    return ((1u << lg) + list_slots(lg) + (words ? word_slots(lg) : 0u)) >> 2;
}

// k_intersect work class of an edge whose smaller endpoint holds cnt entries: tiles of 4, 8, 16, 32
// lanes (one entry per lane) up to tile_max entries, then a warp per edge for up to 256 entries and
// for more.
__host__ __device__ __forceinline__ int bin_of_cnt(uint32_t cnt, uint32_t tile_max) {
    if (cnt > tile_max) return cnt <= 256u ? 4 : 5;
    return cnt <= 4u ? 0 : cnt <= 8u ? 1 : cnt <= 16u ? 2 : 3;
}

// Home slot of neighbour w in a table of 2^lg slots: the first slot of a 4-slot (32-byte) bucket
// chosen by Fibonacci hashing.  Probing is linear from there, so a lookup reads whole sectors.
__device__ __forceinline__ uint32_t home_slot(uint32_t w, uint32_t lg) {
    return ((w * 0x9E3779B1u) >> (32u - lg)) & ~3u;
}

// Word offsets, from the start of a table of 2^lg slots, of slot h's neighbour id and of its stream
// index.  Interleaved (`inter`): bucket h / 4 occupies words 8 (h / 4) .. 8 (h / 4) + 7, ids first.
// Split: ids in words 0 .. 2^lg - 1, indices in the next 2^lg words.  key_quad: the 16-byte quad that
// holds the four ids of the bucket that starts at slot h (h a multiple of 4).
__host__ __device__ __forceinline__ uint32_t key_word(uint32_t h, bool inter) {
    return inter ? (((h >> 2) << 3) | (h & 3u)) : h;
}
__host__ __device__ __forceinline__ uint32_t eidx_word(uint32_t h, uint32_t lg, bool inter) {
    return inter ? key_word(h, true) + 4u : (1u << lg) + h;
}
__host__ __device__ __forceinline__ uint32_t key_quad(uint32_t h, bool inter) { return inter ? h >> 1 : h >> 2; }

__device__ __forceinline__ unsigned long long pack_slot(uint32_t nbr, uint32_t eidx) {
    return ((unsigned long long)eidx << 32) | nbr;
}

// Warp-aggregated atomicAdd: every active lane of the full warp calls it with its own
// increment; returns the lane's exclusive offset from a single atomic per warp.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* ctr, unsigned long long inc) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long incl = inc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (unsigned)o) incl += y;
    }
    unsigned long long total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - inc;
}

}  // namespace rept
