// Kernels of one REPT batch, in launch order:
//   k_classify  colour every edge (all hash groups), find the edges some
//               processor keeps, count new table entries per node, list the
//               touched nodes                                  (Alg. 1 "if h(u,v)==i")
//   k_plan      size the touched nodes' tables for their new entry counts and
//               reserve pool space for the ones that must be re-allocated
//   k_commit    move re-allocated tables (rehash), publish the new counts
//   k_insert    insert each kept edge (nbr, stream index) into both
//               endpoints' tables                              (Alg. 1 E^(i) <- E^(i) + {(u,v)})
//   k_sort_scan, k_sort_scatter
//               order the edges that can close wedges into work classes by
//               their smaller endpoint's entry count, grouped by the larger
//               endpoint
//   k_intersect for every edge t = (u, v): walk the smaller endpoint's list,
//               look up the larger endpoint's table (for streams that store
//               colours, only for entries whose colours may agree), and count
//               the wedges whose two edges both arrived before t and carry
//               the same kept colour; tally tau^(i), tau_u, tau_v, tau_w
//                                                               (Alg. 1 UpdateTriangleCNT)
// Counting after inserting is exact because every entry carries its stream
// index and k_intersect only accepts entries with index < t: the state seen by
// edge t is exactly the sequential algorithm's state before t.
#pragma once

#include <type_traits>

#include "rept_common.cuh"

namespace rept {
// Internal linkage: every translation unit of the library that launches these kernels gets its own copy.
namespace {

// A node's table of 2^lg slots at pool slot `base` holds 2^lg neighbour ids (keys; probed a 4-key,
// 16-byte bucket at a time) and their stream indices, interleaved per bucket or split (key_word,
// eidx_word; `inter`).  Insert (nbr, eidx): claim a key slot with a 32-bit CAS, then store the index
// (in the same sector when interleaved).
// Returns false only if the table has no empty slot left (impossible while cnt <= capacity / 2).
// Lookups read whole 4-key buckets, so where a key sits inside its bucket does not matter: an insert
// tries the slots of a bucket starting from one chosen by other bits of the key, so that keys sharing
// a home bucket seldom contend for the same slot, and moves to the next bucket only when all four are
// taken.
// The slot of its home bucket that an insert of nbr tries first.
__device__ __forceinline__ uint32_t first_slot(uint32_t nbr, uint32_t lg) {
    return home_slot(nbr, lg) + ((nbr * 0x85EBCA6Bu) >> 30);
}

// `tried_first`: the caller's CAS on first_slot(nbr, lg) failed already.
__device__ __forceinline__ bool table_insert(uint2* pool, unsigned long long base, uint32_t lg, uint32_t nbr,
                                             uint32_t eidx, bool inter, bool tried_first = false) {
    uint32_t* keys = reinterpret_cast<uint32_t*>(pool + base);
    const uint32_t mask = (1u << lg) - 1u;
    const uint32_t start = (nbr * 0x85EBCA6Bu) >> 30;
    uint32_t b = home_slot(nbr, lg);
    for (uint32_t probe = 0; probe <= mask; probe += 4u) {
#pragma unroll
        for (uint32_t i = 0; i < 4u; ++i) {
            if (tried_first && probe == 0u && i == 0u) continue;
            const uint32_t h = b + ((start + i) & 3u);
            if (atomicCAS(keys + key_word(h, inter), kEmptyId, nbr) == kEmptyId) {
                keys[eidx_word(h, lg, inter)] = eidx;
                return true;
            }
        }
        b = (b + 4u) & mask;
    }
    return false;
}

__device__ __forceinline__ void k_classify_body(const StreamDev& d, const BatchDev& b, const Grid g) {
    // the previous batch's work list is consumed: clear the counting-sort histogram
    for (uint32_t i = g.bx * blockDim.x + threadIdx.x; i < kSortBuckets; i += g.nbx * blockDim.x)
        d.hist[i] = 0u;
    if (g.bx == 0 && threadIdx.x < kBins) d.ctrl->bin_next[threadIdx.x] = 0ull;
    if (g.bx == 0 && threadIdx.x == 0) d.ctrl->n_pairs = 0ull;
    if (d.ctrl->status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)g.nbx * blockDim.x;
    for (unsigned long long base = (unsigned long long)g.bx * blockDim.x + threadIdx.x - lane; base < b.n;
         base += stride) {
        const unsigned long long e = base + lane;
        const bool valid = e < b.n;
        uint32_t u = 0, v = 0;
        if (valid) { u = b.src[e]; v = b.dst[e]; }
        const bool in_range = u < d.n_nodes && v < d.n_nodes;
        if (valid && !in_range) atomicOr(&d.ctrl->status, kStRange);
        const bool kept = valid && in_range && u != v && kept_by_any(d, u, v);
        bool first_u = false, first_v = false;
        if (kept) {
            first_u = atomicAdd(&d.cnt_add[u], 1u) == 0u;
            first_v = atomicAdd(&d.cnt_add[v], 1u) == 0u;
        }
        unsigned long long o = warp_reserve(&d.ctrl->n_touched, (unsigned)first_u + (unsigned)first_v);
        if (first_u) d.touched[o++] = u;
        if (first_v) d.touched[o] = v;
    }
}

__device__ __forceinline__ void k_plan_body(const StreamDev& d, const Grid g) {
    if (d.ctrl->status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long n_t = d.ctrl->n_touched;
    const unsigned long long stride = (unsigned long long)g.nbx * blockDim.x;
    for (unsigned long long base = (unsigned long long)g.bx * blockDim.x + threadIdx.x - lane; base < n_t;
         base += stride) {
        const unsigned long long i = base + lane;
        const bool valid = i < n_t;
        unsigned long long need = 0;
        if (valid) {
            const uint32_t x = d.touched[i];
            const uint32_t cnt = d.meta[x].y, add = d.cnt_add[x];
            d.cnt_add[x] = 0u;     // zero again for the next batch
            d.meta[x].z = add;     // the count travels with the node's record from here on
            const uint32_t lg_old = table_lg(cnt), lg_new = table_lg(cnt + add);
            if (lg_new != lg_old) need = block_quads(lg_new, has_words(d));
        }
        const unsigned long long rel = warp_reserve(&d.ctrl->need_quads, need);
        if (valid) d.grow_rel[i] = need ? (uint32_t)rel : kNoGrow;
    }
}

// REPT_DEBUG_BOUNDS: the block of 2^lg table slots and its list at `off_quads` lies inside the pool.
__device__ __forceinline__ bool block_fits(const StreamDev& d, unsigned site, unsigned long long off_quads,
                                          uint32_t lg) {
    return REPT_CHECK(d.ctrl, site, 4ull * (off_quads + block_quads(lg, has_words(d))) - 1ull, 4ull * d.pool_quads);
}

// The colour words (kColWords) of the list of a block at `off_quads` with a table of 2^lg slots.
__device__ __forceinline__ uint32_t* list_words(uint2* pool, unsigned long long off_quads, uint32_t lg) {
    return reinterpret_cast<uint32_t*>(pool + 4ull * off_quads + (1ull << lg) + list_slots(lg));
}

// Move node x's entries (list of cnt_old entries at old_off) into its new block at new_off: copy the
// list (and, with `words`, the colour words) and insert each entry's id (`mask` takes it out of the
// entry) into the new table.  Lanes `rank` of `width` share the work.
__device__ __forceinline__ bool move_block(uint2* pool, uint32_t mask, bool words, bool inter, uint32_t old_off,
                                           uint32_t cnt_old, unsigned long long new_off, uint32_t lg_new, uint32_t rank,
                                           uint32_t width) {
    const uint32_t lg_old = table_lg(cnt_old);
    const unsigned long long old_at = 4ull * old_off + (1ull << lg_old);
    const unsigned long long new_at = 4ull * new_off + (1ull << lg_new);
    const uint2* old_list = pool + old_at;
    uint2* new_list = pool + new_at;
    bool ok = true;
    for (uint32_t j = rank; j < cnt_old; j += width) {
        const uint2 e = old_list[j];
        new_list[j] = e;
        if (words) list_words(pool, new_off, lg_new)[j] = list_words(pool, old_off, lg_old)[j];
        ok &= table_insert(pool, 4ull * new_off, lg_new, e.x & mask, e.y, inter);
    }
    return ok;
}

// Set every key of the new table of 2^lg slots at `off_quads` to empty (lanes `rank` of `width`).  The
// pool is not cleared between streams: a block's table gets its empty keys when the block is handed
// out, from here or from the shared-memory builds, which write the whole table.  (Stream indices are
// read only beside a matching key, so they need no initial value.)
__device__ __forceinline__ void init_table_keys(uint2* pool, unsigned long long off_quads, uint32_t lg, bool inter,
                                                uint32_t rank, uint32_t width) {
    uint4* quads = reinterpret_cast<uint4*>(pool + 4ull * off_quads);
    const uint4 empty = make_uint4(kEmptyId, kEmptyId, kEmptyId, kEmptyId);
    for (uint32_t b = rank; b < (1u << lg) / 4u; b += width) quads[inter ? 2u * b : b] = empty;
}

// New tables of at most kMoveSlots slots are rebuilt in shared memory by a warp (k_rehash_big), those
// of at most kBlockMoveSlots by a thread block (k_rehash_huge); larger ones are built in place.
constexpr uint32_t kInlineSlots = 32;  // k_commit's own moves (one thread each)
constexpr uint32_t kMoveSlots = 512;
constexpr uint32_t kBlockMoveSlots = 4096;

// Publish the new entry counts of the touched nodes and move the blocks that were re-allocated.
// One thread per touched node moves a block of at most 8 entries into a new table of at most
// kInlineSlots slots; other blocks are left to k_rehash_big (a warp each, new tables of at most
// kMoveSlots slots) or k_rehash_huge (a thread block each).  meta[x].z
// keeps the batch's new-entry count for k_insert, which counts it back down to zero; a batch that is not
// applied clears it here.
__device__ __forceinline__ void k_commit_body(const StreamDev& d, const Grid g) {
    const unsigned status = d.ctrl->status;
    const unsigned long long n_t = d.ctrl->n_touched;
    const unsigned long long need = d.ctrl->need_quads, top = d.ctrl->pool_top;
    const bool bad = status != 0u || top + need > d.pool_quads;
    if (status == 0u && bad && g.bx == 0 && threadIdx.x == 0) atomicOr(&d.ctrl->status, kStCapacity);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)g.nbx * blockDim.x;
    for (unsigned long long base = (unsigned long long)g.bx * blockDim.x + threadIdx.x - lane; base < n_t;
         base += stride) {
        const unsigned long long i = base + lane;
        bool defer = false, huge = false;
        if (i < n_t) {
            const uint32_t x = d.touched[i];
            if (bad) {
                d.meta[x].z = 0u;
            } else {
                const uint4 m = d.meta[x];
                const uint32_t cnt_new = m.y + m.z;
                const uint32_t rel = d.grow_rel[i];
                if (rel == kNoGrow) {
                    d.meta[x].y = cnt_new;
                } else if (m.y > 8u || (1u << table_lg(cnt_new)) > kInlineSlots) {
                    defer = (1u << table_lg(cnt_new)) <= kMoveSlots;
                    huge = !defer;
                } else {
                    const unsigned long long new_off = top + rel;
                    const bool fits = block_fits(d, 10, m.x, table_lg(m.y)) &&
                                      block_fits(d, 11, new_off, table_lg(cnt_new));
                    if (fits) init_table_keys(d.pool, new_off, table_lg(cnt_new), tables_interleaved(d), 0u, 1u);
                    if (fits && !move_block(d.pool, id_mask(d), has_words(d), tables_interleaved(d), m.x, m.y, new_off,
                                            table_lg(cnt_new), 0u, 1u))
                        atomicOr(&d.ctrl->status, kStInternal);
                    d.meta[x] = make_uint4((uint32_t)new_off, cnt_new, m.z, 0u);
                }
            }
        }
        const unsigned long long o = warp_reserve(&d.ctrl->n_big, defer ? 1ull : 0ull);
        if (defer) d.big[o] = (uint32_t)i;
        const unsigned long long h = warp_reserve(&d.ctrl->n_huge, huge ? 1ull : 0ull);
        if (huge) d.big[d.big_cap - 1 - h] = (uint32_t)i;
    }
}

// move_block with the new table built in shared memory (keys and stream indices of 2^lg_new slots,
// the same placement rule as table_insert) and then written out with coalesced stores, by the lanes
// `rank` of `width` of one warp (BLOCK = false) or of one thread block (BLOCK = true).  The new block
// is the caller's alone until the batch's inserts run.
template <bool BLOCK, bool INTER>
__device__ __forceinline__ bool move_block_smem(uint2* pool, uint32_t id_bits, bool words, uint32_t old_off,
                                                uint32_t cnt_old, unsigned long long new_off, uint32_t lg_new,
                                                uint32_t* s_keys, uint32_t* s_eidx, uint32_t rank, uint32_t width) {
    auto sync = [] {
        if (BLOCK) __syncthreads();
        else __syncwarp();
    };
    const uint32_t cap = 1u << lg_new, mask = cap - 1u;
    for (uint32_t q = rank; q < cap; q += width) {
        s_keys[q] = kEmptyId;
        s_eidx[q] = kEmptyId;
    }
    sync();
    const uint32_t lg_old = table_lg(cnt_old);
    const unsigned long long old_at = 4ull * old_off + (1ull << lg_old);
    const unsigned long long new_at = 4ull * new_off + cap;
    bool ok = true;
    for (uint32_t j = rank; j < cnt_old; j += width) {
        const uint2 e = pool[old_at + j];
        pool[new_at + j] = e;
        if (words) list_words(pool, new_off, lg_new)[j] = list_words(pool, old_off, lg_old)[j];
        const uint32_t key = e.x & id_bits;
        const uint32_t start = (key * 0x85EBCA6Bu) >> 30;
        uint32_t b = home_slot(key, lg_new);
        bool placed = false;
        for (uint32_t probe = 0; probe <= mask && !placed; probe += 4u) {
            for (uint32_t i = 0; i < 4u && !placed; ++i) {
                const uint32_t h = b + ((start + i) & 3u);
                if (atomicCAS(&s_keys[h], kEmptyId, key) == kEmptyId) {
                    s_eidx[h] = e.y;
                    placed = true;
                }
            }
            b = (b + 4u) & mask;
        }
        ok &= placed;
    }
    sync();
    uint32_t* words_out = reinterpret_cast<uint32_t*>(pool + 4ull * new_off);
    if (INTER) {  // word q of the table: bucket q / 8, an id (q % 8 < 4) or a stream index
        for (uint32_t q = rank; q < 2u * cap; q += width) {
            const uint32_t h = ((q >> 3) << 2) | (q & 3u);
            words_out[q] = (q & 4u) ? s_eidx[h] : s_keys[h];
        }
    } else {
        for (uint32_t q = rank; q < cap; q += width) {
            words_out[q] = s_keys[q];
            words_out[cap + q] = s_eidx[q];
        }
    }
    return ok;
}

// Move the blocks listed by k_commit whose new table has at most kMoveSlots slots: one warp per node.
// `smem`: kMoveSmemWords words of shared memory (a key and a stream-index table of kMoveSlots slots
// for each of the block's 8 warps).
constexpr uint32_t kMoveSmemWords = 2u * 8u * kMoveSlots;
static_assert(kMoveSmemWords >= 2u * kBlockMoveSlots, "the block move uses the same shared memory");
__device__ __forceinline__ void k_rehash_big_body(const StreamDev& d, const Grid g, uint32_t* smem) {
    const unsigned long long n_big = d.ctrl->n_big, top = d.ctrl->pool_top;
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned long long warps = ((unsigned long long)g.nbx * blockDim.x) >> 5;
    for (unsigned long long k = ((unsigned long long)g.bx * blockDim.x + threadIdx.x) >> 5; k < n_big;
         k += warps) {
        const uint32_t i = d.big[k];
        const uint32_t x = d.touched[i];
        const uint4 m = d.meta[x];
        const uint32_t cnt_new = m.y + m.z;
        const unsigned long long new_off = top + d.grow_rel[i];
        const bool fits = block_fits(d, 10, m.x, table_lg(m.y)) && block_fits(d, 11, new_off, table_lg(cnt_new));
        const uint32_t lg_new = table_lg(cnt_new);
        bool ok = true;
        if (fits && (1u << lg_new) <= kMoveSlots && REPT_CHECK(d.ctrl, 14, wid, 8u))
            ok = tables_interleaved(d)
                     ? move_block_smem<false, true>(d.pool, id_mask(d), has_words(d), m.x, m.y, new_off, lg_new,
                                                    smem + wid * kMoveSlots, smem + (8u + wid) * kMoveSlots, lane, 32u)
                     : move_block_smem<false, false>(d.pool, id_mask(d), has_words(d), m.x, m.y, new_off, lg_new,
                                                     smem + wid * kMoveSlots, smem + (8u + wid) * kMoveSlots, lane, 32u);
        else if (fits) {
            init_table_keys(d.pool, new_off, lg_new, tables_interleaved(d), lane, 32u);
            __syncwarp();
            ok = move_block(d.pool, id_mask(d), has_words(d), tables_interleaved(d), m.x, m.y, new_off, lg_new, lane, 32u);
        }
        if (!ok) atomicOr(&d.ctrl->status, kStInternal);
        __syncwarp();
        if (lane == 0) d.meta[x] = make_uint4((uint32_t)new_off, cnt_new, m.z, 0u);
    }
}

// Move the blocks listed by k_commit whose new table has more than kMoveSlots slots: thread blocks
// claim one node at a time, and build tables of at most kBlockMoveSlots slots in shared memory.
// `smem`: kMoveSmemWords words of shared memory (a key and a stream-index table of kBlockMoveSlots slots).
__device__ __forceinline__ void k_rehash_huge_body(const StreamDev& d, const Grid g, uint32_t* smem) {
    uint32_t* s_keys = smem;
    uint32_t* s_eidx = smem + kBlockMoveSlots;
    __shared__ unsigned long long s_k;
    __shared__ int s_bad;
    const unsigned long long n_huge = d.ctrl->n_huge, top = d.ctrl->pool_top;
    for (;;) {
        if (threadIdx.x == 0) {
            s_k = atomicAdd(&d.ctrl->huge_next, 1ull);
            s_bad = 0;
        }
        __syncthreads();
        const unsigned long long k = s_k;
        if (k >= n_huge) break;
        const uint32_t i = d.big[d.big_cap - 1 - k];
        const uint32_t x = d.touched[i];
        const uint4 m = d.meta[x];
        const uint32_t cnt_new = m.y + m.z;
        const unsigned long long new_off = top + d.grow_rel[i];
        const bool fits = block_fits(d, 10, m.x, table_lg(m.y)) && block_fits(d, 11, new_off, table_lg(cnt_new));
        const uint32_t lg_new = table_lg(cnt_new);
        bool ok = true;
        if (fits && (1u << lg_new) <= kBlockMoveSlots)  // uniform over the block
            ok = tables_interleaved(d)
                     ? move_block_smem<true, true>(d.pool, id_mask(d), has_words(d), m.x, m.y, new_off, lg_new, s_keys,
                                                   s_eidx, threadIdx.x, blockDim.x)
                     : move_block_smem<true, false>(d.pool, id_mask(d), has_words(d), m.x, m.y, new_off, lg_new, s_keys,
                                                    s_eidx, threadIdx.x, blockDim.x);
        else if (fits) {  // (uniform over the block) built in place: empty keys first
            init_table_keys(d.pool, new_off, lg_new, tables_interleaved(d), threadIdx.x, blockDim.x);
            __syncthreads();
            ok = move_block(d.pool, id_mask(d), has_words(d), tables_interleaved(d), m.x, m.y, new_off, lg_new,
                            threadIdx.x, blockDim.x);
        }
        if (!ok) s_bad = 1;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_bad) atomicOr(&d.ctrl->status, kStInternal);
            d.meta[x] = make_uint4((uint32_t)new_off, cnt_new, m.z, 0u);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void k_insert_body(const StreamDev& d, const BatchDev& b, const Grid g) {
    Ctrl* ct = d.ctrl;
    const unsigned status = ct->status;
    if (g.bx == 0 && threadIdx.x == 0) {
        // the batch's table space is now in use; reset the per-batch counters
        if (status == 0u) ct->pool_top += ct->need_quads;
        ct->need_quads = 0;
        ct->n_touched = 0;
        ct->n_big = 0;
        ct->n_huge = 0;
        ct->huge_next = 0;
    }
    if (status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)g.nbx * blockDim.x;
    unsigned long long n_loops = 0, n_kept = 0;  // this lane's tallies, added once per warp at the end
    for (unsigned long long base = (unsigned long long)g.bx * blockDim.x + threadIdx.x - lane; base < b.n;
         base += stride) {
        const unsigned long long e = base + lane;
        const bool valid = e < b.n;
        uint32_t u = 0, v = 0;
        if (valid) { u = b.src[e]; v = b.dst[e]; }
        const bool loop = valid && u == v;
        // with stored colours the edge's colours decide whether it is kept and ride with its list
        // entries (in the entries' top bits for one hash group, in a word per entry for several): the
        // same hashes serve both
        uint32_t cj = 0u, cw = 0u;
        bool kept;
        if (d.colours == kColInEntry) {
            uint32_t i;
            const uint32_t j = colour_of(u, v, d.seed, d.fm);
            kept = valid && u != v && processor_of(d, 0u, j, i);
            cj = j << kIdBits;
        } else if (has_words(d)) {
            bool any = false;
            uint64_t sk = group_seed(d.seed, d.kbeg);
            for (uint32_t k = d.kbeg; k < d.kend; ++k, sk += kGoldenGamma) {
                uint32_t i;
                const uint32_t j = colour_of(u, v, sk, d.fm);
                cw |= j << (k * d.cbits);
                any |= processor_of(d, k, j, i);
            }
            kept = valid && u != v && any;
        } else {
            kept = valid && u != v && kept_by_any(d, u, v);
        }
        uint32_t key = kNoKey;
        WorkItem it{};
        if (valid && u != v) {
            // list positions: meta[x].z counts this batch's entries of x back down to zero.  The two
            // counters, the two records and then the first CAS of each table insert are issued
            // before any result is used, so that their round trips overlap.
            uint32_t zu = 0u, zv = 0u;
            if (kept) {
                zu = atomicSub(&d.meta[u].z, 1u);
                zv = atomicSub(&d.meta[v].z, 1u);
            }
            const uint4 mu = d.meta[u], mv = d.meta[v];
            if (kept && block_fits(d, 1, mu.x, table_lg(mu.y)) && block_fits(d, 1, mv.x, table_lg(mv.y))) {
                const uint32_t t = (uint32_t)(b.t0 + e);
                const uint32_t lu = table_lg(mu.y), lv = table_lg(mv.y);
                uint32_t* tu = reinterpret_cast<uint32_t*>(d.pool + 4ull * mu.x);
                uint32_t* tv = reinterpret_cast<uint32_t*>(d.pool + 4ull * mv.x);
                const bool inter = tables_interleaved(d);
                const uint32_t hu = first_slot(v, lu), hv = first_slot(u, lv);
                const uint32_t cu = atomicCAS(tu + key_word(hu, inter), kEmptyId, v);
                const uint32_t cv = atomicCAS(tv + key_word(hv, inter), kEmptyId, u);
                bool ok = true;
                if (cu == kEmptyId) tu[eidx_word(hu, lu, inter)] = t;
                else ok = table_insert(d.pool, 4ull * mu.x, lu, v, t, inter, true);
                if (cv == kEmptyId) tv[eidx_word(hv, lv, inter)] = t;
                else ok &= table_insert(d.pool, 4ull * mv.x, lv, u, t, inter, true);
                if (!ok) atomicOr(&ct->status, kStInternal);
                const uint32_t pu = mu.y - zu, pv = mv.y - zv;
                if (REPT_CHECK(ct, 2, pu, list_slots(lu)) && REPT_CHECK(ct, 2, pv, list_slots(lv))) {
                    d.pool[4ull * mu.x + (1ull << lu) + pu] = make_uint2(v | cj, t);
                    d.pool[4ull * mv.x + (1ull << lv) + pv] = make_uint2(u | cj, t);
                    if (has_words(d)) {
                        list_words(d.pool, mu.x, lu)[pu] = cw;
                        list_words(d.pool, mv.x, lv)[pv] = cw;
                    }
                }
                if (d.edge_ends) d.edge_ends[t] = make_uint2(u, v);
            }
            // an edge can close wedges only if both endpoints have stored edges
            if (mu.y != 0u && mv.y != 0u) {
                const bool u_small = mu.y <= mv.y;
                const uint4 ms = u_small ? mu : mv, ml = u_small ? mv : mu;
                it.s = u_small ? u : v;
                it.l = u_small ? v : u;
                it.off_s = ms.x;
                it.off_l = ml.x;
                it.t = (uint32_t)(b.t0 + e);
                it.lgs = table_lg(ms.y) | (table_lg(ml.y) << 8);
                it.cnt_s = ms.y;
                key = (uint32_t)bin_of_cnt(ms.y, d.tile_max) * kKeyBuckets + ((it.l * 0x9E3779B1u) >> (32 - kKeyBits));
            }
        }
        it.key = key;
        if (valid) d.rec[e] = it;
        {
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
            if (key != kNoKey && lane == (unsigned)(__ffs(peers) - 1))
                atomicAdd(&d.hist[key], (uint32_t)__popc(peers));
        }
        n_loops += loop ? 1ull : 0ull;
        n_kept += kept ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_loops += __shfl_down_sync(0xFFFFFFFFu, n_loops, o);
        n_kept += __shfl_down_sync(0xFFFFFFFFu, n_kept, o);
    }
    if (lane == 0) {
        if (n_loops) atomicAdd(&ct->self_loops, n_loops);
        if (n_kept) atomicAdd(&ct->stored, n_kept);
    }
}

// Exclusive scan of the counting-sort histogram (one block of 256 or 1024 threads): counts become
// the first position of each key, and the class boundaries are recorded.  The counters are scanned
// in chunks of 4 * blockDim, thread t holding counters 4t..4t+3 of a chunk (one coalesced 16-byte
// load); both block sizes divide the class size.
__device__ __forceinline__ void k_sort_scan_body(const StreamDev& d, const Grid g) {
    const uint32_t kChunk = 4u * blockDim.x;
    static_assert(kKeyBuckets % 4096u == 0 && kSortBuckets % 4096u == 0, "scan chunks");
    (void)g;
    __shared__ uint32_t warp_sum[33];
    if (d.ctrl->status) return;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < kSortBuckets; base += kChunk) {
        const uint4 v = reinterpret_cast<const uint4*>(d.hist + base)[tid];
        const uint32_t sum = v.x + v.y + v.z + v.w;
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t w = lane < (blockDim.x >> 5) ? warp_sum[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= (uint32_t)o) wi += y;
            }
            warp_sum[lane] = wi - w;
            if (lane == 31) warp_sum[32] = wi;  // the chunk's total
        }
        __syncthreads();
        uint32_t run = carry + warp_sum[wid] + incl - sum;
        const uint32_t key = base + 4u * tid;
        if (key % kKeyBuckets == 0u) d.ctrl->bin_start[key / kKeyBuckets] = run;
        uint4 o;
        o.x = run;
        run += v.x;
        o.y = run;
        run += v.y;
        o.z = run;
        run += v.z;
        o.w = run;
        reinterpret_cast<uint4*>(d.hist + base)[tid] = o;
        carry += warp_sum[32];
        __syncthreads();  // warp_sum is reused by the next chunk
    }
    if (tid == 0) {  // totals (thread 0 wrote every class start): carry is the number of items
        unsigned long long prev = carry;
        for (int c = kBins - 1; c >= 0; --c) {
            d.ctrl->bin_count[c] = prev - d.ctrl->bin_start[c];
            prev = d.ctrl->bin_start[c];
        }
    }
}

// Scatter each edge that can close a wedge to its place in the sorted work list.
__device__ __forceinline__ void k_sort_scatter_body(const StreamDev& d, const BatchDev& b, const Grid g) {
    if (d.ctrl->status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)g.nbx * blockDim.x;
    for (unsigned long long base = (unsigned long long)g.bx * blockDim.x + threadIdx.x - lane; base < b.n;
         base += stride) {
        const unsigned long long e = base + lane;
        WorkItem it{};
        it.key = kNoKey;
        if (e < b.n) it = d.rec[e];
        const uint32_t key = it.key;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t pos = 0;
        if (key != kNoKey && (int)lane == leader) pos = atomicAdd(&d.hist[key], (uint32_t)__popc(peers));
        pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
        if (key != kNoKey) d.srec[pos + __popc(peers & ((1u << lane) - 1u))] = it;
    }
}

// Look neighbour w up in the table of 2^lg slots at `base` (lg >= 2): read 4-key buckets from w's
// home bucket on until w or an empty key shows up.  Returns w's stream index, or kEmptyId when w is
// absent; `slots` receives the number of keys read.
__device__ __forceinline__ uint32_t table_find(const uint2* __restrict__ pool, unsigned long long base, uint32_t lg,
                                               uint32_t w, uint32_t& slots, bool inter) {
    const uint32_t mask = (1u << lg) - 1u;
    const uint32_t* keys = reinterpret_cast<const uint32_t*>(pool + base);
    const uint4* buckets = reinterpret_cast<const uint4*>(keys);
    uint32_t h = home_slot(w, lg);
    for (uint32_t probe = 0; probe <= mask; probe += 4u) {  // h: the first slot of a bucket
        const uint4 k4 = buckets[key_quad(h, inter)];
        slots = probe + 4u;
        int at = -1;
        if (k4.x == w) at = 0;
        else if (k4.y == w) at = 1;
        else if (k4.z == w) at = 2;
        else if (k4.w == w) at = 3;
        if (at >= 0) return keys[eidx_word(h + (uint32_t)at, lg, inter)];
        if (k4.x == kEmptyId || k4.y == kEmptyId || k4.z == kEmptyId || k4.w == kEmptyId) return kEmptyId;
        h = (h + 4u) & mask;
    }
    return kEmptyId;
}

// REPT_FLAG_CHECK_DUPS: before the batch is applied, flag an edge that repeats an earlier stored
// edge (found in its endpoint's table) or another edge of the same batch (found in a set of the
// batch's edge keys, built in the work-record scratch, which is free at this point and was filled
// with ~0 by the host).  `mask` + 1 is the set's capacity, a power of two at least twice the batch.
__global__ void k_check_dups(StreamDev d, BatchDev b, unsigned long long mask) {
    if (d.ctrl->status) return;
    unsigned long long* set = reinterpret_cast<unsigned long long*>(d.rec);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    bool dup = false;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < b.n; e += stride) {
        const uint32_t u = b.src[e], v = b.dst[e];
        if (u == v || u >= d.n_nodes || v >= d.n_nodes) continue;
        const uint4 mu = d.meta[u];
        uint32_t ns;
        if (mu.y != 0u && table_find(d.pool, 4ull * mu.x, table_lg(mu.y), v, ns, tables_interleaved(d)) != kEmptyId) dup = true;
        const unsigned long long key = ((unsigned long long)(u < v ? u : v) << 32) | (u < v ? v : u);
        unsigned long long h = splitmix64(key) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const unsigned long long old = atomicCAS(set + h, ~0ull, key);
            if (old == ~0ull) break;
            if (old == key) { dup = true; break; }
            h = (h + 1u) & mask;
        }
    }
    if (dup) atomicOr(&d.ctrl->status, kStDuplicate);
}

// Work counters of k_intersect<true>, kept per lane in registers.
struct Work {
    unsigned long long entries = 0, slots = 0, probes = 0, pslots = 0, wedges = 0, counted = 0;
};

// Wedge (s, w), (l, w), both edges older than the arriving edge (s, l): count it for every hash group
// whose colour of the two edges agrees and names a kept processor, and add the number of such groups
// to tau_s, tau_l and tau_w (Algorithm 1's local updates, one wedge at a time).
// Algorithm 2's pair counters: one more closed wedge through stored edge t in group k this batch.
__device__ __forceinline__ void pair_event(const StreamDev& d, uint32_t t, uint32_t k) {
    const unsigned long long idx = (unsigned long long)t * d.groups + k;
    if (atomicAdd(&d.pair_evt[idx], 1u) == 0u) d.pair_list[atomicAdd(&d.ctrl->n_pairs, 1ull)] = (uint32_t)idx;
}

// MODE: the stream's colour storage (the kernel variant).  DIFF: decide each group's colour agreement
// from the two hash values' difference (same_colour: one remainder only when they agree), which pays
// where wedges are counted under several groups (streams without colours in their entries); streams
// with colours in their entries form both colours, which keeps their registers lower.  INTER: the
// stream's tables are interleaved (tables_interleaved), i.e. it stores colours.
template <int MODE>
__device__ __forceinline__ uint32_t count_wedge(const StreamDev& d, uint32_t s, uint32_t l, uint32_t w,
                                                unsigned long long* s_proc) {
    constexpr bool DIFF = MODE != (int)kColInEntry, INTER = MODE != (int)kColNone;
    if (!REPT_CHECK(d.ctrl, 9, max(w, max(s, l)), d.n_nodes)) return 0u;
    uint32_t found = 0, found2 = 0;
    uint32_t t_sw = kEmptyId, t_lw = kEmptyId;
    for (uint32_t k = d.kbeg; k < d.kend; ++k) {
        uint32_t js, i;
        bool agree;
        if (DIFF) {
            agree = same_colour(s, l, w, group_seed(d.seed, k), d.fm, js) && processor_of(d, k, js, i);
        } else {
            const uint64_t sk = group_seed(d.seed, k);
            js = colour_of(s, w, sk, d.fm);
            agree = processor_of(d, k, js, i) && colour_of(l, w, sk, d.fm) == js;
        }
        if (agree) {
            atomicAdd(&s_proc[i], 1ull);
            if (d.local2 && k >= d.c1) ++found2; else ++found;
            if (d.local_proc) {
                unsigned long long* lp = d.local_proc + (unsigned long long)i * d.n_nodes;
                atomicAdd(&lp[s], 1ull);
                atomicAdd(&lp[l], 1ull);
                atomicAdd(&lp[w], 1ull);
            }
            if (d.pair_tau) {
                if (t_sw == kEmptyId) {  // the wedge's two stream indices, looked up once
                    uint32_t ns;
                    const uint4 ms = d.meta[s], ml = d.meta[l];
                    t_sw = table_find(d.pool, 4ull * ms.x, table_lg(ms.y), w, ns, INTER);
                    t_lw = table_find(d.pool, 4ull * ml.x, table_lg(ml.y), w, ns, INTER);
                }
                pair_event(d, t_sw, k);
                pair_event(d, t_lw, k);
            }
        }
    }
    if (found) {
        atomicAdd(&d.local[w], (unsigned long long)found);
        atomicAdd(&d.local[s], (unsigned long long)found);
        atomicAdd(&d.local[l], (unsigned long long)found);
    }
    if (found2) {
        atomicAdd(&d.local2[w], (unsigned long long)found2);
        atomicAdd(&d.local2[s], (unsigned long long)found2);
        atomicAdd(&d.local2[l], (unsigned long long)found2);
    }
    return found + found2;
}

// Per-warp queue of closed wedges (s, l, w) in shared memory.  Wedges are pushed as the probes find
// them and coloured 32 at a time, so that the hash work runs on full warps.  `n` is warp-uniform.
constexpr int kMatchQ = 64;
struct MatchQueue {
    uint32_t* s;
    uint32_t* l;
    uint32_t* w;
    uint32_t n;
};

template <bool WORK, int MODE>
__device__ __forceinline__ void mq_flush(const StreamDev& d, MatchQueue& q, uint32_t take,
                                         unsigned long long* s_proc, Work& wk) {
    const unsigned lane = threadIdx.x & 31u;
    if (lane < take) {
        const uint32_t i = q.n - take + lane;
        const uint32_t f = count_wedge<MODE>(d, q.s[i], q.l[i], q.w[i], s_proc);
        if (WORK) wk.counted += f;
    }
    q.n -= take;
    __syncwarp();
}

template <bool WORK, int MODE>
__device__ __forceinline__ void mq_push(const StreamDev& d, MatchQueue& q, bool has, uint32_t s, uint32_t l,
                                        uint32_t w, unsigned long long* s_proc, Work& wk) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, has);
    if (!REPT_CHECK(d.ctrl, 13, q.n + __popc(mask), (unsigned long long)kMatchQ + 1ull)) return;
    if (has) {
        const uint32_t i = q.n + __popc(mask & ((1u << lane) - 1u));
        q.s[i] = s;
        q.l[i] = l;
        q.w[i] = w;
        if (WORK) ++wk.wedges;
    }
    q.n += __popc(mask);
    __syncwarp();
    if (q.n >= 32u) mq_flush<WORK, MODE>(d, q, 32u, s_proc, wk);
}

// Edges whose smaller endpoint has at most TILE entries: one tile of TILE lanes per edge, one list
// entry per lane.
template <int TILE, bool WORK, int MODE>
__device__ __forceinline__ void intersect_tile(const StreamDev& d, const WorkItem& x, bool valid,
                                               unsigned long long* s_proc, MatchQueue& mq, Work& wk) {
    const unsigned lane = threadIdx.x & 31u, j = lane & (TILE - 1);
    bool has = false;
    uint32_t w = 0;
    if (valid && j < x.cnt_s) {
        const unsigned long long at = 4ull * x.off_s + (1ull << (x.lgs & 0xFFu)) + j;
        const bool fits = REPT_CHECK(d.ctrl, 3, at, 4ull * d.pool_quads) && block_fits(d, 4, x.off_l, x.lgs >> 8);
        const uint2 es = fits ? d.pool[at] : make_uint2(kEmptyId, kEmptyId);
        if (WORK && j == 0) { wk.entries += x.cnt_s; wk.slots += x.cnt_s; }
        const uint32_t ws = es.x & id_mask(d);
        bool pass = es.y < x.t;
        if (d.colours == kColInEntry) pass = pass & wedge_may_count(d, x.l, ws, es.x >> kIdBits);
        else if (pass && has_words(d) && block_fits(d, 12, x.off_s, x.lgs & 0xFFu))
            pass = words_may_count(d, x.l, ws, list_words(d.pool, x.off_s, x.lgs & 0xFFu)[j]);
        if (pass) {
            uint32_t nslots = 0;
            // the single-stream kernels' streams: split tables exactly in the probe variant
            const uint32_t tl = table_find(d.pool, 4ull * x.off_l, x.lgs >> 8, ws, nslots, MODE != (int)kColNone);
            if (WORK) { ++wk.probes; wk.pslots += nslots; }
            has = tl < x.t;  // kEmptyId (absent) is never < t
            w = ws;
        }
    }
    mq_push<WORK, MODE>(d, mq, has, x.s, x.l, w, s_proc, wk);
}

// Edges whose smaller endpoint has more entries, streams without stored colours: a warp per edge.
// Each pass reads 128 entries of the smaller endpoint's list (two 16-byte loads per lane) and packs
// those older than the edge into the warp's shared-memory key queue.  The queue is probed with all 32
// lanes, kProbesPerLane keys per lane, whenever it holds a full round; a partial round waits for the
// next pass, so sparse candidates share round trips.
#ifndef REPT_GRAB_MID
#define REPT_GRAB_MID 4
#endif
#ifndef REPT_GRAB_HUB
#define REPT_GRAB_HUB 1
#endif
constexpr uint32_t kGrabMid = REPT_GRAB_MID;  // class 4 items (33..256 entries) claimed per atomic
constexpr uint32_t kGrabHub = REPT_GRAB_HUB;  // class 5 items (more entries) claimed per atomic
// The scan-first path's claims: its items cost less each (about 1/m of the entries are probed), so
// a warp takes more of them per atomic on the class cursor.
#ifndef REPT_SCAN_GRAB_MID
#define REPT_SCAN_GRAB_MID 8
#endif
#ifndef REPT_SCAN_GRAB_HUB
#define REPT_SCAN_GRAB_HUB 2
#endif
constexpr uint32_t kScanGrabMid = REPT_SCAN_GRAB_MID;
constexpr uint32_t kScanGrabHub = REPT_SCAN_GRAB_HUB;
constexpr int kQueue = 192;  // one partial round (< 64 keys) + 128 new keys

#ifndef REPT_PROBES_PER_LANE
#define REPT_PROBES_PER_LANE 2
#endif
constexpr int kProbesPerLane = REPT_PROBES_PER_LANE;  // probes each lane keeps in flight (warp path)
#ifndef REPT_WORDS_BLOCKS
#define REPT_WORDS_BLOCKS 6
#endif

// Streams without stored colours (MODE kColNone): every entry older than the edge is probed, so the
// path is probe-bound and runs with fewer registers and more warps per SM.  Streams that store
// colours take the scan-first path (drain_warp_bin_coloured) instead.
// `push(has, w)` (warp-collective) takes each probed key w and whether it closed a wedge.
template <bool WORK, int MODE, class Push>
__device__ __forceinline__ void intersect_warp(const StreamDev& d, const WorkItem& x, uint32_t* queue, Work& wk,
                                               Push&& push) {
    static_assert(MODE == (int)kColNone, "streams that store colours take the scan-first path");
    constexpr uint32_t kRound = 32u * kProbesPerLane;
    static_assert(kRound - 1 + 128 <= kQueue, "key queue too small");
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t lg_l = x.lgs >> 8, n_s = x.cnt_s;
    const unsigned long long base_l = 4ull * x.off_l;
    if (WORK && lane == 0) { wk.entries += n_s; wk.slots += n_s; }
    if (!(block_fits(d, 5, x.off_s, x.lgs & 0xFFu) && REPT_CHECK(d.ctrl, 6, n_s, list_slots(x.lgs & 0xFFu) + 1u) &&
          block_fits(d, 7, x.off_l, lg_l)))
        return;  // (uniform over the warp: x is)
    // the smaller endpoint's entry list (32-byte aligned), read 128 entries per pass, two per 16-byte
    // load
    const unsigned long long at_s = 4ull * x.off_s + (1ull << (x.lgs & 0xFFu));
    const uint4* list = reinterpret_cast<const uint4*>(d.pool + at_s);
    const uint32_t mask = id_mask(d);
    const uint32_t* keys_l = reinterpret_cast<const uint32_t*>(d.pool + base_l);
    const uint4* buckets_l = reinterpret_cast<const uint4*>(keys_l);
    const bool inter = false;  // these streams keep split tables
    const unsigned below = (1u << lane) - 1u;
    uint4 nq[2];
    auto load_pass = [&](uint32_t j0) {
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            const uint32_t jj = j0 + 64u * half + 2u * lane;
            nq[half] = make_uint4(kEmptyId, kEmptyId, kEmptyId, kEmptyId);
            if (jj < n_s) nq[half] = list[jj >> 1];
        }
    };
    uint32_t n_q = 0;

    for (uint32_t j0 = 0; j0 < n_s; j0 += 128u) {
        if (!REPT_CHECK(d.ctrl, 8, n_q, kRound)) break;
        load_pass(j0);
        const uint4 cq[2] = {nq[0], nq[1]};
#pragma unroll
        for (uint32_t half = 0; half < 2; ++half) {
            if (j0 + 64u * half >= n_s) break;  // an empty half (short lists, last passes): uniform skip
            const uint32_t jj = j0 + 64u * half + 2u * lane;
            const uint4 q = cq[half];
            const uint32_t w1 = q.x & mask, w2 = q.z & mask;
            const bool a1 = jj < n_s && q.y < x.t, a2 = jj + 1u < n_s && q.w < x.t;
            const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1), m2 = __ballot_sync(0xFFFFFFFFu, a2);
            if (a1) queue[n_q + __popc(m1 & below)] = w1;
            n_q += __popc(m1);
            if (a2) queue[n_q + __popc(m2 & below)] = w2;
            n_q += __popc(m2);
        }
        __syncwarp();
        const bool last = j0 + 128u >= n_s;
        // full rounds now, everything after the last pass: kProbesPerLane queued keys per lane, all
        // their home buckets loaded before any is examined, then the stream indices of the hits
        uint32_t k0 = 0;
        for (; last ? k0 < n_q : k0 + kRound <= n_q; k0 += kRound) {
            uint32_t w[kProbesPerLane], h[kProbesPerLane], r[kProbesPerLane];
            uint4 bk[kProbesPerLane];
#pragma unroll
            for (int p = 0; p < kProbesPerLane; ++p) {
                const bool v = k0 + 32u * p + lane < n_q;
                w[p] = v ? queue[k0 + 32u * p + lane] : kEmptyId;
                h[p] = home_slot(w[p], lg_l);
                bk[p] = make_uint4(kEmptyId, kEmptyId, kEmptyId, kEmptyId);
                if (v) bk[p] = __ldg(&buckets_l[key_quad(h[p], inter)]);
            }
#pragma unroll
            for (int p = 0; p < kProbesPerLane; ++p) {
                const uint4 b = bk[p];
                const int at = b.x == w[p] ? 0 : b.y == w[p] ? 1 : b.z == w[p] ? 2 : b.w == w[p] ? 3 : -1;
                r[p] = kEmptyId;
                if (w[p] != kEmptyId) {
                    uint32_t ns = 4u;
                    if (at >= 0) {
                        r[p] = __ldg(&keys_l[eidx_word(h[p] + (uint32_t)at, lg_l, inter)]);
                    } else if (b.x != kEmptyId && b.y != kEmptyId && b.z != kEmptyId && b.w != kEmptyId) {
                        r[p] = table_find(d.pool, base_l, lg_l, w[p], ns, inter);  // rare: the bucket is full
                    }
                    if (WORK) { ++wk.probes; wk.pslots += ns; }
                }
            }
#pragma unroll
            for (int p = 0; p < kProbesPerLane; ++p)
                push(w[p] != kEmptyId && r[p] < x.t, w[p]);
        }
        __syncwarp();
        if (last) break;
        if (k0) {  // move the unprobed rest (< kRound <= k0 keys) to the front; the ranges are disjoint
            const uint32_t rest = n_q - k0;
            for (uint32_t r = lane; r < rest; r += 32u) queue[r] = queue[k0 + r];
            n_q = rest;
            __syncwarp();
        }
    }
}

// Streams that store colours (kColInEntry, kColWords), warp classes: scan first, probe later.  A warp
// reads an item's smaller-endpoint list kScanPass entries per pass (kScanLoads 16-byte loads per
// lane, two entries each) and tests every entry's colour against the larger endpoint by hash alone.
// The few entries that pass (about 1/m) join the warp's candidate queue together with the index of
// their work item; the queue is probed 64 candidates at a time, whatever items they come from, so
// that an item with a handful of candidates does not pay for a probe round of its own.
#ifndef REPT_SCAN_LOADS
#define REPT_SCAN_LOADS 4
#endif
#ifndef REPT_SCAN_FULL
#define REPT_SCAN_FULL 1
#endif
constexpr uint32_t kScanLoads = REPT_SCAN_LOADS;  // 16-byte loads per lane and pass
constexpr uint32_t kScanPass = 64u * kScanLoads;  // entries per pass
constexpr bool kScanFull = REPT_SCAN_FULL != 0;  // passes inside the list skip the position checks
constexpr uint32_t kCandQ = 64u + kScanPass;       // candidate queue slots per warp
struct CandQueue {
    uint32_t* w;     // [kCandQ] candidate neighbour w
    uint32_t* item;  // [kCandQ] its work item, an index into srec
    uint32_t n;      // warp-uniform
};

// Probe candidates k0 .. k0 + take - 1 (take <= 64), two per lane: both items' records and then both
// home buckets are loaded before either is examined.  A hit older than its edge is a closed wedge.
template <bool WORK, int MODE>
__device__ __forceinline__ void cand_probe(const StreamDev& d, const CandQueue& cq, uint32_t k0, uint32_t take,
                                           unsigned long long* s_proc, MatchQueue& mq, Work& wk) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t w[2], h[2], lg[2], tt[2], ss[2], ll[2];
    unsigned long long base[2];
    uint4 bk[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const uint32_t k = 32u * p + lane;
        bool v = k < take;
        w[p] = kEmptyId;
        lg[p] = 2u;
        base[p] = 0ull;
        tt[p] = ss[p] = ll[p] = 0u;
        bk[p] = make_uint4(kEmptyId, kEmptyId, kEmptyId, kEmptyId);
        if (v) {
            const uint4* rec = reinterpret_cast<const uint4*>(d.srec + cq.item[k0 + k]);
            const uint4 r0 = rec[0], r1 = rec[1];  // {s, l, off_s, off_l}, {t, lgs, cnt_s, key}
            w[p] = cq.w[k0 + k];
            ss[p] = r0.x;
            ll[p] = r0.y;
            base[p] = 4ull * r0.w;
            tt[p] = r1.x;
            lg[p] = r1.y >> 8;
            if (!block_fits(d, 7, r0.w, lg[p])) {
                v = false;
                w[p] = kEmptyId;
            }
        }
        h[p] = home_slot(w[p], lg[p]);
        if (v) bk[p] = __ldg(reinterpret_cast<const uint4*>(d.pool + base[p]) + key_quad(h[p], true));
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const uint4 b = bk[p];
        const int at = b.x == w[p] ? 0 : b.y == w[p] ? 1 : b.z == w[p] ? 2 : b.w == w[p] ? 3 : -1;
        uint32_t r = kEmptyId;
        if (w[p] != kEmptyId) {
            uint32_t ns = 4u;
            if (at >= 0)
                r = __ldg(reinterpret_cast<const uint32_t*>(d.pool + base[p]) + eidx_word(h[p] + (uint32_t)at, lg[p], true));
            else if (b.x != kEmptyId && b.y != kEmptyId && b.z != kEmptyId && b.w != kEmptyId)
                r = table_find(d.pool, base[p], lg[p], w[p], ns, true);  // rare: the bucket is full
            if (WORK) { ++wk.probes; wk.pslots += ns; }
        }
        mq_push<WORK, MODE>(d, mq, w[p] != kEmptyId && r < tt[p], ss[p], ll[p], w[p], s_proc, wk);
    }
}

// Probe the queue's full rounds of 64 (`all`: everything) and move the rest to the front.
template <bool WORK, int MODE>
__device__ __forceinline__ void cand_flush(const StreamDev& d, CandQueue& cq, bool all, unsigned long long* s_proc,
                                           MatchQueue& mq, Work& wk) {
    __syncwarp();
    uint32_t k0 = 0;
    for (; all ? k0 < cq.n : k0 + 64u <= cq.n; k0 += 64u)
        cand_probe<WORK, MODE>(d, cq, k0, cq.n - k0 < 64u ? cq.n - k0 : 64u, s_proc, mq, wk);
    if (all) {
        cq.n = 0;
    } else if (k0) {  // the rest (< 64 <= k0 candidates): source and destination ranges are disjoint
        const uint32_t rest = cq.n - k0;
        const unsigned lane = threadIdx.x & 31u;
        for (uint32_t r = lane; r < rest; r += 32u) {
            cq.w[r] = cq.w[k0 + r];
            cq.item[r] = cq.item[k0 + r];
        }
        cq.n = rest;
    }
    __syncwarp();
}

// `t0`: the batch's first stream index.  A list holds the entries of earlier batches first (appends
// and block moves keep list order), so a pass whose last entry is older than t0 holds only entries
// older than every edge of the batch, and its entries skip the age test.
template <bool WORK, int MODE>
__device__ __forceinline__ void drain_warp_bin_coloured(const StreamDev& d, int cls, uint32_t grab,
                                                        unsigned long long* s_proc, CandQueue& cq, MatchQueue& mq,
                                                        Work& wk, uint32_t t0) {
    static_assert(63 + kScanPass <= kCandQ, "candidate queue too small");  // flushed at 64 after a pass
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    const unsigned long long count = d.ctrl->bin_count[cls];
    const uint32_t first = (uint32_t)d.ctrl->bin_start[cls];
    const WorkItem* items = d.srec + first;
    for (;;) {
        unsigned long long i0 = 0;
        if (lane == 0) i0 = atomicAdd(&d.ctrl->bin_next[cls], (unsigned long long)grab);
        i0 = __shfl_sync(0xFFFFFFFFu, i0, 0);
        if (i0 >= count) break;
        const unsigned long long i1 = i0 + grab < count ? i0 + grab : count;
        for (unsigned long long i = i0; i < i1; ++i) {
            const WorkItem x = items[i];
            const uint32_t n_s = x.cnt_s, l = x.l, t = x.t, lgs = x.lgs & 0xFFu;
            if (WORK && lane == 0) { wk.entries += n_s; wk.slots += n_s; }
            if (!(block_fits(d, 5, x.off_s, lgs) && REPT_CHECK(d.ctrl, 6, n_s, list_slots(lgs) + 1u) &&
                  block_fits(d, 7, x.off_l, x.lgs >> 8)))
                continue;  // (uniform over the warp: x is)
            // the list (32-byte aligned), two entries per 16-byte load; a lane past the end re-reads
            // the last pair, and its entries are masked off by position
            const uint4* list = reinterpret_cast<const uint4*>(d.pool + 4ull * x.off_s + (1ull << lgs));
            const uint32_t last_pair = (n_s - 1u) >> 1;
            const uint32_t item = first + (uint32_t)i;
            // kColWords: the entries' colour words, two per 8-byte load beside each entry pair
            const uint2* words = reinterpret_cast<const uint2*>(list_words(d.pool, x.off_s, lgs));
            // the tests of one pass on loaded entries q (and words cw); FULL: inside the list (no
            // position test); OLD: every entry older than the batch (no age test)
            auto test = [&](const uint4 (&q)[kScanLoads], const uint2 (&cw)[kScanLoads], uint32_t j0, auto full,
                            auto old) {
                constexpr bool FULL = decltype(full)::value, OLD = decltype(old)::value;
#pragma unroll
                for (uint32_t h = 0; h < kScanLoads; ++h) {
                    if (!FULL && j0 + 64u * h >= n_s) break;  // an empty part: uniform skip
                    const uint32_t jj = j0 + 64u * h + 2u * lane;
                    const bool words_mode = MODE == (int)kColWords;
                    const uint32_t w1 = words_mode ? q[h].x : q[h].x & kIdMask;
                    const uint32_t w2 = words_mode ? q[h].z : q[h].z & kIdMask;
                    const bool c1 = words_mode ? words_may_match(d, l, w1, cw[h].x) : colour_may_match(d, l, w1, q[h].x >> kIdBits);
                    const bool c2 = words_mode ? words_may_match(d, l, w2, cw[h].y) : colour_may_match(d, l, w2, q[h].z >> kIdBits);
                    const bool a1 = (FULL || jj < n_s) & (OLD || q[h].y < t) & c1;
                    const bool a2 = (FULL || jj + 1u < n_s) & (OLD || q[h].w < t) & c2;
                    const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1), m2 = __ballot_sync(0xFFFFFFFFu, a2);
                    if (m1 | m2) {  // rare (about 1/m of the entries pass): uniform
                        if (a1) {
                            const uint32_t k = cq.n + __popc(m1 & below);
                            cq.w[k] = w1;
                            cq.item[k] = item;
                        }
                        cq.n += __popc(m1);
                        if (a2) {
                            const uint32_t k = cq.n + __popc(m2 & below);
                            cq.w[k] = w2;
                            cq.item[k] = item;
                        }
                        cq.n += __popc(m2);
                    }
                }
                if (cq.n >= 64u) cand_flush<WORK, MODE>(d, cq, false, s_proc, mq, wk);
            };
            auto pass = [&](uint32_t j0, auto full) {
                constexpr bool FULL = decltype(full)::value;
                uint4 q[kScanLoads];
                uint2 cw[kScanLoads];
#pragma unroll
                for (uint32_t h = 0; h < kScanLoads; ++h) {
                    const uint32_t pr = (j0 >> 1) + 32u * h + lane;
                    const uint32_t at = FULL || pr < last_pair ? pr : last_pair;
                    q[h] = list[at];
                    cw[h] = make_uint2(0u, 0u);
                    if (MODE == (int)kColWords) cw[h] = words[at];
                }
                if (FULL && __shfl_sync(0xFFFFFFFFu, q[kScanLoads - 1].w, 31) < t0)
                    test(q, cw, j0, full, std::true_type{});
                else
                    test(q, cw, j0, full, std::false_type{});
            };
            uint32_t j0 = 0;
            if (kScanFull)
                for (; j0 + kScanPass <= n_s; j0 += kScanPass) pass(j0, std::true_type{});
            for (; j0 < n_s; j0 += kScanPass) pass(j0, std::false_type{});
        }
    }
}

template <int TILE, bool WORK, int MODE>
__device__ __forceinline__ void drain_tile_bin(const StreamDev& d, int cls, unsigned long long* s_proc,
                                               MatchQueue& mq, Work& wk) {
    constexpr uint32_t kPerWarp = 32 / TILE, kRounds = 4, kGrab = kPerWarp * kRounds;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long count = d.ctrl->bin_count[cls];
    const WorkItem* items = d.srec + d.ctrl->bin_start[cls];
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&d.ctrl->bin_next[cls], (unsigned long long)kGrab);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= count) break;
#pragma unroll 1
        for (uint32_t r = 0; r < kRounds; ++r) {
            const unsigned long long i = base + r * kPerWarp + lane / TILE;
            const bool valid = i < count;
            WorkItem x{};
            if (valid) x = items[i];
            intersect_tile<TILE, WORK, MODE>(d, x, valid, s_proc, mq, wk);
        }
    }
}

// Warp classes: a warp claims `grab` consecutive items per atomic on the class cursor (one cursor is
// shared by every warp of the grid, so claiming one item at a time serialises on it).
template <bool WORK, int MODE>
__device__ __forceinline__ void drain_warp_bin(const StreamDev& d, int cls, uint32_t grab, unsigned long long* s_proc,
                                               uint32_t* queue, MatchQueue& mq, Work& wk) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long count = d.ctrl->bin_count[cls];
    const WorkItem* items = d.srec + d.ctrl->bin_start[cls];
    for (;;) {
        unsigned long long i0 = 0;
        if (lane == 0) i0 = atomicAdd(&d.ctrl->bin_next[cls], (unsigned long long)grab);
        i0 = __shfl_sync(0xFFFFFFFFu, i0, 0);
        if (i0 >= count) break;
        const unsigned long long i1 = i0 + grab < count ? i0 + grab : count;
        for (unsigned long long i = i0; i < i1; ++i) {
            const WorkItem x = items[i];
            intersect_warp<WORK, MODE>(d, x, queue, wk, [&](bool has, uint32_t w) {
                mq_push<WORK, MODE>(d, mq, has, x.s, x.l, w, s_proc, wk);
            });
        }
    }
}

// UpdateTriangleCNT for every edge of the batch.  The edges were sorted into work classes by
// k_insert; warps claim work dynamically, largest class first.  Dynamic shared memory: c uint64
// counters (tau^(i) of this block).  WORK = true also tallies the table reads.
template <bool WORK, int MODE>
__device__ __forceinline__ void k_intersect_body(const StreamDev& d, const BatchDev& b) {
    extern __shared__ unsigned long long s_proc[];
    // the scan-first warp path (candidate queue): streams that store colours
    constexpr bool CAND = MODE == (int)kColInEntry || MODE == (int)kColWords;
    __shared__ uint32_t s_queue[CAND ? 1 : 256 / 32][kQueue];  // intersect_warp's key queue
    __shared__ uint32_t s_cand[CAND ? 256 / 32 : 1][2][kCandQ];
    __shared__ uint32_t s_match[256 / 32][3][kMatchQ];
    for (uint32_t i = threadIdx.x; i < d.c; i += blockDim.x) s_proc[i] = 0ull;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const unsigned wid = threadIdx.x >> 5;
    uint32_t* queue = s_queue[CAND ? 0 : wid];
    MatchQueue mq{s_match[wid][0], s_match[wid][1], s_match[wid][2], 0u};
    CandQueue cq{s_cand[CAND ? wid : 0][0], s_cand[CAND ? wid : 0][1], 0u};
    Work wk;
    if (d.ctrl->status == 0u) {
        // WORK: per class, the probes issued and the warp-cycles spent (clock64 around each drain)
        long long t0 = WORK ? clock64() : 0;
        unsigned long long p0 = wk.probes;
        auto mark = [&](int cls) {
            if (WORK) {
                const long long t1 = clock64();
                const unsigned long long p1 = wk.probes;
                unsigned long long pr = p1 - p0;
                for (int o = 16; o > 0; o >>= 1) pr += __shfl_down_sync(0xFFFFFFFFu, pr, o);
                if (lane == 0) {
                    atomicAdd(&d.ctrl->class_cycles[cls], (unsigned long long)(t1 - t0));
                    atomicAdd(&d.ctrl->class_probes[cls], pr);
                }
                t0 = t1;
                p0 = p1;
            }
        };
        if constexpr (CAND) {
            drain_warp_bin_coloured<WORK, MODE>(d, 5, kScanGrabHub, s_proc, cq, mq, wk, (uint32_t)b.t0);
            mark(5);
            drain_warp_bin_coloured<WORK, MODE>(d, 4, kScanGrabMid, s_proc, cq, mq, wk, (uint32_t)b.t0);
            if (cq.n) cand_flush<WORK, MODE>(d, cq, true, s_proc, mq, wk);
            mark(4);
        } else {
            drain_warp_bin<WORK, MODE>(d, 5, kGrabHub, s_proc, queue, mq, wk);
            mark(5);
            drain_warp_bin<WORK, MODE>(d, 4, kGrabMid, s_proc, queue, mq, wk);
            mark(4);
        }
        drain_tile_bin<32, WORK, MODE>(d, 3, s_proc, mq, wk);
        mark(3);
        drain_tile_bin<16, WORK, MODE>(d, 2, s_proc, mq, wk);
        mark(2);
        drain_tile_bin<8, WORK, MODE>(d, 1, s_proc, mq, wk);
        mark(1);
        drain_tile_bin<4, WORK, MODE>(d, 0, s_proc, mq, wk);
        mark(0);
        if (mq.n) mq_flush<WORK, MODE>(d, mq, mq.n, s_proc, wk);
        if (WORK && blockIdx.x == 0 && threadIdx.x < kBins)
            d.ctrl->class_items[threadIdx.x] += d.ctrl->bin_count[threadIdx.x];
    }
    if (WORK) {
        for (int o = 16; o > 0; o >>= 1) {
            wk.entries += __shfl_down_sync(0xFFFFFFFFu, wk.entries, o);
            wk.slots += __shfl_down_sync(0xFFFFFFFFu, wk.slots, o);
            wk.probes += __shfl_down_sync(0xFFFFFFFFu, wk.probes, o);
            wk.pslots += __shfl_down_sync(0xFFFFFFFFu, wk.pslots, o);
            wk.wedges += __shfl_down_sync(0xFFFFFFFFu, wk.wedges, o);
            wk.counted += __shfl_down_sync(0xFFFFFFFFu, wk.counted, o);
        }
        if (lane == 0) {
            atomicAdd(&d.ctrl->small_entries, wk.entries);
            atomicAdd(&d.ctrl->small_slots, wk.slots);
            atomicAdd(&d.ctrl->probes, wk.probes);
            atomicAdd(&d.ctrl->probe_slots, wk.pslots);
            atomicAdd(&d.ctrl->wedges, wk.wedges);
            atomicAdd(&d.ctrl->counted, wk.counted);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < d.c; i += blockDim.x)
        if (s_proc[i]) atomicAdd(&d.proc[i], s_proc[i]);
}

// ---------------------------------------------------------------------------------------------
// Intersection for a group of streams with one grid: every warp may work on any stream.  The
// per-class work lists of the k streams are concatenated (k_group_prefix writes, per class, the
// prefix of the streams' item counts); warps claim ranges of the concatenation with one cursor per
// class and find each item's stream from the prefix.  Closed wedges carry their stream in the
// match queue and tau^(i) goes straight to global memory.

// Per class c: pref[c * (k + 1) + i] = sum of the item counts of streams < i; cursors reset.  One
// block of any multiple of 32 threads up to 1024.
__device__ __forceinline__ void group_prefix_body(const StreamDev* __restrict__ ds, uint32_t k,
                                                  unsigned long long* __restrict__ pref,
                                                  unsigned long long* __restrict__ cursor) {
    __shared__ unsigned long long warp_sum[32];
    __shared__ unsigned long long carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5, warps = blockDim.x >> 5;
    for (int c = 0; c < kBins; ++c) {
        if (tid == 0) carry = 0ull;
        __syncthreads();
        for (uint32_t base = 0; base < k; base += blockDim.x) {
            const uint32_t i = base + tid;
            const unsigned long long v = i < k && ds[i].ctrl->status == 0u ? ds[i].ctrl->bin_count[c] : 0ull;
            unsigned long long incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            if (lane == 31) warp_sum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const unsigned long long w = lane < warps ? warp_sum[lane] : 0ull;
                unsigned long long wi = w;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                    if (lane >= (uint32_t)o) wi += y;
                }
                warp_sum[lane] = wi - w;
            }
            __syncthreads();
            const unsigned long long excl = carry + warp_sum[wid] + incl - v;
            if (i < k) pref[c * (k + 1) + i] = excl;
            __syncthreads();
            if (tid == blockDim.x - 1) carry = excl + v;
            __syncthreads();
        }
        if (tid == 0) {
            pref[c * (k + 1) + k] = carry;
            cursor[c] = 0ull;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_group_prefix(const StreamDev* __restrict__ ds, uint32_t k,
                                                       unsigned long long* __restrict__ pref,
                                                       unsigned long long* __restrict__ cursor) {
    group_prefix_body(ds, k, pref, cursor);
}

struct GroupQueue {
    uint32_t* sid;
    uint32_t* s;
    uint32_t* l;
    uint32_t* w;
    uint32_t n;
};

__device__ __forceinline__ void gq_flush(const StreamDev* __restrict__ ds, GroupQueue& q, uint32_t take) {
    const unsigned lane = threadIdx.x & 31u;
    if (lane < take) {
        const uint32_t i = q.n - take + lane;
        const StreamDev& d = ds[q.sid[i]];
        const uint32_t s = q.s[i], l = q.l[i], w = q.w[i];
        uint32_t found = 0;
        for (uint32_t k = d.kbeg; k < d.kend; ++k) {
            const uint64_t sk = group_seed(d.seed, k);
            const uint32_t js = colour_of(s, w, sk, d.fm);
            uint32_t i;
            if (processor_of(d, k, js, i) && colour_of(l, w, sk, d.fm) == js) {
                ++found;
                atomicAdd(&d.proc[i], 1ull);
            }
        }
        if (found) {
            atomicAdd(&d.local[w], (unsigned long long)found);
            atomicAdd(&d.local[s], (unsigned long long)found);
            atomicAdd(&d.local[l], (unsigned long long)found);
        }
    }
    q.n -= take;
    __syncwarp();
}

__device__ __forceinline__ void gq_push(const StreamDev* __restrict__ ds, GroupQueue& q, bool has, uint32_t sid,
                                        uint32_t s, uint32_t l, uint32_t w) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, has);
    if (has) {
        const uint32_t i = q.n + __popc(mask & ((1u << lane) - 1u));
        q.sid[i] = sid;
        q.s[i] = s;
        q.l[i] = l;
        q.w[i] = w;
    }
    q.n += __popc(mask);
    __syncwarp();
    if (q.n >= 32u) gq_flush(ds, q, 32u);
}

// Stream of item `i` of class c: the last stream whose prefix is <= i, searched from `from`.
__device__ __forceinline__ uint32_t group_stream_of(const unsigned long long* __restrict__ pc, uint32_t k,
                                                    unsigned long long i, uint32_t from) {
    uint32_t sidx = from;
    while (sidx + 1 < k && pc[sidx + 1] <= i) ++sidx;
    return sidx;
}

__device__ __forceinline__ uint32_t group_stream_search(const unsigned long long* __restrict__ pc, uint32_t k,
                                                        unsigned long long i) {
    uint32_t lo = 0, hi = k - 1;  // pc[0] = 0 <= i
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pc[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ WorkItem group_item(const StreamDev& d, int cls, unsigned long long local) {
    return d.srec[d.ctrl->bin_start[cls] + local];
}

template <int TILE>
__device__ __forceinline__ void group_drain_tiles(const StreamDev* __restrict__ ds, uint32_t k, int cls,
                                                  const unsigned long long* __restrict__ pref,
                                                  unsigned long long* __restrict__ cursor, GroupQueue& q) {
    constexpr uint32_t kPerWarp = 32 / TILE, kRounds = 4, kGrab = kPerWarp * kRounds;
    const unsigned lane = threadIdx.x & 31u, j = lane & (TILE - 1);
    const unsigned long long* pc = pref + cls * (k + 1);
    const unsigned long long total = pc[k];
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&cursor[cls], (unsigned long long)kGrab);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= total) break;
        const uint32_t s0 = group_stream_search(pc, k, base);
#pragma unroll 1
        for (uint32_t r = 0; r < kRounds; ++r) {
            const unsigned long long i = base + r * kPerWarp + lane / TILE;
            const bool valid = i < total;
            bool has = false;
            uint32_t sid = 0, w = 0;
            WorkItem x{};
            if (valid) {
                sid = group_stream_of(pc, k, i, s0);
                const StreamDev& d = ds[sid];
                x = group_item(d, cls, i - pc[sid]);
                if (j < x.cnt_s) {
                    const unsigned long long at = 4ull * x.off_s + (1ull << (x.lgs & 0xFFu)) + j;
                    const bool fits = REPT_CHECK(d.ctrl, 3, at, 4ull * d.pool_quads) &&
                                      block_fits(d, 4, x.off_l, x.lgs >> 8);
                    const uint2 es = fits ? d.pool[at] : make_uint2(kEmptyId, kEmptyId);
                    const uint32_t ws = es.x & id_mask(d);
                    if (es.y < x.t && (d.colours != kColInEntry || wedge_may_count(d, x.l, ws, es.x >> kIdBits))) {
                        uint32_t nslots = 0;
                        has = table_find(d.pool, 4ull * x.off_l, x.lgs >> 8, ws, nslots, tables_interleaved(d)) < x.t;
                        w = ws;
                    }
                }
            }
            gq_push(ds, q, has, sid, x.s, x.l, w);
        }
    }
}

// Warp classes of a group: the scan-first scheme of drain_warp_bin_coloured over all streams of the
// group, a candidate also naming its stream.  A stream without colours in its entries passes every
// entry older than the edge to the probes.
struct GroupCand {
    uint32_t* w;     // [kCandQ] candidate neighbour w
    uint32_t* item;  // [kCandQ] its work item, an index into its stream's srec
    uint32_t* sid;   // [kCandQ] its stream
    uint32_t n;      // warp-uniform
};

__device__ __forceinline__ void gcand_probe(const StreamDev* __restrict__ ds, const GroupCand& cq, uint32_t k0,
                                            uint32_t take, GroupQueue& q) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t w[2], h[2], lg[2], tt[2], ss[2], ll[2], sd[2];
    const uint2* pool[2];
    bool inter[2];
    unsigned long long base[2];
    uint4 bk[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const uint32_t k = 32u * p + lane;
        bool v = k < take;
        w[p] = kEmptyId;
        lg[p] = 2u;
        base[p] = 0ull;
        tt[p] = ss[p] = ll[p] = sd[p] = 0u;
        pool[p] = nullptr;
        inter[p] = true;
        bk[p] = make_uint4(kEmptyId, kEmptyId, kEmptyId, kEmptyId);
        if (v) {
            sd[p] = cq.sid[k0 + k];
            const StreamDev& d = ds[sd[p]];
            const uint4* rec = reinterpret_cast<const uint4*>(d.srec + cq.item[k0 + k]);
            const uint4 r0 = rec[0], r1 = rec[1];  // {s, l, off_s, off_l}, {t, lgs, cnt_s, key}
            w[p] = cq.w[k0 + k];
            ss[p] = r0.x;
            ll[p] = r0.y;
            base[p] = 4ull * r0.w;
            tt[p] = r1.x;
            lg[p] = r1.y >> 8;
            pool[p] = d.pool;
            inter[p] = tables_interleaved(d);
            if (!block_fits(d, 7, r0.w, lg[p])) {
                v = false;
                w[p] = kEmptyId;
            }
        }
        h[p] = home_slot(w[p], lg[p]);
        if (v) bk[p] = __ldg(reinterpret_cast<const uint4*>(pool[p] + base[p]) + key_quad(h[p], inter[p]));
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const uint4 b = bk[p];
        const int at = b.x == w[p] ? 0 : b.y == w[p] ? 1 : b.z == w[p] ? 2 : b.w == w[p] ? 3 : -1;
        uint32_t r = kEmptyId;
        if (w[p] != kEmptyId) {
            uint32_t ns = 4u;
            if (at >= 0)
                r = __ldg(reinterpret_cast<const uint32_t*>(pool[p] + base[p]) +
                          eidx_word(h[p] + (uint32_t)at, lg[p], inter[p]));
            else if (b.x != kEmptyId && b.y != kEmptyId && b.z != kEmptyId && b.w != kEmptyId)
                r = table_find(pool[p], base[p], lg[p], w[p], ns, inter[p]);  // rare: the bucket is full
        }
        gq_push(ds, q, w[p] != kEmptyId && r < tt[p], sd[p], ss[p], ll[p], w[p]);
    }
}

__device__ __forceinline__ void gcand_flush(const StreamDev* __restrict__ ds, GroupCand& cq, bool all, GroupQueue& q) {
    __syncwarp();
    uint32_t k0 = 0;
    for (; all ? k0 < cq.n : k0 + 64u <= cq.n; k0 += 64u) gcand_probe(ds, cq, k0, cq.n - k0 < 64u ? cq.n - k0 : 64u, q);
    if (all) {
        cq.n = 0;
    } else if (k0) {  // the rest (< 64 <= k0 candidates): source and destination ranges are disjoint
        const uint32_t rest = cq.n - k0;
        const unsigned lane = threadIdx.x & 31u;
        for (uint32_t r = lane; r < rest; r += 32u) {
            cq.w[r] = cq.w[k0 + r];
            cq.item[r] = cq.item[k0 + r];
            cq.sid[r] = cq.sid[k0 + r];
        }
        cq.n = rest;
    }
    __syncwarp();
}

__device__ __forceinline__ void group_drain_warps_cand(const StreamDev* __restrict__ ds, uint32_t k, int cls,
                                                       uint32_t grab, const unsigned long long* __restrict__ pref,
                                                       unsigned long long* __restrict__ cursor, GroupCand& cq,
                                                       GroupQueue& q) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    const unsigned long long* pc = pref + cls * (k + 1);
    const unsigned long long total = pc[k];
    for (;;) {
        unsigned long long i0 = 0;
        if (lane == 0) i0 = atomicAdd(&cursor[cls], (unsigned long long)grab);
        i0 = __shfl_sync(0xFFFFFFFFu, i0, 0);
        if (i0 >= total) break;
        const unsigned long long i1 = i0 + grab < total ? i0 + grab : total;
        uint32_t sid = group_stream_search(pc, k, i0);
        for (unsigned long long i = i0; i < i1; ++i) {
            sid = group_stream_of(pc, k, i, sid);
            const StreamDev& d = ds[sid];
            const uint32_t item = (uint32_t)(d.ctrl->bin_start[cls] + (i - pc[sid]));
            const WorkItem x = d.srec[item];
            const uint32_t n_s = x.cnt_s, l = x.l, t = x.t, lgs = x.lgs & 0xFFu;
            if (!(block_fits(d, 5, x.off_s, lgs) && REPT_CHECK(d.ctrl, 6, n_s, list_slots(lgs) + 1u) &&
                  block_fits(d, 7, x.off_l, x.lgs >> 8)))
                continue;  // (uniform over the warp: x is)
            const uint4* list = reinterpret_cast<const uint4*>(d.pool + 4ull * x.off_s + (1ull << lgs));
            const uint32_t last_pair = (n_s - 1u) >> 1;
            const uint32_t mask = id_mask(d);
            const bool open = d.colours != kColInEntry;  // no colour test: every older entry is probed
            auto pass = [&](uint32_t j0, auto full) {
                constexpr bool FULL = decltype(full)::value;
                uint4 qv[kScanLoads];
#pragma unroll
                for (uint32_t hh = 0; hh < kScanLoads; ++hh) {
                    const uint32_t pr = (j0 >> 1) + 32u * hh + lane;
                    qv[hh] = list[FULL || pr < last_pair ? pr : last_pair];
                }
#pragma unroll
                for (uint32_t hh = 0; hh < kScanLoads; ++hh) {
                    if (!FULL && j0 + 64u * hh >= n_s) break;  // an empty part: uniform skip
                    const uint32_t jj = j0 + 64u * hh + 2u * lane;
                    const uint32_t w1 = qv[hh].x & mask, w2 = qv[hh].z & mask;
                    const bool a1 = (FULL || jj < n_s) & (qv[hh].y < t) &
                                    (open | colour_may_match(d, l, w1, qv[hh].x >> kIdBits));
                    const bool a2 = (FULL || jj + 1u < n_s) & (qv[hh].w < t) &
                                    (open | colour_may_match(d, l, w2, qv[hh].z >> kIdBits));
                    const unsigned m1 = __ballot_sync(0xFFFFFFFFu, a1), m2 = __ballot_sync(0xFFFFFFFFu, a2);
                    if (m1 | m2) {
                        if (a1) {
                            const uint32_t kk = cq.n + __popc(m1 & below);
                            cq.w[kk] = w1;
                            cq.item[kk] = item;
                            cq.sid[kk] = sid;
                        }
                        cq.n += __popc(m1);
                        if (a2) {
                            const uint32_t kk = cq.n + __popc(m2 & below);
                            cq.w[kk] = w2;
                            cq.item[kk] = item;
                            cq.sid[kk] = sid;
                        }
                        cq.n += __popc(m2);
                    }
                }
                if (cq.n >= 64u) gcand_flush(ds, cq, false, q);
            };
            uint32_t j0 = 0;
            if (kScanFull)
                for (; j0 + kScanPass <= n_s; j0 += kScanPass) pass(j0, std::true_type{});
            for (; j0 < n_s; j0 += kScanPass) pass(j0, std::false_type{});
        }
    }
}

// Shared memory of the group intersection, per block of 8 warps: a candidate queue of three arrays
// (w, item, stream) and a match queue of four arrays (stream, s, l, w) per warp.
constexpr uint32_t kGroupSmemWords = 8u * 3u * kCandQ + 8u * 4u * kMatchQ;

__device__ __forceinline__ void intersect_group_body(const StreamDev* __restrict__ ds, uint32_t k,
                                                     const unsigned long long* __restrict__ pref,
                                                     unsigned long long* __restrict__ cursor, uint32_t* smem) {
    const unsigned wid = threadIdx.x >> 5;
    uint32_t* cw = smem + wid * 3u * kCandQ;
    uint32_t* mq = smem + 8u * 3u * kCandQ + wid * 4u * kMatchQ;
    GroupQueue q{mq, mq + kMatchQ, mq + 2u * kMatchQ, mq + 3u * kMatchQ, 0u};
    GroupCand cq{cw, cw + kCandQ, cw + 2u * kCandQ, 0u};
    group_drain_warps_cand(ds, k, 5, kGrabHub, pref, cursor, cq, q);
    group_drain_warps_cand(ds, k, 4, kGrabMid, pref, cursor, cq, q);
    if (cq.n) gcand_flush(ds, cq, true, q);
    group_drain_tiles<32>(ds, k, 3, pref, cursor, q);
    group_drain_tiles<16>(ds, k, 2, pref, cursor, q);
    group_drain_tiles<8>(ds, k, 1, pref, cursor, q);
    group_drain_tiles<4>(ds, k, 0, pref, cursor, q);
    if (q.n) gq_flush(ds, q, q.n);
}

__global__ void __launch_bounds__(256, 4) k_intersect_group(const StreamDev* __restrict__ ds, uint32_t k,
                                                            const unsigned long long* __restrict__ pref,
                                                            unsigned long long* __restrict__ cursor) {
    __shared__ uint32_t smem[kGroupSmemWords];
    intersect_group_body(ds, k, pref, cursor, smem);
}

// Algorithm 2's triangle-pair counters, folded in after the intersection.  Edge e of group k was a
// wedge edge of kcnt closed wedges this batch, all for the processor i = k*m + h_k(e).  In stream
// order they saw the counter values B, B+1, ..., B+kcnt-1 (B its value before the batch), so their
// contribution to eta^(i) and to eta_x, eta_y of e's endpoints is kcnt*B + kcnt*(kcnt-1)/2, whatever
// their order; then the counter advances by kcnt.  (The counter of a newly stored edge starts at 0.)
__global__ void k_pairs(StreamDev d) {
    if (d.ctrl->status) return;
    const unsigned long long n = d.ctrl->n_pairs;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t idx = d.pair_list[q];
        const uint32_t t = idx / d.groups, k = idx % d.groups;
        const unsigned long long kc = d.pair_evt[idx], base = d.pair_tau[idx];
        const unsigned long long add = kc * base + kc * (kc - 1) / 2;
        const uint2 e = d.edge_ends[t];
        const uint32_t i = k * d.m + colour_of(e.x, e.y, group_seed(d.seed, k), d.fm);
        atomicAdd(&d.eta_proc[i], add);
        atomicAdd(&d.eta_local[e.x], add);
        atomicAdd(&d.eta_local[e.y], add);
        d.pair_tau[idx] = (uint32_t)(base + kc);
        d.pair_evt[idx] = 0u;
    }
}

// Algorithm 2's estimates (c > m, c mod m != 0): the two group estimates combined with the plug-in
// inverse-variance weights; with both weights zero the full groups' estimate.  Same expression order
// as the scalar formulas of Section III-B.2.
__device__ __forceinline__ double combine_estimates(double t1, double t2, double eta_hat, double md, double c1,
                                                    double c2) {
    const double w1 = t1 * (md - 1.0) / c1;
    const double w2 = (t1 * (md * md - c2) + 2.0 * eta_hat * (md - c2)) / c2;
    return (w1 + w2 > 0.0) ? (w2 * t1 + w1 * t2) / (w1 + w2) : t1;
}

__global__ void k_global_estimate_partial(const unsigned long long* __restrict__ proc,
                                          const unsigned long long* __restrict__ eta, uint32_t m, uint32_t c,
                                          double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t c1 = c / m, c2 = c % m;
    unsigned long long s1 = 0, s2 = 0, se = 0;
    for (uint32_t i = 0; i < c1 * m; ++i) s1 += proc[i];
    for (uint32_t i = c1 * m; i < c; ++i) s2 += proc[i];
    for (uint32_t i = 0; i < c; ++i) se += eta[i];
    const double md = (double)m;
    const double t1 = (double)s1 * (md / (double)c1), t2 = (double)s2 * (md * md / (double)c2);
    const double eta_hat = (double)se * (md * md * md / (double)c);
    *out = combine_estimates(t1, t2, eta_hat, md, (double)c1, (double)c2);
}

__global__ void k_local_estimates_partial(const unsigned long long* __restrict__ l1,
                                          const unsigned long long* __restrict__ l2,
                                          const unsigned long long* __restrict__ el, uint32_t n, uint32_t m,
                                          uint32_t c, double* __restrict__ out) {
    const uint32_t c1 = c / m, c2 = c % m;
    const double md = (double)m;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double a1 = (double)l1[v] * (md / (double)c1), a2 = (double)l2[v] * (md * md / (double)c2);
        const double eh = (double)el[v] * (md * md * md / (double)c);
        out[v] = combine_estimates(a1, a2, eh, md, (double)c1, (double)c2);
    }
}

// sum_i tau_v^(i) over all processors when the local counts are split in two.
__global__ void k_add_local(const unsigned long long* __restrict__ a, const unsigned long long* __restrict__ b,
                            uint32_t n, unsigned long long* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) out[v] = a[v] + b[v];
}

// Kernel entry points.  Each batch kernel exists twice: for one stream (state and batch passed by
// value) and for many streams at once (`_multi`: blockIdx.y selects the stream, whose state and batch
// descriptors are read from device arrays; blockIdx.x / gridDim.x then range over that stream's blocks).
__device__ __forceinline__ Grid launch_grid() { return Grid{blockIdx.x, gridDim.x}; }

__global__ void k_classify(StreamDev d, BatchDev b) { k_classify_body(d, b, launch_grid()); }

__global__ void k_classify_multi(const StreamDev* __restrict__ ds, const BatchDev* __restrict__ bs) {
    __shared__ StreamDev sd;
    __shared__ BatchDev sb;
    if (threadIdx.x == 0) {
        sd = ds[blockIdx.y];
        sb = bs[blockIdx.y];
    }
    __syncthreads();
    k_classify_body(sd, sb, launch_grid());
}

__global__ void k_plan(StreamDev d) { k_plan_body(d, launch_grid()); }

__global__ void k_plan_multi(const StreamDev* __restrict__ ds, const BatchDev* __restrict__ bs) {
    (void)bs;
    __shared__ StreamDev sd;
    if (threadIdx.x == 0) sd = ds[blockIdx.y];
    __syncthreads();
    k_plan_body(sd, launch_grid());
}

__global__ void k_commit(StreamDev d) { k_commit_body(d, launch_grid()); }

__global__ void k_commit_multi(const StreamDev* __restrict__ ds, const BatchDev* __restrict__ bs) {
    (void)bs;
    __shared__ StreamDev sd;
    if (threadIdx.x == 0) sd = ds[blockIdx.y];
    __syncthreads();
    k_commit_body(sd, launch_grid());
}

__global__ void __launch_bounds__(256) k_rehash_big(StreamDev d) {
    __shared__ uint32_t smem[kMoveSmemWords];
    k_rehash_big_body(d, launch_grid(), smem);
}

__global__ void __launch_bounds__(256) k_rehash_big_multi(const StreamDev* __restrict__ ds,
                                                            const BatchDev* __restrict__ bs) {
    (void)bs;
    __shared__ StreamDev sd;
    __shared__ uint32_t smem[kMoveSmemWords];
    if (threadIdx.x == 0) sd = ds[blockIdx.y];
    __syncthreads();
    k_rehash_big_body(sd, launch_grid(), smem);
}

// Two blocks of 1024 threads per SM (32 registers a thread), so that the whole grid is resident.
__global__ void __launch_bounds__(1024, 2) k_rehash_huge(StreamDev d) {
    __shared__ uint32_t smem[kMoveSmemWords];
    k_rehash_huge_body(d, launch_grid(), smem);
}

__global__ void __launch_bounds__(1024, 2) k_rehash_huge_multi(const StreamDev* __restrict__ ds,
                                                              const BatchDev* __restrict__ bs) {
    (void)bs;
    __shared__ StreamDev sd;
    __shared__ uint32_t smem[kMoveSmemWords];
    if (threadIdx.x == 0) sd = ds[blockIdx.y];
    __syncthreads();
    k_rehash_huge_body(sd, launch_grid(), smem);
}

// 5 blocks of 256 threads per SM (48 registers): 2.79 against 2.93 ms per headline step at 56
// registers and 4 blocks; at 6 blocks (40 registers) it spills.
__global__ void __launch_bounds__(256, 5) k_insert(StreamDev d, BatchDev b) { k_insert_body(d, b, launch_grid()); }

__global__ void k_insert_multi(const StreamDev* __restrict__ ds, const BatchDev* __restrict__ bs) {
    __shared__ StreamDev sd;
    __shared__ BatchDev sb;
    if (threadIdx.x == 0) {
        sd = ds[blockIdx.y];
        sb = bs[blockIdx.y];
    }
    __syncthreads();
    k_insert_body(sd, sb, launch_grid());
}

__global__ void __launch_bounds__(1024) k_sort_scan(StreamDev d) { k_sort_scan_body(d, launch_grid()); }

__global__ void __launch_bounds__(1024) k_sort_scan_multi(const StreamDev* __restrict__ ds,
                                                           const BatchDev* __restrict__ bs) {
    (void)bs;
    __shared__ StreamDev sd;
    if (threadIdx.x == 0) sd = ds[blockIdx.y];
    __syncthreads();
    k_sort_scan_body(sd, launch_grid());
}

__global__ void k_sort_scatter(StreamDev d, BatchDev b) { k_sort_scatter_body(d, b, launch_grid()); }

__global__ void k_sort_scatter_multi(const StreamDev* __restrict__ ds, const BatchDev* __restrict__ bs) {
    __shared__ StreamDev sd;
    __shared__ BatchDev sb;
    if (threadIdx.x == 0) {
        sd = ds[blockIdx.y];
        sb = bs[blockIdx.y];
    }
    __syncthreads();
    k_sort_scatter_body(sd, sb, launch_grid());
}

// ---------------------------------------------------------------------------------------------
// One persistent launch for a whole group round: every step of the batch path (classify, plan,
// commit, both block moves, insert, sort, the group's intersection) for every stream, separated by
// grid-wide barriers.  The grid is co-resident (a cooperative launch); each step runs over virtual
// blocks (stream, block of that stream) exactly as the launch per step would, so the counts are the
// same.  Every barrier wait is bounded in time: when it runs out, the block records kStTimeout in
// every stream's status (REPT_E_TIMEOUT at the next synchronising call) and returns, and the other
// blocks, seeing timed_out, stop waiting and return too.  No block ever waits without a limit.

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks of the grid meet; false if the wait gave up (after wait_ns nanoseconds) or another
// block's did.
__device__ __forceinline__ bool grid_barrier(GroupSync* gs, unsigned long long wait_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &gs->gen;
        volatile unsigned int* vto = &gs->timed_out;
        int ok = 1;
        const unsigned int g = *vgen;  // cannot advance before this block arrives
        __threadfence();               // this block's writes of the step before the barrier
        const unsigned int target = gridDim.x + gs->extra;
        if (atomicAdd(&gs->count, 1u) == target - 1u) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g) {
                if (*vto || global_ns() - t0 > wait_ns) {
                    atomicExch(&gs->timed_out, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Virtual blocks per stream of each step (the multi-launch shape's grid x dimensions).
struct PersistShape {
    uint32_t x_edge, x_big, x_huge;
};

// Dynamic shared memory of the persistent kernel: the larger of the block moves' and the group
// intersection's needs.
constexpr uint32_t kPersistSmemWords = kMoveSmemWords > kGroupSmemWords ? kMoveSmemWords : kGroupSmemWords;

__global__ void __launch_bounds__(256, 3) k_group_persistent(const StreamDev* __restrict__ ds,
                                                           const BatchDev* __restrict__ bs, uint32_t k,
                                                           PersistShape sh, unsigned long long* __restrict__ pref,
                                                           unsigned long long* __restrict__ cursor, GroupSync* gs,
                                                           unsigned long long wait_ns) {
    extern __shared__ __align__(16) uint32_t psmem[];
    __shared__ StreamDev sd;
    __shared__ BatchDev sb;
    __shared__ uint32_t s_cur;
    if (threadIdx.x == 0) s_cur = 0xFFFFFFFFu;
    __syncthreads();
    // run `body` for every virtual block (stream, block x of X) this block is dealt
    auto step = [&](uint32_t X, auto&& body) {
        const unsigned long long total = (unsigned long long)k * X;
        for (unsigned long long vb = blockIdx.x; vb < total; vb += gridDim.x) {
            const uint32_t sid = (uint32_t)(vb / X);
            if (sid != s_cur) {  // uniform over the block
                __syncthreads();
                if (threadIdx.x == 0) {
                    sd = ds[sid];
                    sb = bs[sid];
                    s_cur = sid;
                }
                __syncthreads();
            }
            body(Grid{(uint32_t)(vb % X), X});
        }
    };
    bool ok = true;
    step(sh.x_edge, [&](Grid g) { k_classify_body(sd, sb, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_edge, [&](Grid g) { k_plan_body(sd, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_edge, [&](Grid g) { k_commit_body(sd, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_big, [&](Grid g) { k_rehash_big_body(sd, g, psmem); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_huge, [&](Grid g) { k_rehash_huge_body(sd, g, psmem); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_edge, [&](Grid g) { k_insert_body(sd, sb, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(1u, [&](Grid g) { k_sort_scan_body(sd, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) step(sh.x_edge, [&](Grid g) { k_sort_scatter_body(sd, sb, g); });
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok && blockIdx.x == 0) group_prefix_body(ds, k, pref, cursor);
    ok = ok && grid_barrier(gs, wait_ns);
    if (ok) {
        intersect_group_body(ds, k, pref, cursor, psmem);
        return;
    }
    // a wait ran out: the round is not applied for any stream (every step checks the status first)
    if (threadIdx.x == 0)
        for (uint32_t i = blockIdx.x; i < k; i += gridDim.x) atomicOr(&ds[i].ctrl->status, kStTimeout);
}

// Streams whose entries carry their colour (one hash group, m <= 256): 5 blocks of 256 threads per SM.
#ifndef REPT_COLOURED_BLOCKS
#define REPT_COLOURED_BLOCKS 5
#endif
template <bool WORK>
__global__ void __launch_bounds__(256, REPT_COLOURED_BLOCKS) k_intersect(StreamDev d, BatchDev b) {
    k_intersect_body<WORK, (int)kColInEntry>(d, b);
}

// Streams whose entries have colour words (one hash group whose colour does not fit the entry: m > 256
// or more than 2^24 nodes): the scan-first path with one hash per entry, and probes for about 1/m of
// the entries.
template <bool WORK>
__global__ void __launch_bounds__(256, REPT_WORDS_BLOCKS) k_intersect_words(StreamDev d, BatchDev b) {
    k_intersect_body<WORK, (int)kColWords>(d, b);
}

// Streams without stored colours (parallel MASCOT with several samplers, or too many groups for a
// word): every probe is issued, so the kernel waits on memory and wants every warp an SM can hold.
template <bool WORK>
__global__ void __launch_bounds__(256, 8) k_intersect_probe(StreamDev d, BatchDev b) {
    k_intersect_body<WORK, (int)kColNone>(d, b);
}

// tau_hat_v = f * sum_i tau_v^(i), f formed in double on the host.
__global__ void k_local_estimates(const unsigned long long* __restrict__ local, uint32_t n, double f,
                                  double* __restrict__ out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = (double)local[v] * f;
}

// tau_hat = f * sum_{i < c_used} tau^(i); one block.
__global__ void k_global_estimate(const unsigned long long* __restrict__ proc, uint32_t c_used, double f,
                                  double* __restrict__ out) {
    __shared__ unsigned long long part[32];
    unsigned long long s = 0;
    for (uint32_t i = threadIdx.x; i < c_used; i += blockDim.x) s += proc[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0ull;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if (threadIdx.x == 0) *out = (double)s * f;
    }
}

}  // namespace
}  // namespace rept
