// Kernels of one REPT batch, in launch order:
//   k_classify  colour every edge (all hash groups), find the edges some
//               processor keeps, count new table entries per node, list the
//               touched nodes                                  (Alg. 1 "if h(u,v)==i")
//   k_plan      size the touched nodes' tables for their new entry counts and
//               reserve pool space for the ones that must be re-allocated
//   k_commit    move re-allocated tables (rehash), publish the new counts
//   k_insert    insert each kept edge (nbr, stream index) into both
//               endpoints' tables                              (Alg. 1 E^(i) <- E^(i) + {(u,v)})
//   k_intersect for every edge t = (u, v): walk the smaller endpoint's table,
//               probe the larger endpoint's table, and count the wedges whose
//               two edges both arrived before t and carry the same kept
//               colour; tally tau^(i), tau_u, tau_v, tau_w      (Alg. 1 UpdateTriangleCNT)
// Counting after inserting is exact because every entry carries its stream
// index and k_intersect only accepts entries with index < t: the state seen by
// edge t is exactly the sequential algorithm's state before t.
#pragma once

#include "rept_common.cuh"

namespace rept {

// Insert (nbr, eidx) into the table of 2^lg slots starting at slot `base`.  Returns false
// only if the table has no empty slot left (impossible while cnt <= capacity / 2).
__device__ __forceinline__ bool table_insert(uint2* pool, unsigned long long base, uint32_t lg, uint32_t nbr,
                                             uint32_t eidx) {
    unsigned long long* p = reinterpret_cast<unsigned long long*>(pool) + base;
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = home_slot(nbr, lg);
    const unsigned long long v = pack_slot(nbr, eidx);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        if (atomicCAS(p + h, kEmptySlot, v) == kEmptySlot) return true;
        h = (h + 1u) & mask;
    }
    return false;
}

__global__ void k_classify(StreamDev d, BatchDev b) {
    if (d.ctrl->status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < b.n;
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
            first_u = atomicAdd(&d.add[u], 1u) == 0u;
            first_v = atomicAdd(&d.add[v], 1u) == 0u;
        }
        unsigned long long o = warp_reserve(&d.ctrl->n_touched, (unsigned)first_u + (unsigned)first_v);
        if (first_u) d.touched[o++] = u;
        if (first_v) d.touched[o] = v;
    }
}

__global__ void k_plan(StreamDev d) {
    if (d.ctrl->status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long n_t = d.ctrl->n_touched;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n_t;
         base += stride) {
        const unsigned long long i = base + lane;
        const bool valid = i < n_t;
        unsigned long long need = 0;
        if (valid) {
            const uint32_t x = d.touched[i];
            const uint32_t cnt = d.meta[x].y, add = d.add[x];
            const uint32_t lg_old = table_lg(cnt), lg_new = table_lg(cnt + add);
            if (lg_new != lg_old) need = (1ull << lg_new) >> 2;
        }
        const unsigned long long rel = warp_reserve(&d.ctrl->need_quads, need);
        if (valid) d.grow_rel[i] = need ? (uint32_t)rel : kNoGrow;
    }
}

// One warp per touched node.
__global__ void k_commit(StreamDev d) {
    const unsigned status = d.ctrl->status;
    const unsigned long long n_t = d.ctrl->n_touched;
    const unsigned long long need = d.ctrl->need_quads, top = d.ctrl->pool_top;
    const bool bad = status != 0u || top + need > d.pool_quads;
    if (status == 0u && bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&d.ctrl->status, kStCapacity);
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long i = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_t;
         i += warps) {
        const uint32_t x = d.touched[i];
        if (!bad) {
            const uint2 m = d.meta[x];
            const uint32_t cnt_new = m.y + d.add[x];
            const uint32_t rel = d.grow_rel[i];
            if (rel != kNoGrow) {
                const unsigned long long new_off = top + rel;
                const uint32_t lg_new = table_lg(cnt_new);
                if (m.y > 0) {
                    const uint32_t old_cap = 1u << table_lg(m.y);
                    const unsigned long long old_base = 4ull * m.x;
                    bool ok = true;
                    for (uint32_t j = lane; j < old_cap; j += 32u) {
                        const uint2 s = d.pool[old_base + j];
                        if (s.x != kEmptyId) ok &= table_insert(d.pool, 4ull * new_off, lg_new, s.x, s.y);
                    }
                    if (!ok) atomicOr(&d.ctrl->status, kStInternal);
                }
                __syncwarp();
                if (lane == 0) d.meta[x] = make_uint2((uint32_t)new_off, cnt_new);
            } else if (lane == 0) {
                d.meta[x].y = cnt_new;
            }
        }
        if (lane == 0) d.add[x] = 0u;
    }
}

__global__ void k_insert(StreamDev d, BatchDev b) {
    Ctrl* ct = d.ctrl;
    const unsigned status = ct->status;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the batch's table space is now in use; reset the per-batch counters
        if (status == 0u) ct->pool_top += ct->need_quads;
        ct->need_quads = 0;
        ct->n_touched = 0;
    }
    if (status) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < b.n;
         base += stride) {
        const unsigned long long e = base + lane;
        const bool valid = e < b.n;
        uint32_t u = 0, v = 0;
        if (valid) { u = b.src[e]; v = b.dst[e]; }
        const bool loop = valid && u == v;
        const bool kept = valid && u != v && kept_by_any(d, u, v);
        if (kept) {
            const uint32_t t = (uint32_t)(b.t0 + e);
            const uint2 mu = d.meta[u], mv = d.meta[v];
            bool ok = table_insert(d.pool, 4ull * mu.x, table_lg(mu.y), v, t);
            ok &= table_insert(d.pool, 4ull * mv.x, table_lg(mv.y), u, t);
            if (!ok) atomicOr(&ct->status, kStInternal);
        }
        warp_reserve(&ct->self_loops, loop ? 1ull : 0ull);
        warp_reserve(&ct->stored, kept ? 1ull : 0ull);
    }
}

// Probe the table (2^lg slots at `base`) for neighbour w.  Returns the entry's stream index,
// or kEmptyId when w is absent; `slots` receives the number of slots read.
__device__ __forceinline__ uint32_t table_find(const uint2* __restrict__ pool, unsigned long long base, uint32_t lg,
                                               uint32_t w, uint32_t& slots) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = home_slot(w, lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint2 s = pool[base + h];
        if (s.x == w) { slots = probe + 1u; return s.y; }
        if (s.x == kEmptyId) { slots = probe + 1u; return kEmptyId; }
        h = (h + 1u) & mask;
    }
    slots = mask + 1u;
    return kEmptyId;
}

// One warp per arriving edge.  Dynamic shared memory: c uint64 counters (tau^(i) of this block).
// WORK = true also tallies the table reads into the control block (for the roofline's byte count).
template <bool WORK>
__global__ void __launch_bounds__(256) k_intersect(StreamDev d, BatchDev b) {
    extern __shared__ unsigned long long s_proc[];
    for (uint32_t i = threadIdx.x; i < d.c; i += blockDim.x) s_proc[i] = 0ull;
    __syncthreads();
    const unsigned status = d.ctrl->status;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long w_entries = 0, w_slots = 0, w_probes = 0, w_pslots = 0, w_wedges = 0, w_counted = 0;
    if (status == 0u) {
        for (unsigned long long e = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < b.n;
             e += warps) {
            const uint32_t u = b.src[e], v = b.dst[e];
            if (u == v) continue;
            const uint32_t t = (uint32_t)(b.t0 + e);
            const uint2 mu = d.meta[u], mv = d.meta[v];
            if (mu.y == 0u || mv.y == 0u) continue;
            const bool u_small = mu.y <= mv.y;
            const uint32_t s = u_small ? u : v, l = u_small ? v : u;
            const uint2 ms = u_small ? mu : mv, ml = u_small ? mv : mu;
            const uint32_t cap_s = 1u << table_lg(ms.y);
            const uint32_t lg_l = table_lg(ml.y);
            const unsigned long long base_s = 4ull * ms.x, base_l = 4ull * ml.x;
            if (WORK && lane == 0) { w_entries += ms.y; w_slots += cap_s; }
            uint32_t total = 0;
            for (uint32_t j0 = 0; j0 < cap_s; j0 += 32u) {
                const uint32_t j = j0 + lane;
                uint32_t found = 0;  // groups in which this wedge counts
                if (j < cap_s) {
                    const uint2 es = d.pool[base_s + j];
                    if (es.x != kEmptyId && es.y < t) {
                        uint32_t nslots = 0;
                        const uint32_t tl = table_find(d.pool, base_l, lg_l, es.x, nslots);
                        if (WORK) { ++w_probes; w_pslots += nslots; }
                        if (tl < t) {  // kEmptyId (absent) is never < t
                            const uint32_t w = es.x;
                            if (WORK) ++w_wedges;
                            for (uint32_t k = 0; k < d.groups; ++k) {
                                const uint64_t sk = group_seed(d.seed, k);
                                const uint32_t js = colour_of(s, w, sk, d.m);
                                if (k * d.m + js < d.c && colour_of(l, w, sk, d.m) == js) {
                                    ++found;
                                    atomicAdd(&s_proc[k * d.m + js], 1ull);
                                }
                            }
                            if (found) atomicAdd(&d.local[w], (unsigned long long)found);
                            if (WORK) w_counted += found;
                        }
                    }
                }
                total += __reduce_add_sync(0xFFFFFFFFu, found);
            }
            if (lane == 0 && total) {
                atomicAdd(&d.local[u], (unsigned long long)total);
                atomicAdd(&d.local[v], (unsigned long long)total);
            }
        }
    }
    if (WORK) {
        for (int o = 16; o > 0; o >>= 1) {
            w_entries += __shfl_down_sync(0xFFFFFFFFu, w_entries, o);
            w_slots += __shfl_down_sync(0xFFFFFFFFu, w_slots, o);
            w_probes += __shfl_down_sync(0xFFFFFFFFu, w_probes, o);
            w_pslots += __shfl_down_sync(0xFFFFFFFFu, w_pslots, o);
            w_wedges += __shfl_down_sync(0xFFFFFFFFu, w_wedges, o);
            w_counted += __shfl_down_sync(0xFFFFFFFFu, w_counted, o);
        }
        if (lane == 0) {
            atomicAdd(&d.ctrl->small_entries, w_entries);
            atomicAdd(&d.ctrl->small_slots, w_slots);
            atomicAdd(&d.ctrl->probes, w_probes);
            atomicAdd(&d.ctrl->probe_slots, w_pslots);
            atomicAdd(&d.ctrl->wedges, w_wedges);
            atomicAdd(&d.ctrl->counted, w_counted);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < d.c; i += blockDim.x)
        if (s_proc[i]) atomicAdd(&d.proc[i], s_proc[i]);
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

}  // namespace rept
