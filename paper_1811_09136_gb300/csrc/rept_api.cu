// C ABI of the REPT streaming counter (declared in include/rept.h): handle
// lifetime, pool sizing, batch launch sequence, estimates.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "rept.h"
#include "rept_common.cuh"
#include "rept_kernels.cuh"

using namespace rept;

namespace {

std::atomic<unsigned long long> g_launches{0};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define REPT_CUDA(call)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) {                          \
            if (_e == cudaErrorMemoryAllocation) {        \
                (void)cudaGetLastError();                 \
                return REPT_E_NOMEM;                      \
            }                                             \
            return REPT_E_CUDA;                           \
        }                                                 \
    } while (0)

#define REPT_LAUNCHED()                                   \
    do {                                                  \
        g_launches.fetch_add(1, std::memory_order_relaxed); \
        if (cudaPeekAtLastError() != cudaSuccess) {       \
            (void)cudaGetLastError();                     \
            return REPT_E_CUDA;                           \
        }                                                 \
    } while (0)

}  // namespace

struct rept_state {
    rept_config cfg{};
    int device = 0;
    int sm_count = 0;
    uint32_t groups = 1;
    StreamDev d{};
    unsigned long long max_batch = 0;
    unsigned long long next_t = 0;  // stream index of the next edge
    Ctrl* h_ctrl = nullptr;         // pinned mirror of the control block
    uint32_t* stage_src = nullptr;  // device staging for rept_ingest_host
    uint32_t* stage_dst = nullptr;
    unsigned long long stage_cap = 0;
    double* d_global = nullptr;
    double* h_global = nullptr;  // pinned
    double* d_local_tmp = nullptr;
    int grid_stream = 0;     // blocks for edge/node-parallel kernels
    int grid_intersect = 0;  // blocks for k_intersect
    size_t device_bytes = 0;
    // REPT_FLAG_PROFILE: event pairs recorded around launches, folded into totals on query
    struct Timed { int kernel; cudaEvent_t start, stop; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> spare_events;
    double kernel_ms[REPT_NUM_KERNELS] = {0};
    unsigned long long kernel_launches[REPT_NUM_KERNELS] = {0};
};

namespace {

int dev_alloc(rept_state* s, void** p, size_t bytes) {
    REPT_CUDA(cudaMalloc(p, bytes));
    s->device_bytes += bytes;
    return REPT_OK;
}

void dev_free(rept_state* s, void* p, size_t bytes) {
    if (p) {
        cudaFree(p);
        s->device_bytes -= bytes;
    }
}

// Pool slots that guarantee no batch can run out: a node's block (table plus list) holds at
// most 8 slots per entry (12 with colour words: 4 + 4 + 4 at one entry, at most 4 + 2 + 1 per entry
// beyond), and its successive blocks form a doubling series bounded by twice the last one, so at
// most 16 (24) slots per stored entry, i.e. 32 (48) slots, 8 (12) quads, per stream edge.
unsigned long long quads_bound(unsigned long long edges, bool words) {
    return (words ? 12ull : 8ull) * edges + 64ull;
}

int grow_pool(rept_state* s, unsigned long long min_quads, cudaStream_t st) {
    unsigned long long want = std::max(min_quads, 2ull * s->d.pool_quads);
    if (want > 0xFFFFFFFFull) want = 0xFFFFFFFFull;  // offsets are 32-bit quads
    if (want < min_quads) return REPT_E_CAPACITY;
    uint2* np = nullptr;
    int rc = dev_alloc(s, (void**)&np, want * 32ull);
    if (rc) return rc;
    REPT_CUDA(cudaStreamSynchronize(st));
    const unsigned long long used = s->h_ctrl->pool_top;
    if (s->d.pool && used) REPT_CUDA(cudaMemcpyAsync(np, s->d.pool, used * 32ull, cudaMemcpyDeviceToDevice, st));
    REPT_CUDA(cudaMemsetAsync((char*)np + used * 32ull, 0xFF, (want - used) * 32ull, st));
    REPT_CUDA(cudaStreamSynchronize(st));
    dev_free(s, s->d.pool, s->d.pool_quads * 32ull);
    s->d.pool = np;
    s->d.pool_quads = want;
    return REPT_OK;
}

int read_ctrl(rept_state* s, cudaStream_t st) {
    REPT_CUDA(cudaMemcpyAsync(s->h_ctrl, s->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    REPT_CUDA(cudaStreamSynchronize(st));
    return REPT_OK;
}

int ensure_batch_scratch(rept_state* s, unsigned long long n, cudaStream_t st) {
    if (n <= s->max_batch) return REPT_OK;
    REPT_CUDA(cudaStreamSynchronize(st));
    const unsigned long long old = s->max_batch;
    dev_free(s, s->d.touched, 2 * old * sizeof(uint32_t));
    dev_free(s, s->d.grow_rel, 2 * old * sizeof(uint32_t));
    dev_free(s, s->d.big, 2 * old * sizeof(uint32_t));
    dev_free(s, s->d.rec, old * sizeof(WorkItem));
    dev_free(s, s->d.srec, old * sizeof(WorkItem));
    s->d.touched = s->d.grow_rel = s->d.big = nullptr;
    s->d.rec = s->d.srec = nullptr;
    int rc = dev_alloc(s, (void**)&s->d.touched, 2 * n * sizeof(uint32_t));
    if (!rc) rc = dev_alloc(s, (void**)&s->d.grow_rel, 2 * n * sizeof(uint32_t));
    if (!rc) rc = dev_alloc(s, (void**)&s->d.big, 2 * n * sizeof(uint32_t));
    if (!rc) rc = dev_alloc(s, (void**)&s->d.rec, n * sizeof(WorkItem));
    if (!rc) rc = dev_alloc(s, (void**)&s->d.srec, n * sizeof(WorkItem));
    if (rc) return rc;
    s->max_batch = n;
    s->d.big_cap = 2 * n;
    return REPT_OK;
}

cudaEvent_t take_event(rept_state* s) {
    if (!s->spare_events.empty()) {
        cudaEvent_t e = s->spare_events.back();
        s->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// NVTX range names of the phases (seen by profilers that record NVTX, e.g. ncu --nvtx); the
// ranges cost a check of a function pointer when no tool is attached.
const char* const kPhaseNames[] = {"rept classify", "rept plan", "rept commit", "rept insert",
                                   "rept intersect", "rept estimate", "rept sort"};
static_assert(sizeof(kPhaseNames) / sizeof(kPhaseNames[0]) == REPT_NUM_KERNELS, "a name per phase");

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Launch `fn` on `st` inside an NVTX range named for the phase; with REPT_FLAG_PROFILE bracket it
// with events on the same stream.
template <class F>
int timed_launch(rept_state* s, int kernel, cudaStream_t st, F&& fn, int kernels_in_fn = 1) {
    NvtxRange range(kPhaseNames[kernel]);
    const bool prof = (s->cfg.flags & REPT_FLAG_PROFILE) != 0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (prof) {
        a = take_event(s);
        b = take_event(s);
        if (!a || !b) return REPT_E_CUDA;
        REPT_CUDA(cudaEventRecord(a, st));
    }
    fn();
    g_launches.fetch_add((unsigned long long)kernels_in_fn, std::memory_order_relaxed);
    s->kernel_launches[kernel] += (unsigned long long)kernels_in_fn;
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return REPT_E_CUDA;
    }
    if (prof) {
        REPT_CUDA(cudaEventRecord(b, st));
        s->timed.push_back({kernel, a, b});
    }
    return REPT_OK;
}

int fold_times(rept_state* s) {
    for (auto& t : s->timed) {
        REPT_CUDA(cudaEventSynchronize(t.stop));
        float ms = 0.f;
        REPT_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
        s->kernel_ms[t.kernel] += ms;
        s->spare_events.push_back(t.start);
        s->spare_events.push_back(t.stop);
    }
    s->timed.clear();
    return REPT_OK;
}

// Pair arrays (Algorithm 2) covering stream indices < edges; grows by copying (synchronises).
int ensure_pair_capacity(rept_state* s, unsigned long long edges, cudaStream_t st) {
    StreamDev& d = s->d;
    if (edges <= d.pair_cap) return REPT_OK;
    const unsigned long long cap = std::max(edges, 2 * d.pair_cap), G = s->groups, old = d.pair_cap;
    uint2* ends = nullptr;
    uint32_t *tau = nullptr, *evt = nullptr, *lst = nullptr;
    int rc = dev_alloc(s, (void**)&ends, cap * sizeof(uint2));
    if (!rc) rc = dev_alloc(s, (void**)&tau, cap * G * sizeof(uint32_t));
    if (!rc) rc = dev_alloc(s, (void**)&evt, cap * G * sizeof(uint32_t));
    if (!rc) rc = dev_alloc(s, (void**)&lst, cap * G * sizeof(uint32_t));
    if (rc) return rc;
    REPT_CUDA(cudaMemsetAsync(tau, 0, cap * G * sizeof(uint32_t), st));
    REPT_CUDA(cudaMemsetAsync(evt, 0, cap * G * sizeof(uint32_t), st));
    if (old) {
        REPT_CUDA(cudaMemcpyAsync(ends, d.edge_ends, old * sizeof(uint2), cudaMemcpyDeviceToDevice, st));
        REPT_CUDA(cudaMemcpyAsync(tau, d.pair_tau, old * G * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    REPT_CUDA(cudaStreamSynchronize(st));
    dev_free(s, d.edge_ends, old * sizeof(uint2));
    dev_free(s, d.pair_tau, old * G * sizeof(uint32_t));
    dev_free(s, d.pair_evt, old * G * sizeof(uint32_t));
    dev_free(s, d.pair_list, old * G * sizeof(uint32_t));
    d.edge_ends = ends;
    d.pair_tau = tau;
    d.pair_evt = evt;
    d.pair_list = lst;
    d.pair_cap = cap;
    return REPT_OK;
}

int launch_batch(rept_state* s, const uint32_t* d_src, const uint32_t* d_dst, unsigned long long n, cudaStream_t st) {
    if (s->d.pair_tau) {
        const int prc = ensure_pair_capacity(s, s->next_t + n, st);
        if (prc) return prc;
    }
    BatchDev b{d_src, d_dst, n, s->next_t};
    const int threads = 256;
    const unsigned long long want_blocks = (n + threads - 1) / threads;
    const int grid = (int)std::min<unsigned long long>(want_blocks, (unsigned long long)s->grid_stream);
    int rc = REPT_OK;
    if ((rc = timed_launch(s, REPT_K_CLASSIFY, st, [&] { k_classify<<<grid, threads, 0, st>>>(s->d, b); })))
        return rc;
    if (s->cfg.flags & REPT_FLAG_CHECK_DUPS) {
        // the set of this batch's edge keys: a power of two >= 2n slots of 8 bytes in the work-record
        // scratch (32 bytes per batch edge, so at most half of it)
        unsigned long long cap = 1;
        while (cap < 2 * n) cap <<= 1;
        REPT_CUDA(cudaMemsetAsync(s->d.rec, 0xFF, cap * sizeof(unsigned long long), st));
        if ((rc = timed_launch(s, REPT_K_CLASSIFY, st, [&] { k_check_dups<<<grid, threads, 0, st>>>(s->d, b, cap - 1); })))
            return rc;
    }
    if ((rc = timed_launch(s, REPT_K_PLAN, st, [&] { k_plan<<<grid, threads, 0, st>>>(s->d); }))) return rc;
    const bool fixed = (s->cfg.flags & REPT_FLAG_FIXED_POOL) != 0;
    if (!fixed && s->d.pool_quads < quads_bound(s->next_t + n, has_words(s->d))) {
        // not provably large enough: read this batch's request and grow if needed
        if ((rc = read_ctrl(s, st))) return rc;
        const unsigned long long need = s->h_ctrl->pool_top + s->h_ctrl->need_quads;
        if (s->h_ctrl->status == 0u && need > s->d.pool_quads) {
            if ((rc = grow_pool(s, need + need / 2 + 1024, st))) return rc;
        }
    }
    if ((rc = timed_launch(s, REPT_K_COMMIT, st, [&] {
             k_commit<<<grid, threads, 0, st>>>(s->d);
             k_rehash_big<<<s->sm_count * 4, threads, 0, st>>>(s->d);
             k_rehash_huge<<<s->sm_count * 2, 1024, 0, st>>>(s->d);
         }, 3)))
        return rc;
    if ((rc = timed_launch(s, REPT_K_INSERT, st, [&] { k_insert<<<grid, threads, 0, st>>>(s->d, b); }))) return rc;
    if ((rc = timed_launch(s, REPT_K_SORT, st, [&] {
             k_sort_scan<<<1, 1024, 0, st>>>(s->d);
             k_sort_scatter<<<grid, threads, 0, st>>>(s->d, b);
         }, 2)))
        return rc;
    const unsigned long long want_i = (n * 8 + 255) / 256;  // work is claimed dynamically; >= 1 block
    const int grid_i = (int)std::min<unsigned long long>(want_i, (unsigned long long)s->grid_intersect);
    const size_t smem = s->cfg.c * sizeof(unsigned long long);
    const bool work = (s->cfg.flags & REPT_FLAG_WORK_COUNTERS) != 0;
    rc = timed_launch(s, REPT_K_INTERSECT, st, [&] {
        if (s->d.colours == kColInEntry) {
            if (work) k_intersect<true><<<grid_i, 256, smem, st>>>(s->d, b);
            else k_intersect<false><<<grid_i, 256, smem, st>>>(s->d, b);
        } else if (s->d.colours == kColWords) {
            if (work) k_intersect_words<true><<<grid_i, 256, smem, st>>>(s->d, b);
            else k_intersect_words<false><<<grid_i, 256, smem, st>>>(s->d, b);
        } else {
            if (work) k_intersect_probe<true><<<grid_i, 256, smem, st>>>(s->d, b);
            else k_intersect_probe<false><<<grid_i, 256, smem, st>>>(s->d, b);
        }
    });
    if (rc) return rc;
    if (s->d.pair_tau &&
        (rc = timed_launch(s, REPT_K_INTERSECT, st, [&] { k_pairs<<<s->sm_count * 4, 256, 0, st>>>(s->d); })))
        return rc;
    s->next_t += n;
    return REPT_OK;
}

// f such that tau_hat = f * (integer sum): m^2 / c for c <= m, m / c1 for c = c1 * m; parallel
// MASCOT averages the samplers' m^2 tau^(i), so m^2 / c for every c.
double estimate_factor(const rept_config& c) {
    const double md = (double)c.m;
    if (c.c <= c.m || (c.flags & REPT_FLAG_MASCOT)) return md * md / (double)c.c;
    return md / (double)(c.c / c.m);
}

// tau_hat into s->d_global: Section III-A / III-B.1 factor, or Algorithm 2's combination.
int enqueue_global_estimate(rept_state* s, cudaStream_t st) {
    if (s->d.local2)
        return timed_launch(s, REPT_K_ESTIMATE, st, [&] {
            k_global_estimate_partial<<<1, 32, 0, st>>>(s->d.proc, s->d.eta_proc, s->cfg.m, s->cfg.c, s->d_global);
        });
    const double f = estimate_factor(s->cfg);
    return timed_launch(s, REPT_K_ESTIMATE, st,
                        [&] { k_global_estimate<<<1, 256, 0, st>>>(s->d.proc, s->cfg.c, f, s->d_global); });
}

int sync_status(rept_state* s, cudaStream_t st) {
    int rc = read_ctrl(s, st);
    if (rc) return rc;
#ifdef REPT_DEBUG_BOUNDS
    report_failed_check(s->h_ctrl->dbg);
#endif
    return status_to_code(s->h_ctrl->status);
}


}  // namespace

extern "C" {

int rept_create(const rept_config* cfg, void* stream, rept_state** out) {
    if (!cfg || !out) return REPT_E_INVAL;
    *out = nullptr;
    if (cfg->m == 0 || cfg->c == 0 || cfg->n_nodes == 0 || cfg->n_nodes == 0xFFFFFFFFu) return REPT_E_INVAL;
    if (cfg->c > kMaxProcessors) return REPT_E_INVAL;
    if (cfg->tile_max != 0 && cfg->tile_max != 4 && cfg->tile_max != 8 && cfg->tile_max != 16 &&
        cfg->tile_max != 32)
        return REPT_E_INVAL;
    if (cfg->reserved != 0 || cfg->reserved2 != 0) return REPT_E_INVAL;
    const bool sharded = cfg->proc_begin != 0 || cfg->proc_end != 0;
    if (sharded && (cfg->proc_begin >= cfg->proc_end || cfg->proc_end > cfg->c)) return REPT_E_INVAL;
    if (sharded && !(cfg->flags & REPT_FLAG_MASCOT) && cfg->c > cfg->m && cfg->c % cfg->m != 0)
        return REPT_E_INVAL;  // Algorithm 2's combination needs every processor's counts
    cudaStream_t st = as_stream(stream);
    rept_state* s = new (std::nothrow) rept_state();
    if (!s) return REPT_E_NOMEM;
    s->cfg = *cfg;
    int rc = REPT_OK;
    auto fail = [&](int code) {
        rept_destroy(s);
        return code;
    };
    if (cudaGetDevice(&s->device) != cudaSuccess) return fail(REPT_E_CUDA);
    if (cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        return fail(REPT_E_CUDA);
    // how list entries carry colours, and the intersection grid: as many blocks as fit at once, for
    // the variant this stream uses
    const bool mascot_flag = (cfg->flags & REPT_FLAG_MASCOT) != 0;
    const uint32_t n_groups = mascot_flag ? cfg->c : (cfg->c + cfg->m - 1) / cfg->m;
    uint32_t cbits = 0;
    while (cbits < 32 && (1ull << cbits) < cfg->m) ++cbits;
    const bool coloured = n_groups == 1 && cfg->m >= 2 && cfg->m <= 256 && cfg->n_nodes <= (1u << kIdBits);
    // colour words: one group that cannot carry its colour in the entries.  With several groups an
    // entry would cost a hash per group, which measured slower than probing every entry: the 5-group
    // Chung-Lu stream's intersection took 404 ms per step with words (scan first, candidate queue)
    // against 162 ms probing.
    const bool words = !coloured && !mascot_flag && cfg->m >= 2 && n_groups == 1;
    const void* k3 = coloured ? (const void*)k_intersect<false>
                              : words ? (const void*)k_intersect_words<false> : (const void*)k_intersect_probe<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3, 256, cfg->c * sizeof(unsigned long long)) !=
        cudaSuccess)
        return fail(REPT_E_CUDA);
    s->grid_intersect = s->sm_count * std::max(per_sm, 1);
    s->grid_stream = s->sm_count * 8;
    const bool mascot = (cfg->flags & REPT_FLAG_MASCOT) != 0;
    s->groups = mascot ? cfg->c : cfg->c <= cfg->m ? 1u : (cfg->c + cfg->m - 1) / cfg->m;
    const uint32_t n = cfg->n_nodes;
    StreamDev& d = s->d;
    d.m = cfg->m;
    d.c = cfg->c;
    d.groups = s->groups;
    d.n_nodes = n;
    d.seed = cfg->seed;
    d.fm = make_fastmod(cfg->m);
    d.tile_max = cfg->tile_max == 0 ? 32u : cfg->tile_max;
    const unsigned long long mb = cfg->max_batch ? cfg->max_batch : (1ull << 20);
    unsigned long long quads = quads_bound(cfg->expected_edges ? cfg->expected_edges : mb, words);
    if (quads > 0xFFFFFFFFull) quads = 0xFFFFFFFFull;
    if ((rc = dev_alloc(s, (void**)&d.meta, (size_t)n * sizeof(uint4)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.cnt_add, (size_t)n * sizeof(uint32_t)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.local, (size_t)n * sizeof(unsigned long long)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.proc, (size_t)cfg->c * sizeof(unsigned long long)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.ctrl, sizeof(Ctrl)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.hist, kSortBuckets * sizeof(uint32_t)))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&d.pool, quads * 32ull))) return fail(rc);
    if ((rc = dev_alloc(s, (void**)&s->d_global, sizeof(double)))) return fail(rc);
    d.pool_quads = quads;
    // one hash group, few colours and ids of at most kIdBits: list entries carry their colour;
    // several groups whose colours fit 32 bits: a colour word per entry
    d.colours = coloured ? kColInEntry : words ? kColWords : kColNone;
    d.cbits = words ? cbits : 0u;
    d.cmask = words ? (uint32_t)((1ull << cbits) - 1ull) : 0u;
    d.c1 = mascot || cfg->c <= cfg->m ? cfg->c : cfg->c / cfg->m;
    d.keep = mascot ? 1u : cfg->m;
    d.pstride = mascot ? 1u : cfg->m;
    d.pbeg = sharded ? cfg->proc_begin : 0u;
    d.pcount = sharded ? cfg->proc_end - cfg->proc_begin : cfg->c;
    d.kbeg = d.pbeg / d.pstride;
    d.kend = (d.pbeg + d.pcount - 1u) / d.pstride + 1u;
    if (cfg->flags & REPT_FLAG_LOCAL_PER_PROCESSOR) {
        if ((rc = dev_alloc(s, (void**)&d.local_proc, (size_t)cfg->c * n * sizeof(unsigned long long))))
            return fail(rc);
    }
    if (!mascot && cfg->c > cfg->m && cfg->c % cfg->m != 0) {
        // Algorithm 2: the partial group's local counts and the triangle-pair counters
        if ((rc = dev_alloc(s, (void**)&d.local2, (size_t)n * sizeof(unsigned long long)))) return fail(rc);
        if ((rc = dev_alloc(s, (void**)&d.eta_proc, (size_t)cfg->c * sizeof(unsigned long long)))) return fail(rc);
        if ((rc = dev_alloc(s, (void**)&d.eta_local, (size_t)n * sizeof(unsigned long long)))) return fail(rc);
        if ((rc = ensure_pair_capacity(s, std::max<unsigned long long>(cfg->expected_edges, mb), st))) return fail(rc);
    }
    if ((rc = ensure_batch_scratch(s, mb, st))) return fail(rc);
    if (cudaMallocHost((void**)&s->h_ctrl, sizeof(Ctrl)) != cudaSuccess) return fail(REPT_E_NOMEM);
    if (cudaMallocHost((void**)&s->h_global, sizeof(double)) != cudaSuccess) return fail(REPT_E_NOMEM);
    memset(s->h_ctrl, 0, sizeof(Ctrl));
    if (cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return fail(REPT_E_CUDA);
    if (cudaMemsetAsync(d.pool, 0xFF, quads * 32ull, st) != cudaSuccess) return fail(REPT_E_CUDA);
    if ((rc = rept_reset(s, stream))) return fail(rc);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(REPT_E_CUDA);
    *out = s;
    return REPT_OK;
}

// The pool itself is not cleared: blocks are handed out again from its start, and each new table
// gets its empty keys when its block is handed out (init_table_keys and the shared-memory builds).
int rept_reset(rept_state* s, void* stream) {
    if (!s) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    StreamDev& d = s->d;
    const size_t n = d.n_nodes;
    REPT_CUDA(cudaMemsetAsync(d.meta, 0, n * sizeof(uint4), st));
    REPT_CUDA(cudaMemsetAsync(d.cnt_add, 0, n * sizeof(uint32_t), st));
    REPT_CUDA(cudaMemsetAsync(d.local, 0, n * sizeof(unsigned long long), st));
    REPT_CUDA(cudaMemsetAsync(d.proc, 0, (size_t)d.c * sizeof(unsigned long long), st));
    if (d.local2) REPT_CUDA(cudaMemsetAsync(d.local2, 0, n * sizeof(unsigned long long), st));
    if (d.eta_local) REPT_CUDA(cudaMemsetAsync(d.eta_local, 0, n * sizeof(unsigned long long), st));
    if (d.eta_proc) REPT_CUDA(cudaMemsetAsync(d.eta_proc, 0, (size_t)d.c * sizeof(unsigned long long), st));
    if (d.pair_tau) {
        REPT_CUDA(cudaMemsetAsync(d.pair_tau, 0, d.pair_cap * s->groups * sizeof(uint32_t), st));
        REPT_CUDA(cudaMemsetAsync(d.pair_evt, 0, d.pair_cap * s->groups * sizeof(uint32_t), st));
    }
    if (d.local_proc) REPT_CUDA(cudaMemsetAsync(d.local_proc, 0, (size_t)d.c * n * sizeof(unsigned long long), st));
    REPT_CUDA(cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), st));
    memset(s->h_ctrl, 0, sizeof(Ctrl));
    s->next_t = 0;
    return REPT_OK;
}

int rept_reset_async(rept_state* s, uint64_t seed, void* stream) {
    if (!s) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    StreamDev& d = s->d;
    s->cfg.seed = seed;
    d.seed = seed;
    const size_t n = d.n_nodes;
    REPT_CUDA(cudaMemsetAsync(d.meta, 0, n * sizeof(uint4), st));
    REPT_CUDA(cudaMemsetAsync(d.cnt_add, 0, n * sizeof(uint32_t), st));
    REPT_CUDA(cudaMemsetAsync(d.local, 0, n * sizeof(unsigned long long), st));
    REPT_CUDA(cudaMemsetAsync(d.proc, 0, (size_t)d.c * sizeof(unsigned long long), st));
    if (d.local2) REPT_CUDA(cudaMemsetAsync(d.local2, 0, n * sizeof(unsigned long long), st));
    if (d.eta_local) REPT_CUDA(cudaMemsetAsync(d.eta_local, 0, n * sizeof(unsigned long long), st));
    if (d.eta_proc) REPT_CUDA(cudaMemsetAsync(d.eta_proc, 0, (size_t)d.c * sizeof(unsigned long long), st));
    if (d.pair_tau) {
        REPT_CUDA(cudaMemsetAsync(d.pair_tau, 0, d.pair_cap * s->groups * sizeof(uint32_t), st));
        REPT_CUDA(cudaMemsetAsync(d.pair_evt, 0, d.pair_cap * s->groups * sizeof(uint32_t), st));
    }
    if (d.local_proc) REPT_CUDA(cudaMemsetAsync(d.local_proc, 0, (size_t)d.c * n * sizeof(unsigned long long), st));
    REPT_CUDA(cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), st));
    s->next_t = 0;
    return REPT_OK;
}

int rept_ingest_batch(rept_state* s, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n, void* stream) {
    if (!s) return REPT_E_INVAL;
    if (n == 0) return REPT_OK;
    if (!d_src || !d_dst) return REPT_E_INVAL;
    if (s->next_t + n >= 0xFFFFFFFEull) return REPT_E_INVAL;  // stream indices stay below 2^32 - 2
    cudaStream_t st = as_stream(stream);
    int rc = ensure_batch_scratch(s, n, st);
    if (rc) return rc;
    rc = launch_batch(s, d_src, d_dst, n, st);
    if (rc) return rc;
    if (s->cfg.flags & REPT_FLAG_SYNC) return sync_status(s, st);
    return REPT_OK;
}

int rept_ingest_host(rept_state* s, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n, uint64_t batch,
                     void* stream) {
    if (!s) return REPT_E_INVAL;
    if (n == 0) return REPT_OK;
    if (!h_src || !h_dst) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    const unsigned long long chunk = batch ? batch : s->max_batch;
    int rc = ensure_batch_scratch(s, chunk, st);
    if (rc) return rc;
    if (s->stage_cap < chunk) {
        REPT_CUDA(cudaStreamSynchronize(st));
        dev_free(s, s->stage_src, s->stage_cap * sizeof(uint32_t));
        dev_free(s, s->stage_dst, s->stage_cap * sizeof(uint32_t));
        s->stage_src = s->stage_dst = nullptr;
        s->stage_cap = 0;
        if ((rc = dev_alloc(s, (void**)&s->stage_src, chunk * sizeof(uint32_t)))) return rc;
        if ((rc = dev_alloc(s, (void**)&s->stage_dst, chunk * sizeof(uint32_t)))) return rc;
        s->stage_cap = chunk;
    }
    for (unsigned long long off = 0; off < n; off += chunk) {
        const unsigned long long k = std::min<unsigned long long>(chunk, n - off);
        REPT_CUDA(cudaMemcpyAsync(s->stage_src, h_src + off, k * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        REPT_CUDA(cudaMemcpyAsync(s->stage_dst, h_dst + off, k * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        if (s->next_t + k >= 0xFFFFFFFEull) return REPT_E_INVAL;
        rc = launch_batch(s, s->stage_src, s->stage_dst, k, st);
        if (rc) return rc;
    }
    REPT_CUDA(cudaStreamSynchronize(st));
    if (s->cfg.flags & REPT_FLAG_SYNC) return sync_status(s, st);
    return REPT_OK;
}

int rept_estimates(rept_state* s, double* h_global, double* d_local, void* stream) {
    if (!s || !h_global) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    int rc0 = enqueue_global_estimate(s, st);
    if (rc0) return rc0;
    if (d_local) {
        if (s->d.local2) {
            rc0 = timed_launch(s, REPT_K_ESTIMATE, st, [&] {
                k_local_estimates_partial<<<s->sm_count * 4, 256, 0, st>>>(s->d.local, s->d.local2, s->d.eta_local,
                                                                           s->d.n_nodes, s->cfg.m, s->cfg.c, d_local);
            });
        } else {
            const double f = estimate_factor(s->cfg);
            rc0 = timed_launch(s, REPT_K_ESTIMATE, st, [&] {
                k_local_estimates<<<s->sm_count * 4, 256, 0, st>>>(s->d.local, s->d.n_nodes, f, d_local);
            });
        }
        if (rc0) return rc0;
    }
    REPT_CUDA(cudaMemcpyAsync(s->h_global, s->d_global, sizeof(double), cudaMemcpyDeviceToHost, st));
    int rc = sync_status(s, st);
    *h_global = *s->h_global;
    return rc;
}

int rept_estimates_async(rept_state* s, double* h_global, uint64_t* h_proc, uint32_t* h_status, void* stream) {
    if (!s || !h_global || !h_status) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    int rc = enqueue_global_estimate(s, st);
    if (rc) return rc;
    REPT_CUDA(cudaMemcpyAsync(h_global, s->d_global, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (h_proc)
        REPT_CUDA(cudaMemcpyAsync(h_proc, s->d.proc, (size_t)s->cfg.c * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                  st));
    REPT_CUDA(cudaMemcpyAsync(h_status, &s->d.ctrl->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    return REPT_OK;
}

int rept_estimates_host(rept_state* s, double* h_global, double* h_local, void* stream) {
    if (!s || !h_global) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    double* dl = nullptr;
    if (h_local) {
        if (!s->d_local_tmp) {
            int rc = dev_alloc(s, (void**)&s->d_local_tmp, (size_t)s->d.n_nodes * sizeof(double));
            if (rc) return rc;
        }
        dl = s->d_local_tmp;
    }
    int rc = rept_estimates(s, h_global, dl, stream);
    if (h_local) {
        REPT_CUDA(cudaMemcpyAsync(h_local, dl, (size_t)s->d.n_nodes * sizeof(double), cudaMemcpyDeviceToHost, st));
        REPT_CUDA(cudaStreamSynchronize(st));
    }
    return rc;
}

int rept_counts(rept_state* s, uint64_t* h_proc, uint64_t* d_local, void* stream) {
    if (!s) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    if (h_proc)
        REPT_CUDA(cudaMemcpyAsync(h_proc, s->d.proc, (size_t)s->cfg.c * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                  st));
    if (d_local) {
        if (s->d.local2) {
            k_add_local<<<s->sm_count * 4, 256, 0, st>>>(s->d.local, s->d.local2, s->d.n_nodes,
                                                        reinterpret_cast<unsigned long long*>(d_local));
            g_launches.fetch_add(1, std::memory_order_relaxed);
        } else {
            REPT_CUDA(cudaMemcpyAsync(d_local, s->d.local, (size_t)s->d.n_nodes * sizeof(uint64_t),
                                      cudaMemcpyDeviceToDevice, st));
        }
    }
    return sync_status(s, st);
}

namespace {

struct SnapHeader {
    uint64_t magic, version;
    uint64_t m, c, seed, n_nodes, flags, groups;
    uint64_t next_t, pool_top, self_loops, stored;
    uint64_t proc_begin, proc_end;
};
constexpr uint64_t kSnapMagic = 0x5245505453544154ull;  // "REPTSTAT"
// 3: a table bucket holds its 4 ids and then their 4 stream indices (2: ids and indices in two arrays)
constexpr uint64_t kSnapVersion = 3;

// The arrays of a snapshot after the header, in order: {device pointer, bytes}.
struct SnapPart {
    void* ptr;
    unsigned long long bytes;
};

int snap_parts(rept_state* s, unsigned long long pool_top, SnapPart* parts, int* np) {
    StreamDev& d = s->d;
    const unsigned long long n = d.n_nodes, c = d.c, G = s->groups, T = s->next_t;
    int k = 0;
    parts[k++] = {d.meta, n * sizeof(uint4)};
    parts[k++] = {d.local, n * 8ull};
    parts[k++] = {d.proc, c * 8ull};
    parts[k++] = {d.pool, pool_top * 32ull};
    if (d.local2) {
        parts[k++] = {d.local2, n * 8ull};
        parts[k++] = {d.eta_proc, c * 8ull};
        parts[k++] = {d.eta_local, n * 8ull};
        parts[k++] = {d.edge_ends, T * sizeof(uint2)};
        parts[k++] = {d.pair_tau, T * G * 4ull};
    }
    if (d.local_proc) parts[k++] = {d.local_proc, c * n * 8ull};
    *np = k;
    return REPT_OK;
}

}  // namespace

int rept_snapshot_size(rept_state* s, uint64_t* bytes, void* stream) {
    if (!s || !bytes) return REPT_E_INVAL;
    int rc = sync_status(s, as_stream(stream));
    if (rc) return rc;
    SnapPart parts[16];
    int np = 0;
    snap_parts(s, s->h_ctrl->pool_top, parts, &np);
    unsigned long long total = sizeof(SnapHeader);
    for (int i = 0; i < np; ++i) total += parts[i].bytes;
    *bytes = total;
    return REPT_OK;
}

int rept_snapshot(rept_state* s, void* h_buf, uint64_t bytes, void* stream) {
    if (!s || !h_buf) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    int rc = sync_status(s, st);
    if (rc) return rc;
    SnapPart parts[16];
    int np = 0;
    snap_parts(s, s->h_ctrl->pool_top, parts, &np);
    unsigned long long total = sizeof(SnapHeader);
    for (int i = 0; i < np; ++i) total += parts[i].bytes;
    if (bytes < total) return REPT_E_INVAL;
    SnapHeader h{kSnapMagic, kSnapVersion, s->cfg.m, s->cfg.c, s->cfg.seed, s->cfg.n_nodes, s->cfg.flags, s->groups,
                 s->next_t, s->h_ctrl->pool_top, s->h_ctrl->self_loops, s->h_ctrl->stored,
                 s->cfg.proc_begin, s->cfg.proc_end};
    std::memcpy(h_buf, &h, sizeof(h));
    char* out = static_cast<char*>(h_buf) + sizeof(h);
    for (int i = 0; i < np; ++i) {
        if (parts[i].bytes) REPT_CUDA(cudaMemcpyAsync(out, parts[i].ptr, parts[i].bytes, cudaMemcpyDeviceToHost, st));
        out += parts[i].bytes;
    }
    REPT_CUDA(cudaStreamSynchronize(st));
    return REPT_OK;
}

int rept_restore(rept_state* s, const void* h_buf, uint64_t bytes, void* stream) {
    if (!s || !h_buf || bytes < sizeof(SnapHeader)) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    SnapHeader h;
    std::memcpy(&h, h_buf, sizeof(h));
    if (h.magic != kSnapMagic || h.version != kSnapVersion || h.m != s->cfg.m || h.c != s->cfg.c || h.seed != s->cfg.seed ||
        h.n_nodes != s->cfg.n_nodes || h.flags != s->cfg.flags || h.groups != s->groups ||
        h.proc_begin != s->cfg.proc_begin || h.proc_end != s->cfg.proc_end)
        return REPT_E_INVAL;
    int rc = rept_reset(s, stream);
    if (rc) return rc;
    if (h.pool_top > s->d.pool_quads && (rc = grow_pool(s, h.pool_top, st))) return rc;
    s->next_t = h.next_t;
    if (s->d.local2 && (rc = ensure_pair_capacity(s, std::max<unsigned long long>(h.next_t, 1), st))) return rc;
    SnapPart parts[16];
    int np = 0;
    snap_parts(s, h.pool_top, parts, &np);
    unsigned long long total = sizeof(SnapHeader);
    for (int i = 0; i < np; ++i) total += parts[i].bytes;
    if (bytes < total) return REPT_E_INVAL;
    const char* in = static_cast<const char*>(h_buf) + sizeof(h);
    for (int i = 0; i < np; ++i) {
        if (parts[i].bytes) REPT_CUDA(cudaMemcpyAsync(parts[i].ptr, in, parts[i].bytes, cudaMemcpyHostToDevice, st));
        in += parts[i].bytes;
    }
    // control block: the pool in use and the tallies; every per-batch counter starts at zero
    Ctrl c{};
    c.pool_top = h.pool_top;
    c.self_loops = h.self_loops;
    c.stored = h.stored;
    std::memcpy(s->h_ctrl, &c, sizeof(Ctrl));
    REPT_CUDA(cudaMemcpyAsync(s->d.ctrl, s->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    REPT_CUDA(cudaStreamSynchronize(st));
    return REPT_OK;
}

int rept_local_per_processor(rept_state* s, uint64_t* d_out, void* stream) {
    if (!s || !d_out || !s->d.local_proc) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    REPT_CUDA(cudaMemcpyAsync(d_out, s->d.local_proc, (size_t)s->cfg.c * s->d.n_nodes * sizeof(uint64_t),
                              cudaMemcpyDeviceToDevice, st));
    return sync_status(s, st);
}

int rept_pair_counts(rept_state* s, uint64_t* h_eta_proc, uint64_t* d_eta_local, uint64_t* d_local1,
                     uint64_t* d_local2, void* stream) {
    if (!s) return REPT_E_INVAL;
    if (!s->d.local2) return REPT_E_INVAL;
    cudaStream_t st = as_stream(stream);
    const size_t n = s->d.n_nodes;
    if (h_eta_proc)
        REPT_CUDA(cudaMemcpyAsync(h_eta_proc, s->d.eta_proc, (size_t)s->cfg.c * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, st));
    if (d_eta_local)
        REPT_CUDA(cudaMemcpyAsync(d_eta_local, s->d.eta_local, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    if (d_local1) REPT_CUDA(cudaMemcpyAsync(d_local1, s->d.local, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    if (d_local2) REPT_CUDA(cudaMemcpyAsync(d_local2, s->d.local2, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    return sync_status(s, st);
}

int rept_get_stats(rept_state* s, rept_stats* out, void* stream) {
    if (!s || !out) return REPT_E_INVAL;
    int rc = sync_status(s, as_stream(stream));
    out->edges = s->next_t;
    out->self_loops = s->h_ctrl->self_loops;
    out->stored_edges = s->h_ctrl->stored;
    out->pool_slots = 4ull * s->d.pool_quads;
    out->pool_used = 4ull * s->h_ctrl->pool_top;
    out->device_bytes = s->device_bytes;
    out->small_entries = s->h_ctrl->small_entries;
    out->small_slots = s->h_ctrl->small_slots;
    out->probes = s->h_ctrl->probes;
    out->probe_slots = s->h_ctrl->probe_slots;
    out->wedges = s->h_ctrl->wedges;
    out->counted = s->h_ctrl->counted;
    for (int c = 0; c < kBins; ++c) {
        out->class_items[c] = s->h_ctrl->class_items[c];
        out->class_probes[c] = s->h_ctrl->class_probes[c];
        out->class_cycles[c] = s->h_ctrl->class_cycles[c];
    }
    return rc;
}

int rept_kernel_times(rept_state* s, double* ms, uint64_t* launches, int clear) {
    if (!s || !(s->cfg.flags & REPT_FLAG_PROFILE)) return REPT_E_INVAL;
    int rc = fold_times(s);
    if (rc) return rc;
    for (int k = 0; k < REPT_NUM_KERNELS; ++k) {
        if (ms) ms[k] = s->kernel_ms[k];
        if (launches) launches[k] = s->kernel_launches[k];
        if (clear) {
            s->kernel_ms[k] = 0.0;
            s->kernel_launches[k] = 0;
        }
    }
    return REPT_OK;
}

int rept_sync(rept_state* s, void* stream) {
    if (!s) return REPT_E_INVAL;
    return sync_status(s, as_stream(stream));
}

void rept_destroy(rept_state* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    StreamDev& d = s->d;
    cudaFree(d.meta);
    cudaFree(d.cnt_add);
    cudaFree(d.local);
    cudaFree(d.proc);
    cudaFree(d.ctrl);
    cudaFree(d.pool);
    cudaFree(d.touched);
    cudaFree(d.grow_rel);
    cudaFree(d.big);
    cudaFree(d.rec);
    cudaFree(d.srec);
    cudaFree(d.local2);
    cudaFree(d.eta_proc);
    cudaFree(d.eta_local);
    cudaFree(d.edge_ends);
    cudaFree(d.pair_tau);
    cudaFree(d.pair_evt);
    cudaFree(d.pair_list);
    cudaFree(d.local_proc);
    cudaFree(d.hist);
    cudaFree(s->stage_src);
    cudaFree(s->stage_dst);
    cudaFree(s->d_global);
    cudaFree(s->d_local_tmp);
    for (auto& t : s->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (auto e : s->spare_events) cudaEventDestroy(e);
    if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
    if (s->h_global) cudaFreeHost(s->h_global);
    delete s;
}

}  // extern "C"

namespace rept {
namespace {

// Pool requests of k streams after k_plan: {pool_top, need_quads, status} per stream.
__global__ void k_gather_requests(const StreamDev* __restrict__ ds, uint32_t k, unsigned long long* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) {
        const Ctrl* c = ds[i].ctrl;
        out[3 * i] = c->pool_top;
        out[3 * i + 1] = c->need_quads;
        out[3 * i + 2] = c->status;
    }
}

}  // namespace
}  // namespace rept

struct rept_group {
    uint32_t max_streams = 0, flags = 0;
    int sm_count = 0, intersect_per_sm = 1;
    StreamDev* d_sd = nullptr;  // device descriptor arrays read by the _multi kernels
    BatchDev* d_bd = nullptr;
    unsigned long long* d_req = nullptr;
    unsigned long long* d_pref = nullptr;    // [kBins * (max_streams + 1)] item prefixes (k_group_prefix)
    unsigned long long* d_cursor = nullptr;  // [kBins] claim cursors of k_intersect_group
    // two pinned staging slots, so that a replayed graph's descriptor copy never races the host
    StreamDev* h_sd[2] = {nullptr, nullptr};
    BatchDev* h_bd[2] = {nullptr, nullptr};
    unsigned long long* h_req = nullptr;
    cudaEvent_t slot_done[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    unsigned long long shape[2][6] = {{0}};  // what each slot's graph was captured for
    int slot = 0;
    cudaStream_t capture = nullptr;  // private stream the graphs are captured on (the legacy stream cannot be)
    // REPT_GROUP_PERSISTENT: the grid barrier state, its per-launch initial value (pinned), and the
    // co-resident grid of k_group_persistent
    GroupSync* d_sync = nullptr;
    GroupSync* h_sync = nullptr;
    int persist_grid = 0;
    bool persist_graph_ok = true;  // a captured cooperative launch instantiated (else launched directly)
};

namespace {

struct GroupShape {
    uint32_t k;
    int x_edge, x_big, x_huge, x_int;
    size_t smem;
};

// Enqueue the batch path for all k streams: one launch per step.  With `split`, stop after
// k_plan (the caller reads the pool requests, grows pools, and calls again with split = 2).
int enqueue_group(rept_group* g, const GroupShape& sh, cudaStream_t st, int part) {
    const dim3 blk(256);
    const uint32_t k = sh.k;
    if (part != 2) {
        k_classify_multi<<<dim3(sh.x_edge, k), blk, 0, st>>>(g->d_sd, g->d_bd);
        k_plan_multi<<<dim3(sh.x_edge, k), blk, 0, st>>>(g->d_sd, g->d_bd);
    }
    if (part != 1) {
        k_commit_multi<<<dim3(sh.x_edge, k), blk, 0, st>>>(g->d_sd, g->d_bd);
        k_rehash_big_multi<<<dim3(sh.x_big, k), blk, 0, st>>>(g->d_sd, g->d_bd);
        k_rehash_huge_multi<<<dim3(sh.x_huge, k), dim3(1024), 0, st>>>(g->d_sd, g->d_bd);
        k_insert_multi<<<dim3(sh.x_edge, k), blk, 0, st>>>(g->d_sd, g->d_bd);
        k_sort_scan_multi<<<dim3(1, k), dim3(1024), 0, st>>>(g->d_sd, g->d_bd);
        k_sort_scatter_multi<<<dim3(sh.x_edge, k), blk, 0, st>>>(g->d_sd, g->d_bd);
        // one grid for all streams' intersection work
        k_group_prefix<<<1, 1024, 0, st>>>(g->d_sd, k, g->d_pref, g->d_cursor);
        k_intersect_group<<<g->intersect_per_sm * g->sm_count, blk, 0, st>>>(g->d_sd, k, g->d_pref, g->d_cursor);
    }
    const int launched = part == 1 ? 2 : (part == 2 ? 8 : 10);
    g_launches.fetch_add((unsigned long long)launched, std::memory_order_relaxed);
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return REPT_E_CUDA;
    }
    return REPT_OK;
}

// Time a grid-wide wait of the persistent kernel may take before it gives up: far above any step
// (a step of a 2^20-edge batch takes milliseconds), or 0.1 s under REPT_GROUP_TEST_TIMEOUT.
constexpr unsigned long long kPersistWaitNs = 20ull * 1000 * 1000 * 1000;
constexpr unsigned long long kTestWaitNs = 100ull * 1000 * 1000;

// Enqueue one round as a single cooperative launch: the barrier state is reset from pinned memory
// first (a previous launch that gave up may have left it mid-barrier).
int enqueue_persistent(rept_group* g, const GroupShape& sh, cudaStream_t st) {
    REPT_CUDA(cudaMemcpyAsync(g->d_sync, g->h_sync, sizeof(GroupSync), cudaMemcpyHostToDevice, st));
    const StreamDev* ds = g->d_sd;
    const BatchDev* bs = g->d_bd;
    uint32_t k = sh.k;
    PersistShape ps{(uint32_t)sh.x_edge, (uint32_t)sh.x_big, (uint32_t)sh.x_huge};
    unsigned long long* pref = g->d_pref;
    unsigned long long* cursor = g->d_cursor;
    GroupSync* gs = g->d_sync;
    unsigned long long wait_ns = (g->flags & REPT_GROUP_TEST_TIMEOUT) ? kTestWaitNs : kPersistWaitNs;
    void* args[] = {&ds, &bs, &k, &ps, &pref, &cursor, &gs, &wait_ns};
    REPT_CUDA(cudaLaunchCooperativeKernel((const void*)k_group_persistent, dim3(g->persist_grid), dim3(256), args,
                                          kPersistSmemWords * sizeof(uint32_t), st));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return REPT_OK;
}

}  // namespace

extern "C" {

int rept_group_create(uint32_t max_streams, uint32_t flags, rept_group** out) {
    if (!out || max_streams == 0 || max_streams > 65535u) return REPT_E_INVAL;
    if ((flags & REPT_GROUP_TEST_TIMEOUT) && !(flags & REPT_GROUP_PERSISTENT)) return REPT_E_INVAL;
    *out = nullptr;
    rept_group* g = new (std::nothrow) rept_group();
    if (!g) return REPT_E_NOMEM;
    g->max_streams = max_streams;
    g->flags = flags;
    auto fail = [&](int code) {
        rept_group_destroy(g);
        return code;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(REPT_E_CUDA);
    if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(REPT_E_CUDA);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_intersect_group, 256, 0) != cudaSuccess)
        return fail(REPT_E_CUDA);
    g->intersect_per_sm = std::max(per_sm, 1);
    if (cudaMalloc(&g->d_sd, max_streams * sizeof(StreamDev)) != cudaSuccess) return fail(REPT_E_NOMEM);
    if (cudaMalloc(&g->d_bd, max_streams * sizeof(BatchDev)) != cudaSuccess) return fail(REPT_E_NOMEM);
    if (cudaMalloc(&g->d_req, 3ull * max_streams * sizeof(unsigned long long)) != cudaSuccess)
        return fail(REPT_E_NOMEM);
    if (cudaMalloc(&g->d_pref, (unsigned long long)kBins * (max_streams + 1) * sizeof(unsigned long long)) !=
        cudaSuccess)
        return fail(REPT_E_NOMEM);
    if (cudaMalloc(&g->d_cursor, kBins * sizeof(unsigned long long)) != cudaSuccess) return fail(REPT_E_NOMEM);
    for (int i = 0; i < 2; ++i) {
        if (cudaMallocHost(&g->h_sd[i], max_streams * sizeof(StreamDev)) != cudaSuccess) return fail(REPT_E_NOMEM);
        if (cudaMallocHost(&g->h_bd[i], max_streams * sizeof(BatchDev)) != cudaSuccess) return fail(REPT_E_NOMEM);
        if (cudaEventCreateWithFlags(&g->slot_done[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(REPT_E_CUDA);
    }
    if (cudaMallocHost(&g->h_req, 3ull * max_streams * sizeof(unsigned long long)) != cudaSuccess)
        return fail(REPT_E_NOMEM);
    if ((flags & REPT_GROUP_GRAPH) && cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking) != cudaSuccess)
        return fail(REPT_E_CUDA);
    if (flags & REPT_GROUP_PERSISTENT) {
        int coop = 0, per_sm_p = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
            return fail(REPT_E_CUDA);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, k_group_persistent, 256,
                                                          kPersistSmemWords * sizeof(uint32_t)) != cudaSuccess ||
            per_sm_p < 1)
            return fail(REPT_E_CUDA);
        g->persist_grid = g->sm_count * per_sm_p;
        if (cudaMalloc(&g->d_sync, sizeof(GroupSync)) != cudaSuccess) return fail(REPT_E_NOMEM);
        if (cudaMallocHost(&g->h_sync, sizeof(GroupSync)) != cudaSuccess) return fail(REPT_E_NOMEM);
        *g->h_sync = GroupSync{0u, 0u, 0u, (flags & REPT_GROUP_TEST_TIMEOUT) ? 1u : 0u};
    }
    *out = g;
    return REPT_OK;
}

void rept_group_destroy(rept_group* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i) {
        if (g->exec[i]) cudaGraphExecDestroy(g->exec[i]);
        if (g->slot_done[i]) cudaEventDestroy(g->slot_done[i]);
        if (g->h_sd[i]) cudaFreeHost(g->h_sd[i]);
        if (g->h_bd[i]) cudaFreeHost(g->h_bd[i]);
    }
    if (g->h_req) cudaFreeHost(g->h_req);
    if (g->h_sync) cudaFreeHost(g->h_sync);
    cudaFree(g->d_sync);
    if (g->capture) cudaStreamDestroy(g->capture);
    cudaFree(g->d_sd);
    cudaFree(g->d_bd);
    cudaFree(g->d_req);
    cudaFree(g->d_pref);
    cudaFree(g->d_cursor);
    delete g;
}

int rept_group_ingest(rept_group* g, rept_state* const* hs, const uint32_t* const* d_src,
                      const uint32_t* const* d_dst, const uint64_t* n, uint32_t k, void* stream) {
    if (!g || !hs || !d_src || !d_dst || !n || k == 0 || k > g->max_streams) return REPT_E_INVAL;
    NvtxRange range("rept group ingest");
    cudaStream_t st = as_stream(stream);
    unsigned long long max_n = 0;
    uint32_t max_c = 1;
    bool guaranteed = true;
    for (uint32_t i = 0; i < k; ++i) {
        rept_state* s = hs[i];
        if (!s || s->d.local2) return REPT_E_INVAL;  // c mod m != 0 is served by the single-stream path
        if (n[i] && (!d_src[i] || !d_dst[i])) return REPT_E_INVAL;
        if (s->next_t + n[i] >= 0xFFFFFFFEull) return REPT_E_INVAL;
        int rc = ensure_batch_scratch(s, std::max<unsigned long long>(n[i], 1ull), st);
        if (rc) return rc;
        max_n = std::max<unsigned long long>(max_n, n[i]);
        max_c = std::max(max_c, s->cfg.c);
        const bool fixed = (s->cfg.flags & REPT_FLAG_FIXED_POOL) != 0;
        if (!fixed && s->d.pool_quads < quads_bound(s->next_t + n[i], has_words(s->d))) guaranteed = false;
    }
    // launch shape: the edge kernels cover the largest batch, the rest share the SMs between streams
    GroupShape sh{};
    sh.k = k;
    const unsigned long long pow2 = max_n <= 256 ? 256ull : (1ull << (64 - __builtin_clzll(max_n - 1)));
    const int per_stream_cap = std::max(2, (8 * g->sm_count + (int)k - 1) / (int)k);
    sh.x_edge = (int)std::min<unsigned long long>((pow2 + 255) / 256, (unsigned long long)per_stream_cap);
    sh.x_big = std::max(1, 4 * g->sm_count / (int)k);
    sh.x_huge = std::max(1, 2 * g->sm_count / (int)k);
    sh.x_int = std::max(1, g->intersect_per_sm * g->sm_count / (int)k);
    sh.smem = (size_t)max_c * sizeof(unsigned long long);

    const int slot = g->slot;
    g->slot ^= 1;
    if (cudaEventSynchronize(g->slot_done[slot]) != cudaSuccess) return REPT_E_CUDA;  // slot free again
    StreamDev* hsd = g->h_sd[slot];
    BatchDev* hbd = g->h_bd[slot];
    for (uint32_t i = 0; i < k; ++i) {
        hsd[i] = hs[i]->d;
        hbd[i] = BatchDev{d_src[i], d_dst[i], n[i], hs[i]->next_t};
    }
    auto upload = [&]() -> int {
        REPT_CUDA(cudaMemcpyAsync(g->d_sd, hsd, k * sizeof(StreamDev), cudaMemcpyHostToDevice, st));
        REPT_CUDA(cudaMemcpyAsync(g->d_bd, hbd, k * sizeof(BatchDev), cudaMemcpyHostToDevice, st));
        return REPT_OK;
    };
    int rc = REPT_OK;
    if (!guaranteed) {
        // classify + plan, read every stream's pool request, grow the pools that need it, go on
        if ((rc = upload())) return rc;
        if ((rc = enqueue_group(g, sh, st, 1))) return rc;
        k_gather_requests<<<(k + 255) / 256, 256, 0, st>>>(g->d_sd, k, g->d_req);
        REPT_CUDA(cudaMemcpyAsync(g->h_req, g->d_req, 3ull * k * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  st));
        REPT_CUDA(cudaStreamSynchronize(st));
        bool grew = false;
        for (uint32_t i = 0; i < k; ++i) {
            rept_state* s = hs[i];
            const unsigned long long top = g->h_req[3 * i], need = g->h_req[3 * i + 1];
            const bool fixed = (s->cfg.flags & REPT_FLAG_FIXED_POOL) != 0;
            if (!fixed && g->h_req[3 * i + 2] == 0 && top + need > s->d.pool_quads) {
                s->h_ctrl->pool_top = top;
                if ((rc = grow_pool(s, top + need + (top + need) / 2 + 1024, st))) return rc;
                hsd[i] = s->d;
                grew = true;
            }
        }
        if (grew) REPT_CUDA(cudaMemcpyAsync(g->d_sd, hsd, k * sizeof(StreamDev), cudaMemcpyHostToDevice, st));
        if ((rc = enqueue_group(g, sh, st, 2))) return rc;
    } else if ((g->flags & REPT_GROUP_PERSISTENT) && !((g->flags & REPT_GROUP_GRAPH) && g->persist_graph_ok)) {
        if ((rc = upload())) return rc;
        if ((rc = enqueue_persistent(g, sh, st))) return rc;
    } else if (g->flags & REPT_GROUP_GRAPH) {
        const bool persistent = (g->flags & REPT_GROUP_PERSISTENT) != 0;
        const unsigned long long key[6] = {k, (unsigned long long)sh.x_edge, (unsigned long long)sh.x_big,
                                           (unsigned long long)sh.x_huge, (unsigned long long)sh.x_int, sh.smem};
        bool same = g->exec[slot] != nullptr;
        for (int j = 0; j < 6 && same; ++j) same = g->shape[slot][j] == key[j];
        if (!same) {
            if (g->exec[slot]) {
                cudaGraphExecDestroy(g->exec[slot]);
                g->exec[slot] = nullptr;
            }
            // capture on the private stream (nothing runs), replay on the caller's
            cudaGraph_t graph = nullptr;
            cudaStream_t cs = g->capture;
            REPT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int rc_cap = REPT_OK;
            if (cudaMemcpyAsync(g->d_sd, hsd, k * sizeof(StreamDev), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
                cudaMemcpyAsync(g->d_bd, hbd, k * sizeof(BatchDev), cudaMemcpyHostToDevice, cs) != cudaSuccess)
                rc_cap = REPT_E_CUDA;
            const unsigned long long before = g_launches.load(std::memory_order_relaxed);
            if (!rc_cap) rc_cap = persistent ? enqueue_persistent(g, sh, cs) : enqueue_group(g, sh, cs, 0);
            const cudaError_t e_end = cudaStreamEndCapture(cs, &graph);
            cudaError_t e_inst = cudaErrorUnknown;
            if (!rc_cap && e_end == cudaSuccess) e_inst = cudaGraphInstantiate(&g->exec[slot], graph, 0);
            if (graph) cudaGraphDestroy(graph);
            g_launches.store(before, std::memory_order_relaxed);  // captured, not launched
            if (persistent && (rc_cap || e_end != cudaSuccess || e_inst != cudaSuccess)) {
                // a cooperative launch that cannot be captured: launch it directly from now on
                (void)cudaGetLastError();
                g->exec[slot] = nullptr;
                g->persist_graph_ok = false;
                if ((rc = upload())) return rc;
                if ((rc = enqueue_persistent(g, sh, st))) return rc;
                REPT_CUDA(cudaEventRecord(g->slot_done[slot], st));
                for (uint32_t i = 0; i < k; ++i) hs[i]->next_t += n[i];
                return REPT_OK;
            }
            if (rc_cap) return rc_cap;
            if (e_end != cudaSuccess || e_inst != cudaSuccess) return REPT_E_CUDA;
            for (int j = 0; j < 6; ++j) g->shape[slot][j] = key[j];
        }
        REPT_CUDA(cudaGraphLaunch(g->exec[slot], st));
        g_launches.fetch_add(persistent ? 1 : 10, std::memory_order_relaxed);
    } else {
        if ((rc = upload())) return rc;
        if ((rc = enqueue_group(g, sh, st, 0))) return rc;
    }
    REPT_CUDA(cudaEventRecord(g->slot_done[slot], st));
    for (uint32_t i = 0; i < k; ++i) hs[i]->next_t += n[i];
    return REPT_OK;
}

// rept_ingest_multi: one library-owned group per device, grown (recreated) when a call brings more
// streams than it was made for.
namespace {
std::mutex g_multi_lock;
std::vector<rept_group*> g_multi_groups;  // indexed by device
}  // namespace

int rept_ingest_multi(rept_state* const* hs, const uint32_t* const* d_src, const uint32_t* const* d_dst,
                      const uint64_t* n, uint32_t k, void* stream) {
    if (!hs || !d_src || !d_dst || !n || k == 0) return REPT_E_INVAL;
    int dev = 0;
    REPT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_multi_lock);
    if ((size_t)dev >= g_multi_groups.size()) g_multi_groups.resize((size_t)dev + 1, nullptr);
    rept_group*& g = g_multi_groups[(size_t)dev];
    if (g && g->max_streams < k) {
        rept_group_destroy(g);
        g = nullptr;
    }
    if (!g) {
        const int rc = rept_group_create(std::max<uint32_t>(k, 64u), 0u, &g);
        if (rc) return rc;
    }
    return rept_group_ingest(g, hs, d_src, d_dst, n, k, stream);
}

int rept_estimates_from_counts(uint32_t m, uint32_t c, uint32_t flags, const uint64_t* h_proc,
                               const uint64_t* d_local, uint32_t n_nodes, double* h_global, double* d_local_est,
                               void* stream) {
    if (m == 0 || c == 0 || !h_proc || !h_global || (d_local && !d_local_est)) return REPT_E_INVAL;
    const bool mascot = (flags & REPT_FLAG_MASCOT) != 0;
    if (!mascot && c > m && c % m != 0) return REPT_E_INVAL;
    rept_config cfg{};
    cfg.m = m;
    cfg.c = c;
    cfg.flags = flags & REPT_FLAG_MASCOT;
    const double f = estimate_factor(cfg);
    // the integer sum of the processors that enter the estimate, then one conversion, as
    // k_global_estimate forms it
    const uint32_t c_used = mascot || c <= m ? c : (c / m) * m;
    unsigned long long sum = 0;
    for (uint32_t i = 0; i < c_used; ++i) sum += h_proc[i];
    *h_global = (double)sum * f;
    if (d_local && n_nodes) {
        int dev = 0, sms = 0;
        REPT_CUDA(cudaGetDevice(&dev));
        REPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        k_local_estimates<<<sms * 4, 256, 0, as_stream(stream)>>>(reinterpret_cast<const unsigned long long*>(d_local),
                                                                   n_nodes, f, d_local_est);
        REPT_LAUNCHED();
    }
    return REPT_OK;
}

const char* rept_strerror(int code) {
    switch (code) {
        case REPT_OK: return "ok";
        case REPT_E_INVAL: return "invalid argument";
        case REPT_E_RANGE: return "edge endpoint >= n_nodes";
        case REPT_E_CAPACITY: return "adjacency pool exhausted (fixed pool)";
        case REPT_E_NOMEM: return "out of memory";
        case REPT_E_CUDA: return "CUDA runtime error";
        case REPT_E_TIMEOUT: return "bounded device wait timed out";
        case REPT_E_INTERNAL: return "internal device invariant failed";
        case REPT_E_SCRATCH: return "problem exceeds the fixed scratch area of rept_count_noalloc";
        case REPT_E_DUPLICATE: return "repeated edge in the stream (REPT_FLAG_CHECK_DUPS)";
        default: return "unknown error";
    }
}

uint64_t rept_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
