// rept_count_noalloc (include/rept.h): the whole counting path for one stream, with every piece of
// intermediate state carved out of one file-scope device array instead of cudaMalloc.  The kernels
// are the library's batch kernels, run once over all edges as a single batch on an empty state.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "rept.h"
#include "rept_common.cuh"
#include "rept_kernels.cuh"

using namespace rept;

namespace {

// The scratch area.  In host code `g_scratch` names a host-side stand-in, not device memory: the
// kernels get the device address looked up below.
static __device__ __align__(256) unsigned char g_scratch[REPT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device

inline unsigned long long align256(unsigned long long x) { return (x + 255ull) & ~255ull; }

// Offsets of the state inside the scratch area for n nodes and E edges.
struct Layout {
    unsigned long long meta, cnt_add, touched, grow_rel, big, rec, srec, hist, ctrl, pool, end;
    unsigned long long pool_quads;
};

Layout layout_for(unsigned long long n, unsigned long long E) {
    Layout L{};
    unsigned long long o = 0;
    L.meta = o;     o = align256(o + n * sizeof(uint4));
    L.cnt_add = o;  o = align256(o + n * sizeof(uint32_t));
    L.touched = o;  o = align256(o + 2 * E * sizeof(uint32_t));
    L.grow_rel = o; o = align256(o + 2 * E * sizeof(uint32_t));
    L.big = o;      o = align256(o + 2 * E * sizeof(uint32_t));
    L.rec = o;      o = align256(o + E * sizeof(WorkItem));
    L.srec = o;     o = align256(o + E * sizeof(WorkItem));
    L.hist = o;     o = align256(o + kSortBuckets * sizeof(uint32_t));
    L.ctrl = o;     o = align256(o + sizeof(Ctrl));
    // From an empty state every node's block (table plus list) is allocated once, with at most 8
    // slots per entry: at most 16 slots (4 quads) per edge.
    L.pool_quads = 4 * E + 1;
    L.pool = o;     o = align256(o + L.pool_quads * 32ull);
    L.end = o;
    return L;
}

// The device address of g_scratch on the current device.  Set-up, once per device with that device
// current: look the symbol up and cache it.  Later calls outside a stream capture look it up again
// (a cheap query), so that after cudaDeviceReset, which reloads the module and may move the array,
// no kernel is launched on a stale address; inside a capture the cached address is used, because
// the lookup may not be legal there.
int scratch_address(cudaStream_t st, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return REPT_E_CUDA;
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (p && cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        (void)cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;  // unknown: keep the cached address
    }
    if (!p || cap == cudaStreamCaptureStatusNone) {
        void* q = nullptr;
        if (cudaGetSymbolAddress(&q, g_scratch) != cudaSuccess || !q) {
            (void)cudaGetLastError();
            return REPT_E_CUDA;
        }
        if (q != p) g_scratch_addr[dev].store(q, std::memory_order_release);
        p = q;
    }
    *out = p;
    return REPT_OK;
}

#define NA_CUDA(call)                          \
    do {                                       \
        if ((call) != cudaSuccess) {           \
            (void)cudaGetLastError();          \
            return REPT_E_CUDA;                \
        }                                      \
    } while (0)

}  // namespace

extern "C" int rept_count_noalloc(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n_edges, uint32_t n_nodes,
                                  uint32_t m, uint32_t c, uint64_t seed, uint64_t* d_proc, uint64_t* d_local,
                                  double* d_global, void* stream) {
    if (m == 0 || c == 0 || n_nodes == 0 || n_nodes == 0xFFFFFFFFu || !d_proc || !d_local) return REPT_E_INVAL;
    if (c > m && c % m != 0) return REPT_E_INVAL;
    if (c > kMaxProcessors) return REPT_E_INVAL;
    if (n_edges > 0 && (!d_src || !d_dst)) return REPT_E_INVAL;
    if (n_edges >= 0xFFFFFFFEull) return REPT_E_SCRATCH;
    const Layout L = layout_for(n_nodes, n_edges);
    if (L.end > REPT_NOALLOC_SCRATCH_BYTES) return REPT_E_SCRATCH;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void* base = nullptr;
    int rc = scratch_address(st, &base);
    if (rc) return rc;
    unsigned char* sc = static_cast<unsigned char*>(base);

    StreamDev d{};
    d.m = m;
    d.c = c;
    d.groups = c <= m ? 1u : c / m;
    d.keep = m;
    d.pstride = m;
    d.pbeg = 0;
    d.pcount = c;
    d.kbeg = 0;
    d.kend = d.groups;
    d.n_nodes = n_nodes;
    d.seed = seed;
    d.fm = make_fastmod(m);
    d.tile_max = 32u;
    d.meta = reinterpret_cast<uint4*>(sc + L.meta);
    d.cnt_add = reinterpret_cast<uint32_t*>(sc + L.cnt_add);
    d.touched = reinterpret_cast<uint32_t*>(sc + L.touched);
    d.grow_rel = reinterpret_cast<uint32_t*>(sc + L.grow_rel);
    d.big = reinterpret_cast<uint32_t*>(sc + L.big);
    d.big_cap = 2 * (n_edges ? n_edges : 1);
    d.rec = reinterpret_cast<WorkItem*>(sc + L.rec);
    d.srec = reinterpret_cast<WorkItem*>(sc + L.srec);
    d.hist = reinterpret_cast<uint32_t*>(sc + L.hist);
    d.ctrl = reinterpret_cast<Ctrl*>(sc + L.ctrl);
    d.pool = reinterpret_cast<uint2*>(sc + L.pool);
    d.pool_quads = L.pool_quads;
    d.local = reinterpret_cast<unsigned long long*>(d_local);
    d.proc = reinterpret_cast<unsigned long long*>(d_proc);

    // the scratch keeps the previous call's contents: clear what must start empty
    NA_CUDA(cudaMemsetAsync(d.meta, 0, (size_t)n_nodes * sizeof(uint4), st));
    NA_CUDA(cudaMemsetAsync(d.cnt_add, 0, (size_t)n_nodes * sizeof(uint32_t), st));
    NA_CUDA(cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), st));
    NA_CUDA(cudaMemsetAsync(d.pool, 0xFF, L.pool_quads * 32ull, st));
    NA_CUDA(cudaMemsetAsync(d_proc, 0, (size_t)c * sizeof(uint64_t), st));
    NA_CUDA(cudaMemsetAsync(d_local, 0, (size_t)n_nodes * sizeof(uint64_t), st));

    if (n_edges > 0) {
        int dev = 0, sms = 0;
        NA_CUDA(cudaGetDevice(&dev));
        NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const BatchDev b{d_src, d_dst, n_edges, 0ull};
        const int threads = 256;
        const unsigned long long blocks = (n_edges + threads - 1) / threads;
        const int grid = (int)(blocks < (unsigned long long)sms * 8 ? blocks : (unsigned long long)sms * 8);
        k_classify<<<grid, threads, 0, st>>>(d, b);
        k_plan<<<grid, threads, 0, st>>>(d);
        k_commit<<<grid, threads, 0, st>>>(d);
        k_rehash_big<<<sms * 4, threads, 0, st>>>(d);
        k_rehash_huge<<<sms * 2, 1024, 0, st>>>(d);
        k_insert<<<grid, threads, 0, st>>>(d, b);
        k_sort_scan<<<1, 1024, 0, st>>>(d);
        k_sort_scatter<<<grid, threads, 0, st>>>(d, b);
        const unsigned long long want_i = (n_edges * 8 + 255) / 256;
        const int grid_i = (int)(want_i < (unsigned long long)sms * 4 ? want_i : (unsigned long long)sms * 4);
        k_intersect_probe<false><<<grid_i, 256, c * sizeof(unsigned long long), st>>>(d, b);
        NA_CUDA(cudaPeekAtLastError());
    }
    if (d_global) {
        const double md = (double)m;
        const double f = c <= m ? md * md / (double)c : md / (double)(c / m);
        k_global_estimate<<<1, 256, 0, st>>>(d.proc, c, f, d_global);
        NA_CUDA(cudaPeekAtLastError());
    }
    unsigned int status = 0;
    NA_CUDA(cudaMemcpyAsync(&status, &d.ctrl->status, sizeof(status), cudaMemcpyDeviceToHost, st));
#ifdef REPT_DEBUG_BOUNDS
    unsigned long long dbg[4] = {0, 0, 0, 0};
    NA_CUDA(cudaMemcpyAsync(dbg, d.ctrl->dbg, sizeof(dbg), cudaMemcpyDeviceToHost, st));
#endif
    NA_CUDA(cudaStreamSynchronize(st));
#ifdef REPT_DEBUG_BOUNDS
    report_failed_check(dbg);
#endif
    // the same mapping as the handle path, except that a full pool is internal here: the pool is
    // sized for the worst case of an empty state
    rc = status_to_code(status);
    return rc == REPT_E_CAPACITY ? REPT_E_INTERNAL : rc;
}
