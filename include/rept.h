/*
 * rept.h -- C ABI of the GB300 REPT streaming semi-triangle counter.
 *
 * REPT (Wang et al., "REPT: A Streaming Algorithm of Approximating Global
 * and Local Triangle Counts in Parallel") splits an edge stream among c
 * processors with a hash h: each processor i keeps the edges of one colour
 * and, for every arriving edge (u, v), counts the common neighbours of u and
 * v among the edges it already keeps (Algorithm 1, UpdateTriangleCNT).  The
 * counts tau^(i), tau_v^(i) are combined into estimates of the global and
 * local triangle counts (Section III-A for c <= m, Section III-B.1 for c > m
 * with c mod m = 0, Section III-B.2 / Algorithm 2 for c > m with c mod m != 0).
 *
 * Conventions shared by every entry point
 *   - Processors are 0-based: processor i = k*m + j (i < c) is slot j of hash
 *     group k and keeps the edges e with h_k(e) = j, where
 *       h_k(u, v) = SplitMix64(((min(u,v) << 32) | max(u,v)) ^ s_k) mod m,
 *       s_k       = seed + k * 0x9E3779B97F4A7C15 (mod 2^64),
 *     SplitMix64(x) being one output step of that generator from state x
 *     (the state is advanced by 0x9E3779B97F4A7C15 before mixing).
 *   - Stream indices are 0-based and global to a handle: the first edge of a
 *     batch follows the last edge of the previous batch.  Batch boundaries
 *     never change any count (the result equals the sequential algorithm).
 *   - Node ids lie in [0, n_nodes).  A self-loop (u == v) is skipped: not
 *     stored, not counted, and tallied in rept_stats.self_loops.  A stream
 *     must not repeat an undirected edge (the paper's E is a set); repeated
 *     edges give undefined counts.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.  All device work of a call is enqueued on
 *     that stream in order.
 *   - Device pointers ("d_" prefix) must point to memory of the device that
 *     was current when the handle was created; host pointers ("h_") to
 *     ordinary or pinned host memory.
 *   - Return value: REPT_OK (0) or a negative REPT_E_* code.  Errors detected
 *     on the device (an id >= n_nodes, an exhausted fixed pool, an internal
 *     probe bound) make the handle's status sticky: the failing batch and
 *     every later batch are not applied (the counts stay those of the last
 *     good batch), and the error is returned by the next call that
 *     synchronises (rept_estimates*, rept_counts, rept_stats, rept_sync, or
 *     any ingest when REPT_FLAG_SYNC is set).  rept_reset clears it.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef REPT_H
#define REPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REPT_OK 0
#define REPT_E_INVAL (-1)     /* bad argument (m, c or n_nodes zero, NULL pointer, unsupported combination) */
#define REPT_E_RANGE (-2)     /* an edge endpoint >= n_nodes (device-detected, batch not applied) */
#define REPT_E_CAPACITY (-3)  /* REPT_FLAG_FIXED_POOL set and the adjacency pool is full (batch not applied) */
#define REPT_E_NOMEM (-4)     /* a device or pinned-host allocation failed */
#define REPT_E_CUDA (-5)      /* a CUDA runtime call failed */
#define REPT_E_TIMEOUT (-6)   /* a bounded grid-wide wait of the persistent group kernel
                                 (REPT_GROUP_PERSISTENT) ran out; the call's batches were not applied */
#define REPT_E_INTERNAL (-7)  /* a device-side invariant failed (bounded probe found no slot) */
#define REPT_E_SCRATCH (-8)   /* rept_count_noalloc: the problem does not fit its fixed scratch area */
#define REPT_E_DUPLICATE (-9) /* REPT_FLAG_CHECK_DUPS: a repeated edge (device-detected, batch not applied) */

#define REPT_FLAG_FIXED_POOL 1u /* never grow the adjacency pool; a full pool gives REPT_E_CAPACITY */
#define REPT_FLAG_SYNC 2u       /* synchronise at the end of every ingest and report errors at once */
#define REPT_FLAG_PROFILE 4u    /* time every kernel launch with CUDA events on its stream (rept_kernel_times) */
#define REPT_FLAG_WORK_COUNTERS 8u /* count the intersection's table reads into rept_stats (slower; not for timing) */
#define REPT_FLAG_LOCAL_PER_PROCESSOR 16u /* also keep every tau_v^(i) (c * n_nodes uint64), read with
                                             rept_local_per_processor */
#define REPT_FLAG_MASCOT 32u /* parallel MASCOT instead of REPT (Section I, Section III-C): c independent
                                samplers of probability 1/m, sampler i keeping the edges that hash
                                group i colours 0; tau^(i) as for REPT, estimates (m^2 / c) * sum,
                                never Algorithm 2 */
#define REPT_FLAG_CHECK_DUPS 64u /* debug: before a batch is applied, look for an edge that repeats a stored
                                    edge or another edge of the same batch (E is a set, Section II; a
                                    repeat is a caller error) and fail the batch with REPT_E_DUPLICATE.
                                    A repeat of an earlier edge that no processor stored is not seen.
                                    Checked by rept_ingest_batch / rept_ingest_host, not by group ingest */

/* kernel ids used by rept_kernel_times */
#define REPT_K_CLASSIFY 0
#define REPT_K_PLAN 1
#define REPT_K_COMMIT 2
#define REPT_K_INSERT 3
#define REPT_K_INTERSECT 4
#define REPT_K_ESTIMATE 5
#define REPT_K_SORT 6
#define REPT_NUM_KERNELS 7

typedef struct rept_config {
    uint32_t m;              /* 1/p; m >= 1 (the paper takes m >= 2; m = 1 keeps every edge) */
    uint32_t c;              /* number of processors, 1 <= c <= 4096 */
    uint64_t seed;           /* hash seed s_0 */
    uint32_t n_nodes;        /* node ids are < n_nodes; 1 <= n_nodes < 2^32 - 1 */
    uint32_t flags;          /* REPT_FLAG_* */
    uint64_t expected_edges; /* sizing hint: edges the stream will carry (0: start small and grow) */
    uint64_t max_batch;      /* sizing hint: largest batch passed to an ingest call (0: 2^20) */
    uint32_t tile_max;       /* tuning: edges whose smaller endpoint holds at most this many entries
                                (4, 8, 16 or 32; 0: 32) share a warp with other edges, larger ones get a
                                warp of their own; results do not depend on it */
    uint32_t proc_begin;     /* colour sharding: the handle keeps processors [proc_begin, proc_end) only
                                (stores the edges they keep, counts their semi-triangles); 0, 0: all c.
                                Processors are independent until the final sums (Algorithm 1), so
                                handles whose ranges split 0..c-1 (say one per GPU, each ingesting the
                                whole stream) give, summed, exactly the counts of one handle with all
                                processors: tau^(i) from the handle that keeps i, sum_i tau_v^(i) as the
                                sum over handles.  Not for c > m with c mod m != 0 (Algorithm 2's
                                combination is not a sum): REPT_E_INVAL */
    uint32_t proc_end;       /* see proc_begin; proc_begin < proc_end <= c, or both 0 */
    uint32_t reserved;       /* must be 0 */
    uint32_t reserved2;      /* must be 0 */
} rept_config;

typedef struct rept_stats {
    uint64_t edges;          /* edges ingested (including self-loops) */
    uint64_t self_loops;     /* self-loops skipped */
    uint64_t stored_edges;   /* edges kept by at least one processor (union adjacency) */
    uint64_t pool_slots;     /* adjacency pool capacity in 8-byte slots */
    uint64_t pool_used;      /* slots handed out to per-node tables so far */
    uint64_t device_bytes;   /* device memory held by the handle */
    /* with REPT_FLAG_WORK_COUNTERS, totals over the stream's intersection passes: */
    uint64_t small_entries;  /* entries present in the smaller endpoint's table, summed over edges */
    uint64_t small_slots;    /* slots of those tables read (entries plus empty slots) */
    uint64_t probes;         /* probes of the larger endpoint's table (small-side entries older than the edge
                                and, where colours are kept, coloured alike for a kept processor) */
    uint64_t probe_slots;    /* slots read by those probes */
    uint64_t wedges;         /* closed wedges found in the union adjacency (both edges older than the edge) */
    uint64_t counted;        /* (wedge, hash group) pairs counted for some processor */
    uint64_t class_items[6]; /* edges per intersection work class (smaller endpoint with <= 4, 8, 16,
                                32, 256, more entries) */
    uint64_t class_probes[6];  /* probes issued per work class */
    uint64_t class_cycles[6];  /* warp-cycles spent per work class (clock64, summed over warps) */
} rept_stats;

typedef struct rept_state rept_state;

/*
 * rept_create: allocate an empty stream state (all tau^(i), tau_v^(i) = 0,
 * every E^(i) empty; Algorithm 1's initialisation) on the current device.
 * `cfg` is copied; `*out` receives the handle (owned by the caller, released
 * with rept_destroy).  Returns REPT_E_INVAL for m == 0, c == 0, c > 4096 or
 * n_nodes == 0; REPT_E_NOMEM / REPT_E_CUDA on allocation failure.  For c > m
 * with c mod m != 0 the handle also keeps Algorithm 2's triangle-pair
 * counters (16 + 12 * ceil(c/m) bytes per stream edge).
 * Speed: with one hash group (c <= m, or MASCOT with c == 1) and m >= 2, each
 * stored entry keeps its colour (in the entry's top 8 bits when m <= 256 and
 * n_nodes <= 2^24, else in a word beside it, 25 % more pool), and the
 * intersection tests colours before it looks an edge up, so only about 1/m
 * of the lookups happen; configurations with several hash groups look up
 * every candidate wedge edge (same counts, slower intersection).
 */
int rept_create(const rept_config* cfg, void* stream, rept_state** out);

/*
 * rept_reset: return the handle to the empty stream, keeping its allocations;
 * clears a sticky error.  The clearing is enqueued on `stream` (the call does
 * not wait); the adjacency pool is reused as it is, each table getting its
 * empty keys when its block is handed out again.
 */
int rept_reset(rept_state* s, void* stream);

/*
 * rept_reset_async: as rept_reset, and the next stream uses hash seed `seed`
 * (s_0).  For servers that reuse a handle for the next stream of the same
 * shape.
 */
int rept_reset_async(rept_state* s, uint64_t seed, void* stream);

/*
 * rept_ingest_batch: append n edges (d_src[t], d_dst[t]), t < n, to the
 * stream and process them exactly as Algorithm 1 would, one edge after the
 * other: every edge first closes the wedges of edges that arrived before it
 * and are kept by a common processor (counted for every processor whose
 * colour both wedge edges carry), then is stored by the processors that keep
 * it.  d_src / d_dst are device arrays of n uint32 node ids, caller-owned,
 * and must stay valid and unchanged until the stream reaches this work.
 * Asynchronous on `stream`, except that the call may synchronise once to
 * grow the adjacency pool (never with REPT_FLAG_FIXED_POOL).  n == 0 is a
 * no-op.  Errors: REPT_E_INVAL (NULL pointers with n > 0), REPT_E_NOMEM,
 * REPT_E_CUDA; device-detected errors as described above.
 */
int rept_ingest_batch(rept_state* s, const uint32_t* d_src, const uint32_t* d_dst, uint64_t n, void* stream);

/*
 * rept_ingest_host: the same for host arrays h_src / h_dst of n edges.  The
 * edges are copied to device staging buffers owned by the handle in chunks
 * of at most `batch` edges (0: the handle's max_batch) and each chunk is
 * ingested as one batch.  Returns after the last chunk has been enqueued and
 * its host buffers may be reused (the call synchronises on the copies).
 */
int rept_ingest_host(rept_state* s, const uint32_t* h_src, const uint32_t* h_dst, uint64_t n, uint64_t batch,
                     void* stream);

/*
 * rept_estimates: FP64 estimates from the counts so far.
 *   c <= m              : tau_hat = (m^2 / c) * sum_i tau^(i),  tau_hat_v likewise   (Section III-A)
 *   c > m, c % m == 0   : tau_hat = (m / c1) * sum_i tau^(i), c1 = c / m              (Section III-B.1)
 *   c > m, c % m != 0   : the full groups' estimate t1 = (m / c1) * sum_{i < c1 m} tau^(i) and the
 *                         partial group's t2 = (m^2 / c2) * sum_{i >= c1 m} tau^(i), combined as
 *                         (w2 t1 + w1 t2) / (w1 + w2) with w1 = t1 (m-1) / c1 and
 *                         w2 = (t1 (m^2 - c2) + 2 eta_hat (m - c2)) / c2, eta_hat = (m^3/c) sum_i eta^(i)
 *                         (Algorithm 2; t1 when both weights are 0); locally the same per node
 * Each scale factor is formed in double and multiplied by the exactly
 * converted integer sum.  h_global: host double (required).  d_local: device
 * array of n_nodes doubles, or NULL to skip the local estimates.
 * Synchronises `stream`; returns any sticky device error.
 */
int rept_estimates(rept_state* s, double* h_global, double* d_local, void* stream);

/* rept_estimates_host: as rept_estimates, with the local estimates written to host memory h_local (or NULL). */
int rept_estimates_host(rept_state* s, double* h_global, double* h_local, void* stream);

/*
 * rept_estimates_async: enqueue, without waiting, the computation of tau_hat
 * (as in rept_estimates) and copies to host memory of tau_hat (h_global, one
 * double), the c counters tau^(i) (h_proc, or NULL) and the handle's status
 * word (h_status: 0 when no device error was recorded, else nonzero; the
 * next synchronising call returns the matching REPT_E_* code).  The host
 * buffers should be pinned for the copies to be asynchronous; their contents
 * are valid once `stream` has reached this point (record an event after the
 * call and wait on it).
 */
int rept_estimates_async(rept_state* s, double* h_global, uint64_t* h_proc, uint32_t* h_status, void* stream);

/*
 * rept_counts: the integer counters.  h_proc: host array of c uint64
 * (tau^(i), processor i = k*m + j), or NULL.  d_local: device array of
 * n_nodes uint64 receiving sum_i tau_v^(i) over all processors, or NULL.
 * Synchronises `stream`; returns any sticky device error.
 */
int rept_counts(rept_state* s, uint64_t* h_proc, uint64_t* d_local, void* stream);

/*
 * rept_pair_counts: for c > m with c mod m != 0, Algorithm 2's counters:
 * h_eta_proc (host, c uint64: eta^(i)), d_eta_local (device, n_nodes uint64:
 * sum_i eta_v^(i)), d_local1 / d_local2 (device, n_nodes uint64: sum of
 * tau_v^(i) over the full groups / over the partial group); any may be NULL.
 * The pair counter of a newly stored edge starts at 0 (Table I's eta counts
 * only pairs whose shared edge is last in neither triangle).  REPT_E_INVAL
 * for other c.  Synchronises `stream`; returns any sticky device error.
 */
int rept_pair_counts(rept_state* s, uint64_t* h_eta_proc, uint64_t* d_eta_local, uint64_t* d_local1,
                     uint64_t* d_local2, void* stream);

/*
 * rept_local_per_processor: with REPT_FLAG_LOCAL_PER_PROCESSOR, every
 * processor's local counts tau_v^(i) (Algorithm 1's per-processor counters)
 * into the device array d_out of c * n_nodes uint64, processor-major
 * (d_out[i * n_nodes + v]).  REPT_E_INVAL without the flag.  Synchronises
 * `stream`; returns any sticky device error.
 */
int rept_local_per_processor(rept_state* s, uint64_t* d_out, void* stream);

/* rept_stats: counters describing the handle (see rept_stats).  Synchronises `stream`. */
int rept_get_stats(rept_state* s, rept_stats* out, void* stream);

/*
 * rept_kernel_times: with REPT_FLAG_PROFILE, the summed CUDA-event durations
 * (milliseconds) and launch counts of each kernel (REPT_K_* order) since
 * create or the previous call with `clear` != 0 (rept_reset keeps them).  ms and launches are
 * host arrays of REPT_NUM_KERNELS entries (either may be NULL).  Synchronises
 * the handle's recorded events.  REPT_E_INVAL without REPT_FLAG_PROFILE.
 */
int rept_kernel_times(rept_state* s, double* ms, uint64_t* launches, int clear);

/*
 * Snapshot and resume.  rept_snapshot_size reports the bytes of the handle's
 * current state (configuration, stream position, node tables, counters and,
 * when kept, the pair counters and per-processor local counts); rept_snapshot
 * copies it into caller-owned host memory h_buf of that many bytes.
 * rept_restore loads such a snapshot into a handle created with the same
 * m, c, seed, n_nodes and flags (REPT_E_INVAL otherwise), replacing its
 * state; ingesting the rest of the stream then gives exactly the counts of
 * an uninterrupted run.  All three synchronise `stream`.
 */
int rept_snapshot_size(rept_state* s, uint64_t* bytes, void* stream);
int rept_snapshot(rept_state* s, void* h_buf, uint64_t bytes, void* stream);
int rept_restore(rept_state* s, const void* h_buf, uint64_t bytes, void* stream);

/* rept_sync: wait for `stream` and return the handle's sticky device error, if any. */
int rept_sync(rept_state* s, void* stream);

/* rept_destroy: free every allocation of the handle (NULL is a no-op).  Waits for the handle's pending work. */
void rept_destroy(rept_state* s);

/*
 * Batched ingestion of many independent streams.  A rept_group ingests one
 * batch into each of up to max_streams handles with one kernel launch per
 * step of the batch path for all of them (the launch grid's y dimension
 * ranges over the streams), instead of one launch sequence per stream.  The
 * paper runs its processors on one stream; a group runs many streams' REPT
 * side by side.  Counts are exactly those of calling rept_ingest_batch on
 * each handle in turn.
 *
 * rept_group_create: max_streams >= 1; flags REPT_GROUP_GRAPH captures the
 * launch sequence in a CUDA graph and replays it on later calls with the same
 * shape (used only when no stream's pool can run out during the call);
 * REPT_GROUP_PERSISTENT makes that sequence one cooperative launch (see the
 * flag).  REPT_E_CUDA when the device cannot launch cooperative kernels.
 */
#define REPT_GROUP_GRAPH 1u
#define REPT_GROUP_PERSISTENT 2u  /* one cooperative launch per call runs every step of the batch path
                                     for every stream, the streams' work dealt out over one co-resident
                                     grid, with grid-wide waits between the steps; each wait is bounded
                                     in time, and when it runs out the call's streams report
                                     REPT_E_TIMEOUT (nothing is applied).  Used when no stream's pool can
                                     run out during the call (otherwise the launch-per-step path runs);
                                     with REPT_GROUP_GRAPH the launch is replayed from a CUDA graph */
#define REPT_GROUP_TEST_TIMEOUT 4u /* test hook for the timeout path, with REPT_GROUP_PERSISTENT only: the
                                      first grid-wide wait expects one block more than the grid holds,
                                      so it runs out after 0.1 s; REPT_E_INVAL without the other flag */
typedef struct rept_group rept_group;
int rept_group_create(uint32_t max_streams, uint32_t flags, rept_group** out);

/*
 * rept_group_ingest: append d_src[i][0..n[i]), d_dst[i][0..n[i]) to stream
 * hs[i] for i < k (k <= max_streams; n[i] may be 0; the handles must be
 * distinct and belong to the current device; device arrays as in
 * rept_ingest_batch).  Enqueued on `stream`; the call synchronises once when
 * some stream's pool might have to grow (never when every handle was created
 * with expected_edges covering its stream, or with REPT_FLAG_FIXED_POOL).
 * Handle flags REPT_FLAG_PROFILE and REPT_FLAG_WORK_COUNTERS are ignored here.
 * Errors: REPT_E_INVAL (bad arguments), REPT_E_NOMEM, REPT_E_CUDA; device
 * errors stay sticky on the handle they concern.
 */
int rept_group_ingest(rept_group* g, rept_state* const* hs, const uint32_t* const* d_src,
                      const uint32_t* const* d_dst, const uint64_t* n, uint32_t k, void* stream);

/* rept_group_destroy: release the group (not the handles).  NULL is a no-op. */
void rept_group_destroy(rept_group* g);

/*
 * rept_ingest_multi: rept_group_ingest through a group that the library
 * keeps for the current device, for callers that do not want to manage one:
 * the same arguments, counts and errors.  The group is made on the first call
 * (sized for max(k, 64) streams), made again, larger, when a call brings more
 * streams (that call synchronises the device), and kept until the process
 * exits.  Calls from several host threads are serialised.
 */
int rept_ingest_multi(rept_state* const* hs, const uint32_t* const* d_src, const uint32_t* const* d_dst,
                      const uint64_t* n, uint32_t k, void* stream);

/*
 * rept_count_noalloc: count a whole edge stream in one call without
 * allocating any memory.  The paper has no counterpart; this is a library
 * convenience for callers that cannot call cudaMalloc -- for example code
 * whose device memory is entirely owned by another allocator (a framework's
 * caching allocator that has reserved the free memory), or a latency-critical
 * loop that cannot afford the device-wide synchronisation that cudaFree
 * implies.  It computes the same counts as rept_create + one
 * rept_ingest_batch of all n_edges edges + rept_counts, and the same global
 * estimate as rept_estimates.
 *
 * Scratch: all intermediate state (per-node tables, batch work lists, the
 * control block) lives in one statically allocated device array of
 * REPT_NOALLOC_SCRATCH_BYTES (64 MiB) inside this library; every GPU that
 * loads the library holds that array until the process exits.  A problem
 * needs 20 * n_nodes + 216 * n_edges + 200 KiB bytes of it (for example
 * 2^20 nodes and 210,000 edges); larger problems return REPT_E_SCRATCH
 * before any device work is enqueued.  c must be at most 4096.
 *
 * Arguments: d_src / d_dst: device arrays of n_edges uint32 endpoints
 * (self-loops skipped as in rept_ingest_batch).  Outputs, caller-allocated on
 * the same device and overwritten: d_proc[c] (tau^(i), uint64), d_local[n_nodes]
 * (sum_i tau_v^(i), uint64), d_global (tau_hat, one double; may be NULL).
 * m, c, seed, n_nodes have the meaning of rept_config; c > m needs c % m == 0.
 *
 * Behaviour: the first call on a device looks up the scratch array's device
 * address on that device (cudaGetSymbolAddress) and caches it; make that first
 * call before any stream capture.  Later calls on a stream that is not being
 * captured look the address up again, so a cudaDeviceReset between calls
 * (which reloads the library's device code) is safe; a call inside a capture
 * uses the cached address, so no device reset may happen between the last
 * uncaptured call and a capture.  Every call enqueues its work on `stream`,
 * then waits for the stream and returns REPT_E_RANGE if an endpoint was
 * >= n_nodes (outputs then undefined).  All calls share the one scratch array
 * and the call clears the parts that must start at zero, so sequential calls
 * are independent; calls whose work overlaps on the GPU (other host threads,
 * other streams) race on the scratch and give undefined results.
 */
#define REPT_NOALLOC_SCRATCH_BYTES (64ull << 20)
int rept_count_noalloc(const uint32_t* d_src, const uint32_t* d_dst, uint64_t n_edges, uint32_t n_nodes, uint32_t m,
                       uint32_t c, uint64_t seed, uint64_t* d_proc, uint64_t* d_local, double* d_global,
                       void* stream);

/*
 * rept_estimates_from_counts: the FP64 estimates of Section III-A (c <= m) and Section III-B.1
 * (c > m, c mod m = 0), or parallel MASCOT's average (flags = REPT_FLAG_MASCOT), from integer
 * counts that the caller holds, typically the sums over colour shards (rept_config.proc_begin).
 * h_proc: host array of c uint64 tau^(i).  d_local: device array of n_nodes uint64 sum_i tau_v^(i),
 * or NULL.  Outputs: h_global (host, one double), d_local_est (device, n_nodes doubles; ignored when
 * d_local is NULL).  The factors and rounding are those of rept_estimates, so summed shard counts
 * give exactly the estimates of an unsharded handle.  Allocates nothing; d_local_est is written on
 * `stream` and the call returns after enqueueing it (h_global is written before it returns).
 * REPT_E_INVAL for c > m with c mod m != 0 (not linear in the counts), m or c zero, NULL h_proc /
 * h_global, or a NULL d_local_est with a non-NULL d_local.
 */
int rept_estimates_from_counts(uint32_t m, uint32_t c, uint32_t flags, const uint64_t* h_proc,
                               const uint64_t* d_local, uint32_t n_nodes, double* h_global, double* d_local_est,
                               void* stream);

/* rept_strerror: static English text for a REPT_* code. */
const char* rept_strerror(int code);

/* rept_kernel_launches: kernels this library has launched in this process (all handles). */
uint64_t rept_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* REPT_H */
