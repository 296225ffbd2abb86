/*
 * tc.h -- C ABI of the GB300-native exact triangle counter.
 *
 * Method (Wang, Wang, Yang, Owens, "A Comparative Study on Exact Triangle
 * Counting Algorithms on the GPU", HPGP'16), Sec. 3.2 "TC using Set
 * Intersection", Alg. 2, and Sec. 4.2 (its implementation):
 *   1. Form the filtered edge list: keep every undirected edge once, oriented
 *      from the lower to the higher rank, rank(v) = (d(v), v)  (Sec. 4.2.1);
 *   2. compact the kept edges into an oriented CSR, the induced subgraph of
 *      Sec. 4.2.1: N+(u) = { v : {u,v} in E, rank(u) < rank(v) }, ascending;
 *   3. partition the oriented edges by list size (Alg. 2 Partition, Sec. 4.2.2
 *      dynamic grouping) and intersect N+(u) with N+(v) for every oriented
 *      edge (u, v); each common w closes triangle {u, v, w} (Sec. 3.2);
 *   4. reduce the intersection sizes to the total (Alg. 2 Reduce) and, on
 *      request, to per-vertex counts t(v) = number of triangles containing v.
 * Results are exact int64 integers; there is exactly one correct answer.
 *
 * Conventions for every entry point:
 *   - Every call returns tc_status; nothing throws across the ABI.  On an
 *     error, tc_last_error(ctx) holds a one-line reason.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued asynchronously on it unless a call says it
 *     synchronises; device results are valid once the stream reaches them.
 *   - Input buffers are borrowed for the duration of the call (for device
 *     inputs: until the enqueued work has read them).  Output buffers are
 *     owned by the caller.  tc_ocsr and tc_server handles are owned by the
 *     library and freed by the caller with tc_ocsr_free / tc_server_destroy.
 *   - Vertex ids are int32 (n < 2^31); offsets are int64.
 *   - Library-owned device memory comes from the device's stream-ordered
 *     memory pool (cudaMallocAsync on the call's stream).
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tc_status {
    TC_OK = 0,
    TC_PENDING = 1,              /* tc_poll: request not finished yet */
    TC_ERR_INVALID_ARG = -1,     /* NULL handle, negative size, bad flag combination */
    TC_ERR_INVALID_GRAPH = -2,   /* TC_VALIDATE found a non-simple / asymmetric / unsorted CSR, or an id outside [0,n) */
    TC_ERR_OOM = -3,             /* device allocation failed */
    TC_ERR_BUDGET = -4,          /* serving: request larger than the whole HBM budget */
    TC_ERR_TIMEOUT = -5,         /* a bounded wait gave up */
    TC_ERR_CUDA = -6,            /* any other CUDA runtime error (message in tc_last_error) */
    TC_ERR_NOT_FOUND = -7,       /* serving: unknown ticket */
    TC_ERR_DEVICE = -8           /* a device-side check failed (see tc_check); the results are not valid */
} tc_status;

/* tc_graph.flags / tc_batch.flags */
#define TC_IN_DEVICE     0x0u  /* input pointers are device memory (default) */
#define TC_IN_HOST       0x1u  /* input pointers are host memory; the call copies them to the device */
#define TC_VALIDATE      0x2u  /* check a CSR input (sorted, no loops, no duplicates, symmetric, ids in range);
                                  synchronises the stream once to read the verdict */

/* An undirected simple graph, as the paper states the problem (Sec. 3):
 *   CSR form   (row_ptr != NULL): row_ptr[n+1] (int64, row_ptr[0] = 0,
 *              row_ptr[n] = nnz), col[nnz] (int32), both directions of every
 *              edge present, each row strictly ascending, no self-loops.
 *              nnz = 2m.
 *   Edge list  (row_ptr == NULL): src[nnz], dst[nnz] pairs.  Self-loops,
 *              duplicates and either or both directions are allowed; they
 *              are dropped and symmetrised (the paper's dataset treatment,
 *              Table 1 caption).  Ids outside [0, n) give TC_ERR_INVALID_GRAPH. */
typedef struct tc_graph {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* src;
    const int32_t* dst;
    uint32_t flags;
} tc_graph;

/* Tuning knobs (Alg. 2 Partition thresholds; the paper leaves them open,
 * Sec. 4.2.2).  Zero means "use the built-in default".  No knob changes a
 * result, only the speed. */
typedef struct tc_config {
    int32_t small_max;     /* oriented edges with max(d+(u), d+(v)) <= small_max are merged by one
                              thread each (the paper's TwoSmall); default 8 */
    int32_t warp_max;      /* pivots with d+ <= warp_max probe a warp-private table; larger pivots a
                              CTA-wide table (the paper's TwoLarge role); default 128 */
    int32_t table_cap;     /* keys per CTA table segment (power of two, 16..4096); longer lists are
                              split into segments; default 1024 */
    int32_t probe;         /* 0/1 = open-addressing hash probe, 2 = binary search of the sorted list */
    int32_t cta_threads;   /* threads per CTA of the CTA-table kernel (64..1024); default 256 */
    int32_t chunk;         /* partners per work item of the warp-table class (CTA-table items take
                              twice as many, at most 32767 and at most (2^31 - 1) / (sqrt(2m) + 4));
                              default 512 */
    int32_t bitmap_bits;   /* CTA items whose pivot list spans at most this many rank ids (vertices
                              renamed in (degree, id) order) probe a shared-memory bitmap instead of
                              the hash table; multiple of 32, <= 262144; default 131072; -1 = never */
    int32_t direct_span;   /* ... and those spanning at most this many rank ids one counter cell per
                              rank id (presence and hits in one probe; 32-bit cells up to half this
                              span, 16-bit above); <= 16384; default 16384;
                              -1 = never (needs bitmap_bits > 0) */
    int32_t merge_ratio;   /* degree-ratio switch between the two intersection strategies of Sec. 4.2.2:
                              an oriented edge that is not thread-merged, whose longer list has at most
                              merge_max elements and whose ratio r = max(d+)/min(d+) is at most
                              merge_ratio/100, is intersected by a warp-cooperative merge path over
                              both sorted lists (balanced lists); every other edge probes its pivot's
                              table (skewed lists).  Percent, >= 100; default 0 = no merge class */
    int32_t merge_max;     /* see merge_ratio; 16..4096, default 256 */
    int32_t stage;         /* CTA-table kernel: 1 = the partner lists walked by 4 or more lanes are
                              staged into shared memory by the copy engine (cp.async.bulk), one batch
                              ahead of the probing; 0 (default) or -1 = every lane loads its own
                              vectors (faster on GB300: the small copies wait longer than the loads) */
    int32_t small_lanes;   /* threads per source row of the thread-merge class (threads per edge of
                              Sec. 4.2.2's TwoSmall): lane j of a row's group takes its edges j, j+L, ...;
                              1, 2, 4, 8, 16 or 32; default 1 */
    int32_t reserved[4];
} tc_config;

typedef struct tc_ctx tc_ctx;
typedef struct tc_ocsr tc_ocsr;

/* Tracing: CUDA events around each phase, recorded on the stream the phase
 * runs on, plus a count of the library's kernel launches.  Off by default;
 * never active inside a CUDA-graph capture. */
#define TC_TRACE_PHASES 20
enum {
    TC_PH_DEGREE = 0, TC_PH_VALIDATE, TC_PH_ORIENT_COUNT, TC_PH_ORIENT_SCAN, TC_PH_ORIENT_SCATTER,
    TC_PH_PIVOT_COUNT, TC_PH_PIVOT_SCAN, TC_PH_PIVOT_SCATTER, TC_PH_ITEMS, TC_PH_COUNT_SMALL,
    TC_PH_COUNT_WARP, TC_PH_COUNT_CTA, TC_PH_EDGE_SORT, TC_PH_COUNT_INIT, TC_PH_RANK, TC_PH_ROW_SORT,
    TC_PH_COUNT_MERGE, TC_PH_FUSED
};
typedef struct tc_trace {
    int64_t launches;                        /* kernel launches since the last read */
    double phase_ms[TC_TRACE_PHASES];        /* summed device time per phase */
    int32_t phase_calls[TC_TRACE_PHASES];    /* event pairs summed per phase */
} tc_trace;

/* Create a context on CUDA device `device` (made current for the call).
 * cfg may be NULL (all defaults).  Cheap; holds no graph memory. */
tc_status tc_ctx_create(int device, const tc_config* cfg, tc_ctx** out);
void tc_ctx_destroy(tc_ctx* ctx);
/* Device-side checks.  The count kernels never spin without a bound and never
 * access memory their invariants do not allow: when such a state is met the
 * kernel skips the step and raises a bit of a per-device check word, which is
 * sticky until tc_check reads it.  TC_DEVERR_PROBE: an open-addressing lookup
 * or insert visited every slot of its table (tables are at most a quarter
 * full, so this means a table left dirty).  TC_DEVERR_WAIT: a wait for a
 * staged copy of partner lists gave up (about a second); the warp went on
 * without staging.  The TC_DEBUG build of the library
 * (compiled with -DTC_DEBUG=1) adds bounds checks: TC_DEVERR_BOUNDS, an index
 * of a list, table or cell array out of range; TC_DEVERR_DIRTY, a table region
 * not all zeros at the start of a work item. */
#define TC_DEVERR_PROBE  0x1u
#define TC_DEVERR_BOUNDS 0x2u
#define TC_DEVERR_DIRTY  0x4u
#define TC_DEVERR_WAIT   0x8u  /* a wait for a staged copy of the count kernel gave up (about 1 s) */
/* Synchronise `stream`, read and clear the check word of the current device;
 * *bits (nullable) receives it.  TC_ERR_DEVICE if any bit was set, else TC_OK.
 * tc_count and tc_count_batch with host outputs check it themselves (they
 * synchronise anyway); with device outputs call tc_check after the counts. */
tc_status tc_check(tc_ctx* ctx, uint32_t* bits, void* stream);

/* One-line description of the last error on this context ("" if none). */
const char* tc_last_error(const tc_ctx* ctx);
/* Replace the tuning knobs (same meaning as in tc_ctx_create). */
tc_status tc_ctx_set_config(tc_ctx* ctx, const tc_config* cfg);
tc_status tc_ctx_get_config(const tc_ctx* ctx, tc_config* out);
/* Turn phase tracing on (1) or off (0). */
tc_status tc_ctx_set_trace(tc_ctx* ctx, int enable);
/* Wait for the recorded events, sum them into *out and reset the trace. */
tc_status tc_ctx_read_trace(tc_ctx* ctx, tc_trace* out);

/* Steps 1-3 of the method (Sec. 4.2.1 edge-list filtering and induced
 * subgraph; Alg. 2 Partition): from an undirected graph, build on the device
 * the oriented CSR N+ and the work partition that tc_count consumes.
 * Asynchronous on `stream` (no host synchronisation) for a CSR input without
 * TC_VALIDATE; an edge-list input synchronises once (to learn the number of
 * distinct edges), and so does TC_VALIDATE (to read the verdict).  *out receives a
 * library-owned handle; free it with tc_ocsr_free after the last tc_count on
 * it has completed. */
tc_status tc_build_oriented_csr(tc_ctx* ctx, const tc_graph* g, tc_ocsr** out, void* stream);

/* Steps 3-4 (Sec. 3.2 intersection, Alg. 2 Compute_Intersection and
 * Reduce): total = number of triangles; per_vertex[v] = t(v) when
 * per_vertex != NULL (n entries).  Both may be device or host pointers:
 * device outputs are written asynchronously; if either is host memory the
 * call copies the results back and synchronises `stream` before returning.
 * Any number of tc_count calls may run on one tc_ocsr, on any streams. */
tc_status tc_count(tc_ctx* ctx, const tc_ocsr* o, int64_t* total, int64_t* per_vertex, void* stream);

/* All four steps in one call, without a handle: degree and (degree, id)
 * rank, orientation filter and compaction (Sec. 4.2.1, Alg. 2
 * Form_Filtered_Edge_List), intersection of N+(u) and N+(v) for every oriented
 * edge (Sec. 3.2, Alg. 2 Compute_Intersection) and the reduction (Alg. 2
 * Reduce).  A CSR graph with at most 8192 vertices whose arrays fit one CTA's
 * shared memory (4 * (3n + m + 2W + 35) bytes <= 224 KiB, m = nnz/2,
 * W = ceil(nnz/32)), without TC_VALIDATE, is counted by one kernel
 * launch of ceil(m/1024) CTAs of 1024 threads (at most one per SM), each CTA
 * orienting the whole graph in its own shared memory and counting its share
 * of the oriented edges, instead of the thirty-odd launches of the general
 * path, with the same exact results.  Any other graph takes tc_build_oriented_csr +
 * tc_count and releases the handle in stream order.  Inputs as in
 * tc_build_oriented_csr (TC_IN_HOST copies them first); outputs as in tc_count
 * (total required, per_vertex nullable; device outputs are written
 * asynchronously, host outputs are copied back and `stream` is synchronised).
 * The input must be a simple symmetric CSR (as for tc_build_oriented_csr
 * without TC_VALIDATE): other input gives meaningless counts, but every index
 * the fused kernel forms stays inside its arrays. */
tc_status tc_count_graph(tc_ctx* ctx, const tc_graph* g, int64_t* total, int64_t* per_vertex, void* stream);

/* Triangle-derived metrics, the use of the counts the paper names (Sec. 5,
 * clustering coefficient and transitivity).  With d(v) the undirected degree:
 *   wedges(v) = d(v)(d(v)-1)/2;  local[v] = t(v)/wedges(v), 0 when d(v) < 2;
 *   *wedges = sum_v wedges(v);   *transitivity = 3T / *wedges, 0 without wedges.
 * total and per_vertex are tc_count's device outputs for this handle;
 * local (n doubles), transitivity and wedges may each be NULL, host or device
 * memory.  Each ratio is one correctly rounded fp64 division of exact
 * integers.  Synchronises `stream`.  Not available for batch handles. */
tc_status tc_clustering(tc_ctx* ctx, const tc_ocsr* o, const int64_t* total, const int64_t* per_vertex, double* local,
                        double* transitivity, int64_t* wedges, void* stream);

/* Per-edge support and triangle listing (Sec. 1: enumerating the triangles
 * is the subroutine of k-truss; every method the paper compares lists them).
 * For every oriented edge (u, v) the sorted lists N+(u), N+(v) are merged;
 * each common w gives the triangle (u, v, w), rank(u) < rank(v) < rank(w).
 *   support    NULL or m int64: support[e] = triangles containing the edge
 *              {u, col[e]} of the oriented CSR (the order of tc_ocsr_copy).
 *   triangles  NULL or 3*capacity int32: the first `capacity` triangles found,
 *              (u, v, w) vertex ids, in no particular order.
 *   *count     the number of triangles (all of them, also beyond capacity).
 * Outputs may be host or device memory; synchronises `stream`. */
tc_status tc_edge_support(tc_ctx* ctx, const tc_ocsr* o, int64_t* support, int32_t* triangles, int64_t capacity,
                          int64_t* count, void* stream);

/* Alg. 3 (Sec. 3.3) as the masked sparse product the paper proposes as future
 * work (Sec. 5: upper triangle only, only where A is nonzero, B = LU never
 * written).  With vertices in decreasing rank order, the upper-triangle entry
 * of C = A o (LU) at the oriented edge e = (u, v) is |N+(u) & N+(v)|; c[e]
 * receives it for every oriented edge (m int64, the order of tc_ocsr_copy)
 * and *total (nullable) their sum, T.  Host or device outputs; synchronises. */
tc_status tc_masked_product(tc_ctx* ctx, const tc_ocsr* o, int64_t* c, int64_t* total, void* stream);

/* Subgraph matching of a labelled triangle (Alg. 1, Sec. 3.1): the number of
 * triangles whose three vertex labels are the multiset {query[0..2]}.
 * g is a device CSR (as in tc_graph, TC_IN_HOST not accepted), labels[n] device
 * int32, query[3] host int32, total host or device.  Candidate edges (label
 * pair of a query edge) are filtered on the device, then joined by the
 * set-intersection count; for a query {a, a, b} the {a, a, a} triangles of
 * the a-a subgraph are subtracted.  Synchronises `stream`. */
tc_status tc_count_labelled(tc_ctx* ctx, const tc_graph* g, const int32_t* labels, const int32_t* query,
                            int64_t* total, void* stream);

/* One shard of tc_count, the building block of counting one graph on several
 * GPUs (the paper counts on one GPU; each oriented edge is an independent unit
 * of Sec. 3.2, so the work shards without changing the result).  Every GPU
 * builds the same oriented CSR, shard s of nshards runs that equal part of
 * the partition's work lists and source rows, and the caller sums `total`
 * and `per_vertex` over the shards (an all-reduce): the sums equal tc_count's
 * result exactly.  Outputs and synchronisation as in tc_count;
 * TC_ERR_INVALID_ARG unless 0 <= shard < nshards. */
tc_status tc_count_shard(tc_ctx* ctx, const tc_ocsr* o, int32_t shard, int32_t nshards, int64_t* total,
                         int64_t* per_vertex, void* stream);

/* Read-only view of a built oriented CSR (device pointers, owned by the handle). */
typedef struct tc_ocsr_view {
    int64_t n;                 /* vertices */
    int64_t m;                 /* |E+| = undirected edges */
    const int64_t* row_ptr;    /* device [n+1]: N+(u) = col[row_ptr[u] .. row_ptr[u+1]) */
    const int32_t* col;        /* device [m], ascending within a row */
    int64_t bytes;             /* device bytes held by the handle */
} tc_ocsr_view;
tc_status tc_ocsr_get_view(const tc_ocsr* o, tc_ocsr_view* out);
/* Copy the oriented CSR (Sec. 4.2.1 induced subgraph) into caller buffers
 * row_ptr[n+1] and col[m], host or device memory; synchronises `stream`. */
tc_status tc_ocsr_copy(const tc_ocsr* o, int64_t* row_ptr, int32_t* col, void* stream);
/* Free the handle's device memory; synchronises the device first. */
void tc_ocsr_free(tc_ocsr* o);
/* Free in stream order (no host synchronisation): every use of the handle
 * must already be enqueued on `stream` or ordered before it. */
void tc_ocsr_release(tc_ocsr* o, void* stream);

/* ---- oriented CSR without device allocation --------------------------------
 * The paper has no counterpart; this serves callers that cannot allocate
 * device memory while running: serving loops with a latency budget (cudaMalloc
 * and cudaFree may synchronise the device) and processes whose HBM is already
 * reserved in full by another allocator.
 *
 * tc_orient_noalloc writes the same oriented CSR as tc_build_oriented_csr
 * followed by tc_ocsr_copy: rpp_out[n+1] (int64) and colp_out[nnz/2] (int32),
 * both device buffers owned by the caller, N+(u) ascending.  The input is a
 * device CSR as in tc_graph (it is not validated).  Work is enqueued on
 * `stream` on the current device; the call allocates nothing and does not
 * synchronise.  Its only scratch is a fixed 64 KiB device array inside the
 * library, which every GPU that loads the library keeps until the process
 * exits; that caps n at TC_NOALLOC_MAX_VERTICES, and larger graphs get
 * TC_ERR_INVALID_ARG (use tc_build_oriented_csr for them).  The first call on
 * a device looks the array's address up (cudaGetSymbolAddress) and keeps it for
 * the life of the process, so make that first call before any stream capture,
 * and do not call it again after cudaDeviceReset on that device (the array
 * then moves).  All calls share the array: calls whose work overlaps on the
 * GPU race and must be serialised by the caller. */
#define TC_NOALLOC_MAX_VERTICES (1LL << 24)
tc_status tc_orient_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                            int64_t* rpp_out, int32_t* colp_out, void* stream);

/* A batch of G independent graphs (no counterpart in the paper, which counts
 * one graph at a time; each graph is the problem of Sec. 3).  Graph i has
 * n_i = vtx_off[i+1]-vtx_off[i] vertices and nnz_i = edge_off[i+1]-edge_off[i]
 * CSR entries; row_ptr[sum n_i + 1] holds offsets into the concatenated col
 * array, and col holds LOCAL ids in [0, n_i).  All four arrays are device
 * memory, or host memory with TC_IN_HOST.  Each graph must be a valid CSR as
 * in tc_graph (TC_VALIDATE checks it). */
typedef struct tc_batch {
    int64_t G;
    const int64_t* vtx_off;    /* [G+1] */
    const int64_t* edge_off;   /* [G+1] */
    const int64_t* row_ptr;    /* [vtx_off[G]+1] */
    const int32_t* col;        /* [edge_off[G]] */
    uint32_t flags;
} tc_batch;

/* Count every graph of the batch in one pass of the pipeline over their
 * disjoint union: totals[i] = triangles of graph i (G entries);
 * per_vertex[vtx_off[i] + v] = t(v) of graph i when per_vertex != NULL.
 * Output placement and synchronisation as in tc_count. */
tc_status tc_count_batch(tc_ctx* ctx, const tc_batch* b, int64_t* totals, int64_t* per_vertex, void* stream);

/* Capture the whole batch pipeline (build + count) once into a CUDA graph and
 * replay it: for repeated batches of the same shape (same G, offsets and
 * sizes; contents of row_ptr/col may change in place).  The first call
 * captures and replays; later calls with the same plan replay only.  All
 * pointers must be device memory and stay valid while the plan lives. */
typedef struct tc_batch_plan tc_batch_plan;
tc_status tc_batch_plan_create(tc_ctx* ctx, const tc_batch* b, int64_t* totals, int64_t* per_vertex,
                               void* stream, tc_batch_plan** out);
tc_status tc_batch_plan_launch(tc_batch_plan* plan, void* stream);
void tc_batch_plan_destroy(tc_batch_plan* plan);

/* ---- serving: continuous batching of count requests ----------------------
 * A server owns a request thread, `slots` CUDA streams and an HBM budget.
 * tc_submit copies the request's host arrays, queues it and returns at once
 * with a ticket.  The request thread admits queued requests in arrival order
 * while a slot is free and the bytes of resident oriented CSRs plus the
 * request's estimate fit the budget, builds the oriented CSR on the slot's
 * stream, counts it, and retires it when its stream is done; requests that
 * arrive while others are on the GPU overlap with them.  Oriented CSRs of
 * retired requests stay resident (keyed by the caller's graph_key, LRU
 * eviction under the budget), so a repeated key skips the build.
 * Results are exact and identical whether a request runs alone or in a mix. */
typedef struct tc_server tc_server;
typedef struct tc_server_config {
    int32_t device;
    int32_t slots;             /* concurrent requests on the GPU (streams); default 8 */
    int64_t hbm_budget_bytes;  /* default 40 GiB */
    int32_t per_vertex;        /* 1 = also return t(v) */
    int32_t batch_graphs;      /* up to this many small requests waiting at the head of the queue
                                  (host CSR, no TC_VALIDATE, not resident) are fused into one batched
                                  build + count on one slot; default 32; 1 = never fuse */
    int64_t batch_nnz;         /* a request is small when its CSR has at most this many entries and
                                  vertices; a fused batch holds at most 8x this many entries;
                                  default 2^20 */
    int32_t reserved[4];
} tc_server_config;

typedef struct tc_result {
    tc_status status;          /* TC_OK, TC_PENDING or an error */
    int64_t total;
    int64_t n;                 /* length of per_vertex */
    const int64_t* per_vertex; /* host memory owned by the server; valid until the ticket is released */
    double submit_to_done_ms;  /* latency: tc_submit -> result ready on the host */
    double queue_ms;           /* time spent waiting for admission */
    int32_t cache_hit;         /* 1 if the oriented CSR was resident */
} tc_result;

tc_status tc_server_create(const tc_server_config* cfg, const tc_config* tuning, tc_server** out);
/* Stops the request thread after finishing admitted work; frees everything. */
void tc_server_destroy(tc_server* s);
/* g must be a host-memory CSR (flags may include TC_VALIDATE); graph_key != 0
 * names the graph for the resident cache (0 = do not cache). */
tc_status tc_submit(tc_server* s, const tc_graph* g, uint64_t graph_key, uint64_t* ticket);
/* Non-blocking.  TC_PENDING until done; then the result (and its status). */
tc_status tc_poll(tc_server* s, uint64_t ticket, tc_result* out);
/* Block until the ticket is done or timeout_ms elapses (TC_ERR_TIMEOUT). */
tc_status tc_wait(tc_server* s, uint64_t ticket, int64_t timeout_ms, tc_result* out);
/* Forget a finished ticket and free its host result. */
tc_status tc_release(tc_server* s, uint64_t ticket);
/* Counters: requests admitted, finished, cache hits, bytes resident, fused batches. */
typedef struct tc_server_stats {
    int64_t submitted, admitted, finished, cache_hits, evictions;
    int64_t resident_bytes, peak_inflight_bytes;
    int32_t peak_inflight;
    int64_t batches, batched_requests;  /* fused batches run, and the requests they carried */
} tc_server_stats;
tc_status tc_server_get_stats(const tc_server* s, tc_server_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
