// tc_internal.cuh -- shared declarations of the CUDA path (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

constexpr int kWarp = 32;

// Device-side counters of one oriented CSR (written by the build, read by the
// count kernels).
struct DevCounters {
    unsigned long long n_items_warp;   // work items of the warp-table class
    unsigned long long n_items_cta;    // work items of the CTA-table class
    unsigned long long n_pivot_edges;  // oriented edges assigned to a pivot
    unsigned long long n_small_edges;  // oriented edges merged thread-per-edge
    unsigned long long n_merge_edges;  // oriented edges of the warp merge-path class
    int error;                         // validation verdict (0 = ok)
    int max_dplus;                     // max out-degree after orientation
    int max_deg;                       // max degree of the input
};

// One unit of pivot work: intersect the pivot's list segment
// N+(p)[seg*cap .. seg*cap+cap) with N+(q) for the partners q in
// pcol[prp[p]+pb .. prp[p]+pe).
struct __align__(16) Item {
    int p, seg, pb, pe;
};

struct Tuning {
    int small_max = 8;
    int warp_max = 128;
    int table_cap = 1024;
    int probe = 1;          // 1 hash, 2 binary search
    int cta_threads = 256;
    int chunk = 512;
    int bitmap_bits = 131072;  // CTA items whose list spans <= this many rank ids use a bitmap
    int direct_span = 16384;   // ... and <= this many a direct 16-bit cell per rank id
    int merge_ratio = 0;       // percent; balanced edges (max/min d+ <= ratio, max <= merge_max) merge; 0 = off
    int merge_max = 256;
    int stage = 0;             // CTA kernel: 1 = lists of >= 4 lanes per partner staged by the copy engine; 0 = per-lane loads
    int small_lanes = 1;       // threads per row of the thread-merge class (power of two, <= 32)
};

}  // namespace tc

namespace tc {
// Start of row u in colr: rpp[u] + 3u rounded up to a multiple of 4.  Rows
// are 16-byte aligned and disjoint: the gap to the next start is a multiple
// of 4 of at least d+(u), so each row has room for its padding, and no offset
// array or scan is needed (colr holds at most m + 3n + 3 entries).
__host__ __device__ __forceinline__ int64_t colr_row_of(int64_t rpp_u, int64_t u) {
    return (rpp_u + 3 * u + 3) & ~(int64_t)3;
}
__host__ __device__ __forceinline__ int64_t colr_row(const int64_t* rpp, int64_t u) { return colr_row_of(rpp[u], u); }
// colr rows with kSortedMin <= d+(u) <= kSortedMax are partitioned by the
// level of each rank id x, rank_level(n - x) (an eighth of an octave of the
// distance to the top rank: non-increasing in x), into buckets of descending
// level, i.e. ascending x from bucket to bucket (unordered inside a bucket).
// A count kernel walking such a list from the top may stop at a vector whose
// elements all lie in levels above that of a table's smallest key: every
// element before it is then below that key.  Other rows keep vertex-id order.
#ifndef TC_SORTED_MIN
#define TC_SORTED_MIN 64
#endif
#ifndef TC_SORTED_MAX
#define TC_SORTED_MAX 1024
#endif
constexpr int kSortedMin = TC_SORTED_MIN;
constexpr int kSortedMax = TC_SORTED_MAX;
constexpr int kRankLevels = 256;  // 32 octaves x 8
__device__ __forceinline__ int rank_level(unsigned y) {  // 1 <= y < 2^32
    const int e = 31 - __clz(y);
    const unsigned sub = e >= 3 ? (y >> (e - 3)) & 7u : (y << (3 - e)) & 7u;
    return e * 8 + (int)sub;
}
}  // namespace tc

// Library-owned oriented CSR and its work partition.
struct tc_ocsr {
    int device = 0;
    int64_t n = 0, m = 0;
    int64_t* rpp = nullptr;     // [n+1] oriented row offsets
    int32_t* colp = nullptr;    // [m]
    int32_t* dplus = nullptr;   // [n] out-degrees
    int32_t* deg = nullptr;     // [n] undirected degrees
    int32_t* rank = nullptr;    // [n] position of each vertex in (degree, id) order
    int32_t* perm = nullptr;    // [n] inverse of rank
    int32_t* colr = nullptr;    // colp relabelled to rank ids; row u at colr_row(rpp, u), padded with -1 to 4k entries
    int2* rspan = nullptr;      // [n] smallest and largest rank id of each row with d+ > warp_max (others unset)
    int64_t* prp = nullptr;     // [n+1] partner row offsets
    int32_t* pcol = nullptr;    // [m] partners (only the first n_pivot_edges used)
    int2* pdesc = nullptr;      // [m] beside pcol: (first 16-byte vector of the partner's colr row, its d+)
    tc::Item* items_warp = nullptr;
    tc::Item* items_cta = nullptr;
    int64_t items_warp_cap = 0, items_cta_cap = 0;
    int2* medge = nullptr;      // oriented edges (u, v) of the merge-path class (first n_merge_edges used)
    int64_t medge_cap = 0;
    tc::DevCounters* dc = nullptr;
    // batch mode: vertex -> graph id and the number of graphs
    int32_t* row_graph = nullptr;
    int64_t G = 0;
    tc::Tuning tun;             // thresholds the partition was built with
    int64_t bytes = 0;
};

struct tc_ctx {
    int device = 0;
    int num_sms = 0;
    tc::Tuning tun;
    std::string err;
    // tracing: kernel launches issued, and CUDA-event pairs per phase
    bool trace = false;
    long long launches = 0;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
};

namespace tc {

// Phase ids of the trace (tc_trace.phase_ms index).
enum Phase {
    kPhDegree = 0, kPhValidate, kPhOrientCount, kPhOrientScan, kPhOrientScatter, kPhPivotCount, kPhPivotScan,
    kPhPivotScatter, kPhItems, kPhCountSmall, kPhCountWarp, kPhCountCta, kPhEdgeSort, kPhCountInit, kPhRank,
    kPhRowSort, kPhCountMerge, kPhFused, kNumPhases
};

// RAII phase marker: records an event pair on `s` when tracing is on.
struct PhaseScope {
    tc_ctx* c;
    int id;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(tc_ctx* c_, int id_, cudaStream_t s_);
    ~PhaseScope();
};
#define TC_LAUNCH(ctx) ((ctx)->launches++)

// status helpers
tc_status set_err(tc_ctx* ctx, tc_status st, const std::string& msg);
tc_status cuda_err(tc_ctx* ctx, cudaError_t e, const char* where);

// stream-ordered allocation from the device pool
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// device-wide exclusive scan: out[0..n] (n+1 entries) of int32 in[0..n)
cudaError_t scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                            cudaStream_t s);
size_t scan_tmp_bytes(int64_t n);

// Build the oriented CSR and its partition from a device CSR (rows may be a
// batch: row_graph/vtx_off non-null map local neighbour ids to global ones).
// col_src (single graph, no validation): the entries are read from this
// device-accessible address of a pinned host array by the first pass over
// them, which writes them into col, then a device buffer of nnz entries.
tc_status build_from_device_csr(tc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                const int32_t* col, const int64_t* vtx_off, int64_t G,
                                bool validate, tc_ocsr** out, cudaStream_t s, const int32_t* col_src = nullptr);

// Stable LSD radix sort of uint64 keys on bits [low_bit, key_bits).  With
// maxv (device), bits [vbase, ...) of every key are at most *maxv, and the
// passes over digits that are then zero for all keys do nothing: the result
// is then in ka after an even number of real passes, in kb after an odd one.
cudaError_t radix_sort_u64(unsigned long long* ka, unsigned long long* kb, int64_t K, int key_bits, cudaStream_t s,
                           unsigned long long** sorted, long long* launches, int low_bit,
                           const int* maxv = nullptr, int vbase = 0);

// Canonicalise a device edge list into a device CSR (library-owned buffers).
tc_status edges_to_csr(tc_ctx* ctx, int64_t n, int64_t npairs, const int32_t* src, const int32_t* dst,
                       int64_t** row_ptr, int32_t** col, int64_t* nnz, cudaStream_t s);

// Launch the count kernels.  totals: device int64 [G or 1], zeroed here.
// shard/nshards: the launch covers that equal part of the work lists (0/1 = all).
// tc_fused.cu: the whole method for one small graph in one kernel launch
// (n <= kFusedMaxN, its arrays within kFusedMaxSmem bytes of one CTA's shared
// memory; every CTA of the launch holds the whole oriented graph)
constexpr int64_t kFusedMaxN = 8192;
constexpr int64_t kFusedMaxSmem = 224 * 1024;
bool fused_fits(int64_t n, int64_t nnz);
cudaError_t launch_fused(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col, unsigned long long* total,
                         unsigned long long* per_vertex, cudaStream_t s);
tc_status count_device(tc_ctx* ctx, const tc_ocsr* o, unsigned long long* totals,
                       unsigned long long* per_vertex, cudaStream_t s, int shard = 0, int nshards = 1);

// Read and clear the device check word of the current device (synchronises s).
cudaError_t take_device_error(cudaStream_t s, unsigned* bits);
// Enqueue a copy of the check word (not cleared) into pinned host memory on s.
cudaError_t peek_device_error_async(unsigned* h_pinned, cudaStream_t s);

}  // namespace tc
