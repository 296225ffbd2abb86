// tc_build.cu -- steps 1-3 of the method on the device: degrees, orientation
// filter, compaction into the oriented CSR, and the work partition.
//
// Paper: Sec. 4.2.1 (advance V2E + filter by degree, ties by id; segmented
// reduction into the induced subgraph), Alg. 2 Form_Filtered_Edge_List and
// Partition, Sec. 4.2.2 (dynamic grouping by list size).
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "tc_internal.cuh"

namespace tc {

// ============================================================================
// Device-wide exclusive scan (reduce-then-scan over 2048-element tiles)
// ============================================================================
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long warp_incl_scan(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan; sm needs blockDim/32 + 1 slots.  Returns the
// exclusive prefix; *total receives the block sum.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sm, long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc = warp_incl_scan(v);
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long t = lane < nw ? sm[lane] : 0;
        long long ti = warp_incl_scan(t);
        if (lane < nw) sm[lane] = ti - t;
        if (lane == 31) sm[32] = ti;
    }
    __syncthreads();
    long long r = sm[w] + inc - v;
    *total = sm[32];
    __syncthreads();
    return r;
}

// skip (nullable): a device count; when it is zero the scan is not needed
// (its input is all zeros and its consumers skip too) and every kernel of
// the scan returns at once.
__device__ __forceinline__ bool scan_skipped(const unsigned long long* skip) { return skip && *skip == 0ull; }

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                              long long* __restrict__ tile_sum,
                                                              const unsigned long long* __restrict__ skip) {
    if (scan_skipped(skip)) return;
    __shared__ long long sm[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    long long tot;
    block_excl_scan(s, sm, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(long long* __restrict__ tile_sum, int64_t ntiles,
                                                    int64_t* __restrict__ out, int64_t n,
                                                    const unsigned long long* __restrict__ skip) {
    if (scan_skipped(skip)) return;
    __shared__ long long sm[33];
    long long carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        long long v = i < ntiles ? tile_sum[i] : 0;
        long long tot;
        long long ex = block_excl_scan(v, sm, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                                                             const long long* __restrict__ tile_off,
                                                             int64_t* __restrict__ out,
                                                             const unsigned long long* __restrict__ skip) {
    if (scan_skipped(skip)) return;
    __shared__ long long sm[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        s += v[j];
    }
    long long tot;
    long long run = tile_off[blockIdx.x] + block_excl_scan(s, sm, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}

size_t scan_tmp_bytes(int64_t n) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    return (size_t)std::max<int64_t>(nt, 1) * sizeof(long long);
}

// scan_i32_to_i64 that does nothing (out left unwritten) when *skip (device) is 0
static cudaError_t scan_i32_to_i64_unless_zero(const int32_t* in, int64_t* out, int64_t n, void* tmp,
                                               size_t tmp_bytes, cudaStream_t s, const unsigned long long* skip) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (tmp_bytes < scan_tmp_bytes(n)) return cudaErrorInvalidValue;
    long long* ts = (long long*)tmp;
    if (nt > 0) k_scan_reduce<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ts, skip);
    k_scan_sums<<<1, 1024, 0, s>>>(ts, nt, out, n, skip);
    if (nt > 0) k_scan_apply<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ts, out, skip);
    return cudaGetLastError();
}

cudaError_t scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                            cudaStream_t s) {
    return scan_i32_to_i64_unless_zero(in, out, n, tmp, tmp_bytes, s, nullptr);
}

// ============================================================================
// a-1  degree: d(v) = row_ptr[v+1] - row_ptr[v]
// ============================================================================
__global__ void k_degree(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ deg, int* __restrict__ max_deg) {
    int mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int32_t)(rp[v + 1] - rp[v]);
        deg[v] = d;
        mx = max(mx, d);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(max_deg, mx);
}

// batch: row_graph[v] = graph of global vertex v
__global__ void k_row_graph(int64_t G, const int64_t* __restrict__ vtx_off, int32_t* __restrict__ row_graph) {
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x)
        for (int64_t v = vtx_off[g] + threadIdx.x; v < vtx_off[g + 1]; v += blockDim.x) row_graph[v] = (int32_t)g;
}

// rank(v) = position of v in (degree, id) order: sort keys deg << b | v
__global__ void k_rank_keys(int64_t n, const int32_t* __restrict__ deg, int b, unsigned long long* __restrict__ keys) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((unsigned long long)deg[v] << b) | (unsigned long long)v;
}

// The sort ran 8-bit passes over the degree bits [b, 2b) of the keys; the
// passes above the highest set bit of the maximum degree did nothing, so the
// keys are in ka after an even number of real passes, in kb after an odd one.
__global__ void k_rank_from_sorted(int64_t n, const unsigned long long* __restrict__ ka,
                                   const unsigned long long* __restrict__ kb, const int* __restrict__ max_deg, int b,
                                   int32_t* __restrict__ rank, int32_t* __restrict__ perm) {
    int real = 0;
    for (int shift = b; shift < 2 * b; shift += 8) real += ((unsigned)*max_deg >> (shift - b)) != 0u;
    const unsigned long long* __restrict__ sorted = (real & 1) ? kb : ka;
    const unsigned long long mask = (1ull << b) - 1ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(sorted[r] & mask);
        perm[r] = v;
        rank[v] = (int32_t)r;
    }
}

// ============================================================================
// validation of a CSR input (TC_VALIDATE): ids in range, rows strictly
// ascending (sorted, no duplicates), no self-loops, symmetric.
// ============================================================================
__device__ __forceinline__ bool row_contains(const int32_t* __restrict__ col, int64_t b, int64_t e, int32_t x) {
    while (b < e) {
        int64_t mid = (b + e) >> 1;
        int32_t y = col[mid];
        if (y == x) return true;
        if (y < x) b = mid + 1; else e = mid;
    }
    return false;
}

__global__ void k_validate(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ row_graph, const int64_t* __restrict__ vtx_off,
                           int* __restrict__ err) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(err, 1);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = rp[u], e = rp[u + 1];
        if (b > e || b < 0 || e > nnz) { atomicOr(err, 2); continue; }
        int64_t lo = 0, hi = n;  // id range of u's graph (global ids)
        if (row_graph) { int g = row_graph[u]; lo = vtx_off[g]; hi = vtx_off[g + 1]; }
        int64_t base = row_graph ? lo : 0;
        int32_t prev = -1;
        for (int64_t i = b; i < e; ++i) {
            int64_t v = (int64_t)col[i] + base;
            if (col[i] < 0 || v >= hi) { atomicOr(err, 4); break; }
            if (col[i] <= prev) { atomicOr(err, 8); break; }
            if (v == u) { atomicOr(err, 16); break; }
            prev = col[i];
            int32_t want = (int32_t)(u - base);
            int64_t vb = rp[v], ve = rp[v + 1];
            if (vb > ve || vb < 0 || ve > nnz || !row_contains(col, vb, ve, want)) { atomicOr(err, 32); break; }
        }
    }
}

// ============================================================================
// Merge-path tiles over a CSR (rows i, entries j).  The merged sequence of the
// n row ends and the nnz entries is cut into tiles of kMpTile items, so every
// tile carries the same work whatever the degrees: a tile of one hub row and
// a tile of a thousand one-entry rows cost the same.  Boundary t of the cut is
// the coordinate (i, j) = (rows ended, entries consumed) on diagonal
// t * kMpTile, found by binary search (a row end is taken before an entry
// with the same offset).
// ============================================================================
// CTA work items carry this many times `chunk` partners (one table build and
// flush serve them all).  At most 32767 partners keep the 16-bit direct cells
// exact.  At most (2^31 - 1) / (max d+ + 15) partners keep every 32-bit direct
// cell of the count kernel below its marker bit: a cell inside the table's
// span gains at most one count per partner (a list holds each id once), and
// each of the 32 dummy cells past the span belongs to one lane and takes that
// lane's probes outside the span.  A lane probes at most its share of a
// partner's list rounded up to whole batches of 16 elements (row padding and
// the -1 fill past the list's start included), at most d+ + 15 per partner,
// so at most partners x (max d+ + 15) in all.
#ifndef TC_CTA_CHUNK_MUL
#define TC_CTA_CHUNK_MUL 2
#endif
constexpr int kMpThreads = 256;
#ifndef TC_MP_IPT
#define TC_MP_IPT 8
#endif
constexpr int kMpIpt = TC_MP_IPT;   // items per thread of a tile (a multiple of 8)
static_assert(kMpIpt % 8 == 0, "tile rows are handled as 16-byte vectors of 8 entries");
constexpr int kRowVec = kMpIpt / 8;
constexpr int kMpTile = kMpThreads * kMpIpt;
// resident CTAs per SM the tile kernels are compiled for (registers permitting):
// they wait on scattered loads, so more warps in flight hide more latency
#ifndef TC_MP_MIN_BLOCKS
#define TC_MP_MIN_BLOCKS 5
#endif
#ifndef TC_MP_SCATTER_MIN_BLOCKS
#define TC_MP_SCATTER_MIN_BLOCKS 4
#endif

int64_t mp_tiles(int64_t n, int64_t nnz) { return (n + nnz + kMpTile - 1) / kMpTile; }

__global__ void k_mp_coords(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, int64_t ntiles,
                            longlong2* __restrict__ coord) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = min(t * (int64_t)kMpTile, n + nnz);
        int64_t lo = max((int64_t)0, d - nnz), hi = min(d, n);
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid + 1] <= d - 1 - mid) lo = mid + 1;
            else hi = mid;
        }
        coord[t] = make_longlong2(lo, d - lo);
    }
}

// Shared state of one tile: local rows i0 .. i0+nr-1 and entries j0 .. j0+ne-1.
template <bool BATCH>
struct MpTile {
    int cs[kMpTile + 2];                        // row starts relative to j0, clamped to [0, ne]
    int du[kMpTile + 1];                        // full length of each local row
    int base[BATCH ? kMpTile + 1 : 1];          // batch: first global id of the row's graph
    __align__(16) unsigned short row[kMpTile];  // local row of each entry
    int wmax[kMpThreads / 32];
    long long i0, j0;
    int nr, ne, nend;                           // rows whose end lies in the tile: the first nend
    int first_full;                             // local row 0 starts at j0 (it is not a continuation)
};

// Fill S for the tile between cut coordinates c0 and c1.  Ends with a
// barrier.  The callers issue their loads of the tile's entries (which need
// only c0 and c1) before this call, so that those loads are in flight while
// the rows are laid out here.
template <bool BATCH>
__device__ void mp_tile(MpTile<BATCH>& S, longlong2 c0, longlong2 c1, int64_t n, const int64_t* __restrict__ rp,
                        const int32_t* __restrict__ row_graph, const int64_t* __restrict__ vtx_off) {
    const int64_t i0 = c0.x, j0 = c0.y;
    const int ne = (int)(c1.y - j0);
    const int nr = (int)max((int64_t)0, min((int64_t)c1.x, n - 1) - i0 + 1);
    for (int k = threadIdx.x; k <= nr; k += blockDim.x) {
        const int64_t s = rp[i0 + k];
        S.cs[k] = (int)min(max(s - j0, (int64_t)0), (int64_t)ne);
        if (k < nr) {
            S.du[k] = (int)(rp[i0 + k + 1] - s);
            if (BATCH) S.base[k] = (int)vtx_off[row_graph[i0 + k]];
        }
    }
#pragma unroll
    for (int c = 0; c < kRowVec; ++c) reinterpret_cast<uint4*>(S.row)[threadIdx.x * kRowVec + c] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        S.i0 = i0;
        S.j0 = j0;
        S.nr = nr;
        S.ne = ne;
        S.nend = (int)(c1.x - i0);
        S.first_full = nr > 0 && rp[i0] == j0;
    }
    __syncthreads();
    // every row with entries here marks its first one; a running maximum then
    // gives each entry its row (rows with entries have distinct starts)
    for (int k = 1 + threadIdx.x; k < nr; k += blockDim.x)
        if (S.cs[k] < S.cs[k + 1]) S.row[S.cs[k]] = (unsigned short)k;
    __syncthreads();
    uint4 pk[kRowVec];
#pragma unroll
    for (int c = 0; c < kRowVec; ++c) pk[c] = reinterpret_cast<uint4*>(S.row)[threadIdx.x * kRowVec + c];
    unsigned short* v = reinterpret_cast<unsigned short*>(pk);
    int run = 0;
#pragma unroll
    for (int q = 0; q < kMpIpt; ++q) {
        run = max(run, (int)v[q]);
        v[q] = (unsigned short)run;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, y);
    }
    if (lane == 31) S.wmax[w] = inc;
    int before = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) before = 0;
    __syncthreads();
    for (int k = 0; k < w; ++k) before = max(before, S.wmax[k]);
#pragma unroll
    for (int q = 0; q < kMpIpt; ++q) v[q] = (unsigned short)max(before, (int)v[q]);
#pragma unroll
    for (int c = 0; c < kRowVec; ++c) reinterpret_cast<uint4*>(S.row)[threadIdx.x * kRowVec + c] = pk[c];
    __syncthreads();
}

// Batch mode: the first global id of the graph that owns every row of the
// tile between cut coordinates c0 and c1, or -1 when the tile spans more
// than one graph (graphs hold tens of thousands of entries, tiles 2048 items,
// so almost every tile lies inside one graph).  Needs no shared state, so a
// tile kernel can offset and gather its entries before mp_tile.
__device__ __forceinline__ int64_t tile_graph_base(longlong2 c0, longlong2 c1, int64_t n,
                                                   const int32_t* __restrict__ row_graph,
                                                   const int64_t* __restrict__ vtx_off) {
    if (n <= 0) return -1;
    const int64_t ia = min((int64_t)c0.x, n - 1), ib = min((int64_t)c1.x, n - 1);
    const int32_t ga = row_graph[ia];
    return ga == row_graph[ib] ? vtx_off[ga] : -1;
}

// OR the ballot of 32 consecutive entries starting at global index g into a bitmask.
__device__ __forceinline__ void or_bits(unsigned* __restrict__ mask, int64_t g, unsigned bal) {
    if (!bal) return;
    const int64_t w = g >> 5;
    const int sh = (int)(g & 31);
    atomicOr(&mask[w], bal << sh);
    if (sh) {
        const unsigned hi = bal >> (32 - sh);
        if (hi) atomicOr(&mask[w + 1], hi);
    }
}

// number of set bits of mask before global index g (pre = exclusive prefix of word popcounts)
__device__ __forceinline__ int64_t bits_before(const unsigned* __restrict__ mask, const int64_t* __restrict__ pre, int64_t g) {
    const int64_t w = g >> 5;
    return pre[w] + __popc(mask[w] & ((1u << (g & 31)) - 1u));
}

__global__ void k_popc(const unsigned* __restrict__ mask, int64_t nw, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __popc(mask[i]);
}

// ============================================================================
// a-2 / a-3  orientation filter and compaction (Sec. 4.2.1).
// Entry (u, v) is kept iff rank(u) < rank(v), rank = (d, id).  Pass 1 sets
// one bit per kept entry.  Kept entries keep their input order, so the
// position of a kept entry in the oriented CSR is the number of kept entries
// before it (a prefix count over the bitmask) and rpp[u] is that count at
// row_ptr[u] (k_rows).  Pass 2 scatters the kept neighbours: vertex ids to
// colp, rank ids to colr, whose rows start at multiples of 4 (colr_row) and
// are padded with -1 (colr is cleared to -1 first) so that the count kernels
// read them as whole aligned 16-byte vectors.
// ============================================================================
// Arrays a build kernel reads or writes once, in a stream (the input col,
// the oriented lists while they are scattered and re-read, pcol and pdesc),
// go through the evict-first cache operator (.cs), so that they leave L2
// before the per-vertex arrays (deg, (rank, d+), descriptors) that the same
// kernels gather at random.
template <class T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <class T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// Partition classes of an oriented edge (u, v) with a = d+(u), b = d+(v); see a-4 below.
enum { kSkip = 0, kSmall = 1, kPivot = 2, kMerge = 3 };

__device__ __forceinline__ int edge_class(int a, int b, int small_max, int merge_ratio, int merge_max) {
    if (a <= 1 || b == 0) return kSkip;
    const int hi = max(a, b), lo = min(a, b);
    if (hi <= small_max) return kSmall;
    // the degree-ratio switch: balanced lists of moderate length merge
    if (merge_ratio > 0 && hi <= merge_max && 100ll * hi <= (long long)merge_ratio * lo) return kMerge;
    return kPivot;
}

template <bool BATCH>
__global__ void __launch_bounds__(kMpThreads, TC_MP_MIN_BLOCKS) k_orient_flags(int64_t n, int64_t ntiles, const longlong2* __restrict__ coord,
                                                             const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                             const int32_t* __restrict__ deg, const int32_t* __restrict__ row_graph,
                                                             const int64_t* __restrict__ vtx_off, unsigned* __restrict__ keep,
                                                             int32_t* __restrict__ col_copy) {
    __shared__ MpTile<BATCH> S;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const longlong2 c0 = coord[t], c1 = coord[t + 1];
        const int64_t j0 = c0.y;
        const int ne = (int)(c1.y - j0);
        // the tile's entries and their degree gathers first (8 independent
        // streams, then 8 gathers), in flight while mp_tile lays out the rows
        int32_t vv[kMpIpt];
        int dv[kMpIpt];
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            vv[q] = e < ne ? ld_stream(col + j0 + e) : 0;
        }
        if (col_copy) {  // col is the caller's pinned host array: leave a device copy for the later passes
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int e = q * kMpThreads + threadIdx.x;
                if (e < ne) col_copy[j0 + e] = vv[q];
            }
        }
        // batch: local ids become global with the graph's base, known here
        // when the whole tile lies in one graph
        const int64_t gbase = BATCH ? tile_graph_base(c0, c1, n, row_graph, vtx_off) : 0;
        if (gbase >= 0) {
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                if (BATCH) vv[q] += (int32_t)gbase;
                dv[q] = q * kMpThreads + (int)threadIdx.x < ne ? deg[vv[q]] : 0;
            }
        }
        mp_tile<BATCH>(S, c0, c1, n, rp, row_graph, vtx_off);
        const int64_t i0 = S.i0;
        if (BATCH && gbase < 0) {  // the tile spans graphs: each entry takes its row's base
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int e = q * kMpThreads + threadIdx.x;
                if (e < ne) vv[q] += S.base[S.row[e]];
            }
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) dv[q] = q * kMpThreads + (int)threadIdx.x < ne ? deg[vv[q]] : 0;
        }
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            bool kp = false;
            if (e < ne) {
                const int k = S.row[e];
                const int du = S.du[k];
                kp = du < dv[q] || (du == dv[q] && i0 + k < (int64_t)vv[q]);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) or_bits(keep, j0 + q * kMpThreads + w * 32, bal);
        }
        __syncthreads();
    }
}

// rpp[u] = kept entries before row u, and d+(u) (and its maximum)
// (and (rank(u), d+(u)) packed, so that the scatter gathers both of a
// neighbour with one 8-byte load, and (first vector of u's colr row, d+(u)),
// the descriptor the count kernels read for a partner u)
// ... and the list of the rows k_sort_rows works on (kSortedMin <= d+ <=
// kSortedMax, or d+ > warp_max), appended one global atomic per block and
// iteration (one shared atomic per warp below it).
__global__ void k_rows(int64_t n, const int64_t* __restrict__ rp, const unsigned* __restrict__ keep,
                       const int64_t* __restrict__ kpre, const int32_t* __restrict__ rank, int64_t* __restrict__ rpp,
                       int32_t* __restrict__ dplus, int2* __restrict__ rd2, int2* __restrict__ pd2,
                       int* __restrict__ max_dplus, int warp_max, int32_t* __restrict__ srows,
                       unsigned* __restrict__ n_srows) {
    __shared__ unsigned s_cnt, s_base;
    int mx = 0;
    const int lane = threadIdx.x & 31;
    // block-uniform trip count, so that every thread takes part in each append
    for (int64_t u0 = (int64_t)blockIdx.x * blockDim.x; u0 <= n; u0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = u0 + threadIdx.x;
        bool listed = false;
        if (u <= n) {
            const int64_t s = bits_before(keep, kpre, rp[u]);
            rpp[u] = s;
            if (u < n) {
                const int d = (int)(bits_before(keep, kpre, rp[u + 1]) - s);
                dplus[u] = d;
                rd2[u] = make_int2(rank[u], d);
                pd2[u] = make_int2((int)((s + 3 * u + 3) >> 2), d);  // colr_row(rpp, u) / 4
                mx = max(mx, d);
                listed = (d >= kSortedMin && d <= kSortedMax) || d > warp_max;
            }
        }
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const unsigned m = __ballot_sync(0xffffffffu, listed);
        const int lead = m ? __ffs(m) - 1 : 0;
        unsigned at = 0;
        if (m && lane == lead) at = atomicAdd(&s_cnt, (unsigned)__popc(m));
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt) s_base = atomicAdd(n_srows, s_cnt);
        __syncthreads();
        at = __shfl_sync(0xffffffffu, at, lead);
        if (listed) srows[s_base + at + __popc(m & ((1u << lane) - 1u))] = (int32_t)u;
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(max_dplus, mx);
}

template <bool BATCH>
__global__ void __launch_bounds__(kMpThreads, TC_MP_SCATTER_MIN_BLOCKS) k_orient_scatter(int64_t n, int64_t ntiles, const longlong2* __restrict__ coord,
                                                               const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                               const int2* __restrict__ rd2, const int32_t* __restrict__ row_graph,
                                                               const int64_t* __restrict__ vtx_off, const unsigned* __restrict__ keep,
                                                               const int64_t* __restrict__ kpre, const int64_t* __restrict__ rpp,
                                                               int small_max,
                                                               int merge_ratio, int merge_max, int2* __restrict__ medge,
                                                               int64_t medge_cap,
                                                               int32_t* __restrict__ colp, int32_t* __restrict__ colr,
                                                               unsigned* __restrict__ umask,
                                                               unsigned* __restrict__ vmask, int32_t* __restrict__ nv,
                                                               DevCounters* __restrict__ dc) {
    __shared__ MpTile<BATCH> S;
    __shared__ unsigned long long s_piv, s_small;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) { s_piv = 0; s_small = 0; }
    unsigned long long my_piv = 0, my_small = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const longlong2 c0 = coord[t], c1 = coord[t + 1];
        const int64_t j0 = c0.y;
        const int ne = (int)(c1.y - j0);
        // the tile's keep bits and entries, and the (rank, d+) gathers of the
        // kept ones, first: in flight while mp_tile lays out the rows
        unsigned kmask = 0;  // bit q: entry q is kept
        int32_t vv[kMpIpt];
        int rr[kMpIpt], bb[kMpIpt];
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            vv[q] = 0;
            rr[q] = bb[q] = 0;
            if (e < ne) {
                const int64_t g = j0 + e;
                kmask |= ((keep[g >> 5] >> (g & 31)) & 1u) << q;
                vv[q] = ld_stream(col + g);
            }
        }
        const int64_t gbase = BATCH ? tile_graph_base(c0, c1, n, row_graph, vtx_off) : 0;
        if (gbase >= 0) {  // batch: the whole tile lies in one graph
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                if (BATCH) vv[q] += (int32_t)gbase;
                const int2 rv = (kmask >> q) & 1u ? rd2[vv[q]] : make_int2(0, 0);
                rr[q] = rv.x;
                bb[q] = rv.y;
            }
        }
        // the first row of this thread's share of the tile's rows: its rpp
        // and d+ loads, too, need only the cut coordinates
        const int64_t ia = c0.x;
        const int nr0 = (int)max((int64_t)0, min((int64_t)c1.x, n - 1) - ia + 1);
        int r3 = 0, dr = 0;
        if ((int)threadIdx.x < nr0) {
            const int64_t u = ia + threadIdx.x;
            r3 = (int)((rpp[u] + 3 * u + 3) & 3);
            dr = rd2[u].y;
        }
        mp_tile<BATCH>(S, c0, c1, n, rp, row_graph, vtx_off);
        const int64_t i0 = S.i0;
        const int nr = S.nr;
        // colr position of a kept entry = its colp position + colr_row(u) - rpp[u]
        // = pos + 3u + 3 - r, r = (rpp[u] + 3u + 3) mod 4 (kept in du, which is
        // not needed here; the offset itself exceeds 32 bits for large u).
        // cs, used only to find each entry's row, now holds d+ of the row.
        if ((int)threadIdx.x < nr) {
            S.du[threadIdx.x] = r3;
            S.cs[threadIdx.x] = dr;
        }
        for (int k = threadIdx.x + blockDim.x; k < nr; k += blockDim.x) {
            const int64_t u = i0 + k;
            S.du[k] = (int)((rpp[u] + 3 * u + 3) & 3);
            S.cs[k] = rd2[u].y;
        }
        __syncthreads();
        if (BATCH && gbase < 0) {  // the tile spans graphs: each entry takes its row's base
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int e = q * kMpThreads + threadIdx.x;
                if (e < ne) vv[q] += S.base[S.row[e]];
            }
#pragma unroll
            for (int q = 0; q < kMpIpt; ++q) {
                const int2 rv = (kmask >> q) & 1u ? rd2[vv[q]] : make_int2(0, 0);
                rr[q] = rv.x;
                bb[q] = rv.y;
            }
        }
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            const bool valid = e < ne;
            const bool kq = (kmask >> q) & 1u;
            // the warp's 32 entries are consecutive, so its kept ones sit at
            // consecutive positions from the first one's: p0 + the kept lanes below
            const unsigned kb = __ballot_sync(0xffffffffu, kq && valid);
            int64_t p0 = 0, pos = 0;
            if (kb) {
                p0 = bits_before(keep, kpre, j0 + q * kMpThreads + (threadIdx.x & ~31u));  // the same for the warp
                pos = p0 + __popc(kb & ((1u << lane) - 1u));
            }
            bool pu = false, pv = false, mg = false;
            int mu = 0;
            if (valid) {
                const int k = S.row[e];
                if (kq) {
                    st_stream(colp + pos, vv[q]);
                    st_stream(colr + pos + 3 * (i0 + k) + 3 - S.du[k], rr[q]);
                    // a-4 classification of the oriented edge (u, v) at position pos
                    const int a = S.cs[k], b = bb[q];
                    const int cls = edge_class(a, b, small_max, merge_ratio, merge_max);
                    pu = cls == kPivot && a >= b;
                    pv = cls == kPivot && a < b;
                    mg = cls == kMerge;
                    mu = (int)(i0 + k);
                    my_small += cls == kSmall;
                    my_piv += pu || pv;
                    if (pv) atomicAdd(&nv[vv[q]], 1);
                }
            }
            // merge-class edges are appended to their list, one atomic per warp
            const unsigned mb = merge_ratio > 0 ? __ballot_sync(0xffffffffu, mg) : 0u;
            if (mb) {
                const int lead = __ffs(mb) - 1;
                unsigned long long base = 0;
                if (lane == lead) base = atomicAdd(&dc->n_merge_edges, (unsigned long long)__popc(mb));
                base = __shfl_sync(0xffffffffu, base, lead);
                const unsigned long long at = base + __popc(mb & ((1u << lane) - 1u));
                if (mg && at < (unsigned long long)medge_cap) medge[at] = make_int2(mu, vv[q]);
            }
            // one bit pattern per mask, placed at the first kept entry's position
            if (kb) {
                const unsigned lt = (1u << lane) - 1u;
                const int idx = __popc(kb & lt);
                const unsigned ub = __reduce_or_sync(0xffffffffu, pu ? (1u << idx) : 0u);
                const unsigned vb2 = __reduce_or_sync(0xffffffffu, pv ? (1u << idx) : 0u);
                const int first = __ffs(kb) - 1;
                if (lane == first) {
                    or_bits(umask, p0, ub);
                    or_bits(vmask, p0, vb2);
                }
            }
        }
        __syncthreads();
    }
    for (int o = 16; o; o >>= 1) {
        my_piv += __shfl_xor_sync(0xffffffffu, my_piv, o);
        my_small += __shfl_xor_sync(0xffffffffu, my_small, o);
    }
    if (lane == 0) { atomicAdd(&s_piv, my_piv); atomicAdd(&s_small, my_small); }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&dc->n_pivot_edges, s_piv);
        atomicAdd(&dc->n_small_edges, s_small);
    }
}


// Two jobs on the colr rows, one warp per row:
//  * rspan[u] = (smallest, largest) rank id of every row with d+ > warp_max,
//    the rows a CTA table may be built from (the CTA kernel reads it to pick
//    the table kind of a whole-row item);
//  * rows with kSortedMin <= d+ <= kSortedMax are partitioned into buckets of
//    descending rank_level(n - x) (see tc_internal.cuh): the row is staged in
//    the warp's shared-memory buffer, levels are counted, their exclusive
//    prefix taken in descending order, and the row scattered back.
#ifndef TC_SORT_WARPS
#define TC_SORT_WARPS 4
#endif
constexpr int kSortWarps = TC_SORT_WARPS;

__global__ void __launch_bounds__(32 * kSortWarps) k_sort_rows(int64_t n, const int64_t* __restrict__ rpp,
                                                               const int32_t* __restrict__ dplus,
                                                               const int32_t* __restrict__ srows,
                                                               const unsigned* __restrict__ n_srows,
                                                               int32_t* __restrict__ colr, int2* __restrict__ rspan) {
    const unsigned nl = *n_srows;  // the rows k_rows listed
    if (nl == 0u) return;
    extern __shared__ int sbuf[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* buf = sbuf + w * (kSortedMax + kRankLevels);
    int* cur = buf + kSortedMax;  // per level: count, then next free position
    const unsigned nwarps = gridDim.x * kSortWarps;
    for (unsigned li = blockIdx.x * kSortWarps + w; li < nl; li += nwarps) {  // one listed row per warp
        {
            const int64_t u = srows[li];
            const int d = dplus[u];
            const bool part = d >= kSortedMin && d <= kSortedMax;
            int32_t* row = colr + colr_row(rpp, u);
            int mn = 0x7fffffff, mx = -1;
            if (part) {
                for (int i = lane; i < kRankLevels; i += 32) cur[i] = 0;
                __syncwarp();
            }
            for (int i = lane; i < d; i += 32) {
                const int x = row[i];
                mn = min(mn, x);
                mx = max(mx, x);
                if (part) {
                    buf[i] = x;
                    atomicAdd(&cur[rank_level((unsigned)(n - x))], 1);
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) rspan[u] = make_int2(mn, mx);
            if (!part) continue;
            __syncwarp();
            // exclusive prefix over levels kRankLevels-1 .. 0 (lane l: 8 levels)
            int c[8], t = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = cur[kRankLevels - 1 - (lane * 8 + j)];
                t += c[j];
            }
            int inc = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int run = inc - t;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                cur[kRankLevels - 1 - (lane * 8 + j)] = run;
                run += c[j];
            }
            __syncwarp();
            for (int i = lane; i < d; i += 32) {
                const int x = buf[i];
                row[atomicAdd(&cur[rank_level((unsigned)(n - x))], 1)] = x;
            }
            __syncwarp();
        }
    }
}

// ============================================================================
// a-4  partition (Alg. 2 Partition; Sec. 4.2.2 dynamic grouping).
// Every oriented edge (u, v) with a = d+(u), b = d+(v) falls in one class:
//   skip  : a <= 1 or b == 0 (N+(u) = {v} or N+(v) empty: no common vertex);
//   small : max(a, b) <= small_max -> one thread merges the two lists;
//   merge : (when the degree-ratio switch is on) max(a, b) <= merge_max and
//           max(a, b) <= merge_ratio/100 * min(a, b): balanced lists, merged
//           by one warp along the merge path of both (the paper's TwoLarge
//           intersection of Sec. 4.2.2); appended to the merge edge list;
//   pivot : otherwise.  The endpoint with the longer list is the pivot p (u
//           on ties), the other is the partner q.  The pivot's list becomes a
//           shared-memory table and the partner's (shorter) list is streamed
//           against it: the "small x large" kernel the paper proposes in its
//           Sec. 5 discussion, applied to every non-small edge.
// The partners of pivot p are stored at pcol[prp[p] .. prp[p+1]): first the
// U-part, the entries of p's own row with p as pivot, in row order; then the
// V-part, the rows u whose entry (u, p) made p the pivot.  With
//   U(x)    = number of U-part entries of the oriented CSR before entry x,
//   nV(p)   = size of p's V-part, Vpre(p) = sum of nV(q) over q < p,
// prp[p] = U(rpp[p]) + Vpre(p), a U-part entry x of row u lands at
// U(x) + Vpre(u), and the V-part of p fills the slots just below prp[p+1].
// The classification itself (the U and V bit masks over the oriented entries
// and nV) is done by k_orient_scatter as it places each kept entry.
// ============================================================================

// prp[p] = U(rpp[p]) + Vpre(p), p = 0 .. n; vtop[p] = prp[p+1], the end of
// p's V-part, which the scatter counts down from
// With no pivot edge at all (n_pivot = 0: a graph of short lists only) the
// masks, counts and scans are all zero and were skipped: prp is all zeros.
__global__ void k_pivot_offsets(int64_t n, const int64_t* __restrict__ rpp, const unsigned* __restrict__ umask,
                                const int64_t* __restrict__ upre, const int64_t* __restrict__ vpre,
                                int64_t* __restrict__ prp, unsigned long long* __restrict__ vtop,
                                const unsigned long long* __restrict__ n_pivot) {
    if (*n_pivot == 0ull) {
        for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= n; p += (int64_t)gridDim.x * blockDim.x)
            prp[p] = 0;
        return;
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = bits_before(umask, upre, rpp[p]) + vpre[p];
        prp[p] = o;
        if (p > 0) vtop[p - 1] = (unsigned long long)o;
    }
}

// vtop[p] counts down from the end of p's V-part while it is filled (one
// returned 64-bit atomic gives the slot).
#ifndef TC_PSCATTER_MIN_BLOCKS
#define TC_PSCATTER_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(kMpThreads, TC_PSCATTER_MIN_BLOCKS) k_pivot_scatter(int64_t n, int64_t ntiles, const longlong2* __restrict__ coord,
                                                              const int64_t* __restrict__ rpp, const int32_t* __restrict__ colp,
                                                              const unsigned* __restrict__ umask, const unsigned* __restrict__ vmask,
                                                              const int64_t* __restrict__ upre, const int64_t* __restrict__ vpre,
                                                              unsigned long long* __restrict__ vtop,
                                                              int32_t* __restrict__ pcol,
                                                              const unsigned long long* __restrict__ n_pivot) {
    if (*n_pivot == 0ull) return;  // no pivot edge: nothing to place
    __shared__ MpTile<false> S;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        mp_tile<false>(S, coord[t], coord[t + 1], n, rpp, nullptr, nullptr);
        const int64_t i0 = S.i0, j0 = S.j0;
        const int ne = S.ne;
        unsigned uw[kMpIpt], vw[kMpIpt];
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            uw[q] = vw[q] = 0;
            if (e < ne) {
                const int64_t g = j0 + e;
                uw[q] = umask[g >> 5];
                vw[q] = vmask[g >> 5];
            }
        }
        // every load and atomic of the tile first, then the stores: the V-part
        // slots come from returned atomics, whose latency the batch hides
        int32_t vv[kMpIpt];
        int cu[kMpIpt];      // U-part: set bits of the entry's mask word below it; -1 otherwise
        unsigned pvm = 0;    // V-part entries (bit q)
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int64_t g = j0 + q * kMpThreads + threadIdx.x;
            const unsigned bit = (unsigned)(g & 31);
            const bool pu = (uw[q] >> bit) & 1u, pv = (vw[q] >> bit) & 1u;  // 0 past the tile
            cu[q] = pu ? __popc(uw[q] & ((1u << bit) - 1u)) : -1;
            if (pv) pvm |= 1u << q;
            vv[q] = (pu || pv) ? ld_stream(colp + g) : 0;
        }
        int64_t dst[kMpIpt];
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            const int e = q * kMpThreads + threadIdx.x;
            const int64_t g = j0 + e;
            dst[q] = -1;
            if (cu[q] >= 0) dst[q] = upre[g >> 5] + cu[q] + vpre[i0 + S.row[e]];
            else if ((pvm >> q) & 1u) dst[q] = (int64_t)atomicAdd(&vtop[vv[q]], ~0ull) - 1;
        }
#pragma unroll
        for (int q = 0; q < kMpIpt; ++q) {
            if (dst[q] < 0) continue;
            const int e = q * kMpThreads + threadIdx.x;
            st_stream(pcol + dst[q], cu[q] >= 0 ? vv[q] : (int32_t)(i0 + S.row[e]));
        }
        __syncthreads();
    }
}

// pdesc[i] = (first vector of pcol[i]'s colr row, its d+) for every partner
// entry: what the count kernels read per partner, stored beside pcol so that
// they load it with pcol instead of gathering it through the partner's id.
__global__ void k_pdesc(const unsigned long long* __restrict__ n_pivot, const int32_t* __restrict__ pcol,
                        const int2* __restrict__ pd2, int2* __restrict__ pdesc) {
    const int64_t np = (int64_t)*n_pivot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        st_stream(pdesc + i, pd2[ld_stream(pcol + i)]);
}

// Work items per pivot, pivots taken in descending rank order.  Warp class
// (d+(p) <= warp_max): one item per chunk of partners.  CTA class: one item per
// (segment of the pivot list, chunk_c partners); a segment holds at most
// table_cap keys.
__global__ void __launch_bounds__(256) k_items(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ dp,
                                               const int32_t* __restrict__ deg, int small_max,
                                               const int64_t* __restrict__ prp,
                                               int warp_max, int table_cap, int chunk, int chunk_c,
                                               Item* __restrict__ iw, int64_t iw_cap,
                                               Item* __restrict__ ic, int64_t ic_cap,
                                               DevCounters* __restrict__ dc) {
    __shared__ long long sm[33];
    __shared__ unsigned long long s_bw, s_bc;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < n; t0 += (int64_t)gridDim.x * blockDim.x) {
        // A pivot's list is longer than small_max, so its degree is too.  The
        // degree does not increase along descending rank: once the block's
        // first vertex has degree <= small_max, no later one is a pivot.
        if (deg[perm[n - 1 - t0]] <= small_max) break;  // the same address for the whole block
        // pivots in descending rank order: pivots of similar rank share many
        // partners, so the partner lists that concurrent items stream stay in L2
        const int64_t r = t0 + threadIdx.x;
        const int64_t p = r < n ? perm[n - 1 - r] : n;
        int pcnt = 0, d = 0;
        if (p < n) { pcnt = (int)(prp[p + 1] - prp[p]); d = dp[p]; }
        const bool is_warp = d <= warp_max;
        const int ck = is_warp ? chunk : chunk_c;
        const int nch = (pcnt + ck - 1) / ck;
        const int nseg = is_warp ? 1 : (d + table_cap - 1) / table_cap;
        const long long cw = (pcnt > 0 && is_warp) ? nch : 0;
        const long long cc = (pcnt > 0 && !is_warp) ? (long long)nch * nseg : 0;
        long long tw, tcnt;
        const long long ow = block_excl_scan(cw, sm, &tw);
        const long long oc = block_excl_scan(cc, sm, &tcnt);
        if (threadIdx.x == 0) {
            s_bw = tw ? atomicAdd(&dc->n_items_warp, (unsigned long long)tw) : 0;
            s_bc = tcnt ? atomicAdd(&dc->n_items_cta, (unsigned long long)tcnt) : 0;
        }
        __syncthreads();
        const long long bw = (long long)s_bw + ow, bc = (long long)s_bc + oc;
        for (int c = 0; c < (int)cw; ++c) {
            if (bw + c < iw_cap) iw[bw + c] = Item{(int)p, 0, c * chunk, (int)min((int64_t)pcnt, (int64_t)(c + 1) * chunk)};
        }
        if (cc) {
            long long k = 0;
            for (int sg = 0; sg < nseg; ++sg)
                for (int c = 0; c < nch; ++c, ++k)
                    if (bc + k < ic_cap) ic[bc + k] = Item{(int)p, sg, c * chunk_c, (int)min((int64_t)pcnt, (int64_t)(c + 1) * chunk_c)};
        }
        __syncthreads();
    }
}

// ============================================================================
// host side
// ============================================================================
static unsigned grid_for(int64_t work, int threads, int num_sms, int per_sm = 8) {
    int64_t want = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

static int64_t isqrt_bound(int64_t x) {
    int64_t r = (int64_t)std::sqrt((double)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r + 1;
}

tc_status build_from_device_csr(tc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                const int64_t* vtx_off, int64_t G, bool validate, tc_ocsr** out, cudaStream_t s,
                                const int32_t* col_src) {
    if (col_src && (vtx_off || validate)) return set_err(ctx, TC_ERR_INVALID_ARG, "internal: col_src with a batch or validation");
    const Tuning tun = ctx->tun;
    const bool batch = vtx_off != nullptr;
    const int64_t m = nnz / 2;
    // partner descriptors hold colr vector indexes as int32
    if ((m + 3 * n + 4) / 4 > (int64_t)0x7fffffff)
        return set_err(ctx, TC_ERR_INVALID_ARG, "graph too large: m + 3n must stay below 2^33");
    tc_ocsr* o = new tc_ocsr();
    o->device = ctx->device;
    o->n = n;
    o->m = m;
    o->G = batch ? G : 0;
    o->tun = tun;
    const int64_t n1 = n + 1;
    // upper bounds for the item lists (no host read-back of device sizes)
    const int64_t dmax = std::min<int64_t>(std::max<int64_t>(n, 1), isqrt_bound(2 * m));
    const int64_t chunk = tun.chunk, cap = tun.table_cap;
    const int64_t chunk_c =
        std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(chunk * TC_CTA_CHUNK_MUL, 32767),
                                               ((int64_t(1) << 31) - 1) / (dmax + 15)));
    const int64_t chunk_min = std::min(chunk, chunk_c);  // partners of the shortest item of either list
    auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
    // warp items: sum over warp pivots of ceil(pc/chunk) <= #pivots + m/chunk
    o->items_warp_cap = std::min<int64_t>(n, m) + cdiv(m, chunk) + 1;
    // CTA items: sum of ceil(d/cap)*ceil(pc/chunk) <= sum (d/cap+1)(pc/chunk+1); d+ <= sqrt(2m)
    // (each of the d+(u) out-neighbours has degree >= d(u) >= d+(u)), sum pc <= m, sum d <= m,
    // and a CTA pivot has d > warp_max.
    o->items_cta_cap = cdiv(dmax * m, cap * chunk_min) + cdiv(m, cap) + cdiv(m, chunk_min) + cdiv(m, tun.warp_max + 1) + 4;

    int32_t* deg = nullptr;
    int32_t* pc = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = dev_alloc(p, std::max<size_t>(b, 16), s);
    };
    A((void**)&o->rpp, sizeof(int64_t) * n1);
    // +4: the count kernels read lists as aligned 16-byte vectors
    A((void**)&o->colp, sizeof(int32_t) * (std::max<int64_t>(m, 1) + 4));
    A((void**)&o->dplus, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&o->rank, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&o->perm, sizeof(int32_t) * std::max<int64_t>(n, 1));
    // padded rank-id rows (colr_row): at most m + 3n + 3 entries
    A((void**)&o->colr, sizeof(int32_t) * (std::max<int64_t>(m, 1) + 3 * n + 4));
    A((void**)&o->rspan, sizeof(int2) * std::max<int64_t>(n, 1));
    A((void**)&o->prp, sizeof(int64_t) * n1);
    A((void**)&o->pcol, sizeof(int32_t) * std::max<int64_t>(m, 1));
    A((void**)&o->pdesc, sizeof(int2) * std::max<int64_t>(m, 1));
    A((void**)&o->items_warp, sizeof(Item) * o->items_warp_cap);
    A((void**)&o->items_cta, sizeof(Item) * o->items_cta_cap);
    A((void**)&o->dc, sizeof(DevCounters));
    if (tun.merge_ratio > 0) {  // the merge class holds at most every oriented edge
        o->medge_cap = std::max<int64_t>(m, 1);
        A((void**)&o->medge, sizeof(int2) * o->medge_cap);
    }
    if (batch) A((void**)&o->row_graph, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&o->deg, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&pc, sizeof(int32_t) * std::max<int64_t>(n, 1));
    if (e != cudaSuccess) {
        tc_ocsr_free(o);
        dev_free(pc, s);
        return set_err(ctx, TC_ERR_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    deg = o->deg;
    o->bytes = (int64_t)(sizeof(int64_t) * n1 * 2 + sizeof(int32_t) * (5 * m + 9 * n) + sizeof(Item) * (o->items_warp_cap + o->items_cta_cap)
                         + (batch ? sizeof(int32_t) * n : 0) + sizeof(int2) * o->medge_cap);
    cudaMemsetAsync(o->dc, 0, sizeof(DevCounters), s);

    const int ns = ctx->num_sms;
    {
        PhaseScope ph(ctx, kPhDegree, s);
        if (batch && G > 0) {
            k_row_graph<<<(unsigned)std::min<int64_t>(G, 65535), 256, 0, s>>>(G, vtx_off, o->row_graph);
            TC_LAUNCH(ctx);
        }
        if (n > 0) {
            k_degree<<<grid_for(n, 256, ns), 256, 0, s>>>(n, row_ptr, deg, &o->dc->max_deg);
            TC_LAUNCH(ctx);
        }
    }
    if (validate && n > 0) {
        {
            PhaseScope ph(ctx, kPhValidate, s);
            k_validate<<<grid_for(n, 256, ns), 256, 0, s>>>(n, nnz, row_ptr, col, o->row_graph, vtx_off, &o->dc->error);
            TC_LAUNCH(ctx);
        }
        int herr = 0;
        cudaMemcpyAsync(&herr, &o->dc->error, sizeof(int), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || herr != 0) {
            dev_free(pc, s);
            tc_ocsr_free(o);
            if (e != cudaSuccess) return cuda_err(ctx, e, "validate");
            return set_err(ctx, TC_ERR_INVALID_GRAPH, "input is not a simple symmetric sorted CSR (code " + std::to_string(herr) + ")");
        }
    }
    // rank order (degree, id): one stable radix sort of n keys
    if (n > 0) {
        PhaseScope ph(ctx, kPhRank, s);
        int b = 1;
        while (((int64_t)1 << b) < n) ++b;
        unsigned long long *ka = nullptr, *kb = nullptr, *sorted = nullptr;
        e = dev_alloc((void**)&ka, sizeof(unsigned long long) * n, s);
        if (e == cudaSuccess) e = dev_alloc((void**)&kb, sizeof(unsigned long long) * n, s);
        if (e == cudaSuccess) {
            k_rank_keys<<<grid_for(n, 256, ns), 256, 0, s>>>(n, deg, b, ka);
            // the keys are written in id order and the sort is stable, so
            // sorting the degree bits alone yields (degree, id) order
            radix_sort_u64(ka, kb, n, 2 * b, s, &sorted, &ctx->launches, b, &o->dc->max_deg, b);
            k_rank_from_sorted<<<grid_for(n, 256, ns), 256, 0, s>>>(n, ka, kb, &o->dc->max_deg, b, o->rank, o->perm);
            ctx->launches += 2;
        }
        dev_free(ka, s);
        dev_free(kb, s);
        if (e != cudaSuccess) {
            dev_free(pc, s);
            tc_ocsr_free(o);
            return set_err(ctx, TC_ERR_OOM, "rank: device allocation failed");
        }
    }
    // merge-path tiles: nt1 over the input CSR, nt2 over the oriented CSR
    const int64_t nt1 = mp_tiles(n, nnz), nt2 = mp_tiles(n, m);
    const int64_t kw = (nnz >> 5) + 1, uw = (m >> 5) + 1;  // bitmask words (one spare: prefix at the end)
    longlong2* coord = nullptr;
    unsigned *keep = nullptr, *umask = nullptr, *vmask = nullptr;
    int32_t* wpc = nullptr;
    int64_t *kpre = nullptr, *upre = nullptr, *vpre = nullptr;
    int2* rd2 = nullptr;
    int2* pd2 = nullptr;
    unsigned long long* vtop = nullptr;
    int32_t* srows = nullptr;     // rows for k_sort_rows, listed by k_rows
    unsigned* n_srows = nullptr;
    void* wtmp = nullptr;
    const size_t wtb = scan_tmp_bytes(std::max(kw, std::max(uw, n)));
    auto B = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = dev_alloc(p, std::max<size_t>(b, 16), s);
    };
    B((void**)&coord, sizeof(longlong2) * (std::max(nt1, nt2) + 1));
    B((void**)&keep, sizeof(unsigned) * kw);
    B((void**)&umask, sizeof(unsigned) * uw);
    B((void**)&vmask, sizeof(unsigned) * uw);
    B((void**)&wpc, sizeof(int32_t) * std::max(kw, uw));
    B((void**)&kpre, sizeof(int64_t) * (kw + 1));
    B((void**)&upre, sizeof(int64_t) * (uw + 1));
    B((void**)&vpre, sizeof(int64_t) * n1);
    B((void**)&rd2, sizeof(int2) * std::max<int64_t>(n, 1));
    B((void**)&pd2, sizeof(int2) * std::max<int64_t>(n, 1));
    B((void**)&vtop, sizeof(unsigned long long) * std::max<int64_t>(n, 1));
    B((void**)&srows, sizeof(int32_t) * std::max<int64_t>(n, 1));
    B((void**)&n_srows, sizeof(unsigned));
    B(&wtmp, wtb);
    auto free_tmp = [&]() {
        dev_free(coord, s); dev_free(keep, s); dev_free(umask, s); dev_free(vmask, s); dev_free(wpc, s);
        dev_free(kpre, s); dev_free(upre, s); dev_free(vpre, s); dev_free(wtmp, s);
        dev_free(rd2, s); dev_free(pd2, s); dev_free(vtop, s); dev_free(srows, s); dev_free(n_srows, s);
        dev_free(pc, s);
    };
    if (e != cudaSuccess) {
        free_tmp();
        tc_ocsr_free(o);
        return set_err(ctx, TC_ERR_OOM, "orient: device allocation failed");
    }
    const int per_sm = 8;
    const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt1, (int64_t)ns * per_sm));
    const unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt2, (int64_t)ns * per_sm));
    // a-2: one bit per kept entry
    {
        PhaseScope ph(ctx, kPhOrientCount, s);
        cudaMemsetAsync(keep, 0, sizeof(unsigned) * kw, s);
        k_mp_coords<<<grid_for(nt1 + 1, 256, ns), 256, 0, s>>>(n, nnz, row_ptr, nt1, coord);
        if (nt1 > 0) {
            if (batch) k_orient_flags<true><<<g1, kMpThreads, 0, s>>>(n, nt1, coord, row_ptr, col, deg, o->row_graph, vtx_off, keep,
                                                                       nullptr);
            else if (col_src)  // reads the pinned host entries and leaves their device copy in col
                k_orient_flags<false><<<g1, kMpThreads, 0, s>>>(n, nt1, coord, row_ptr, col_src, deg, nullptr, nullptr, keep,
                                                                const_cast<int32_t*>(col));
            else k_orient_flags<false><<<g1, kMpThreads, 0, s>>>(n, nt1, coord, row_ptr, col, deg, nullptr, nullptr, keep, nullptr);
        }
        ctx->launches += 2;
    }
    // a-3: prefix counts over the bitmask give every kept entry its place
    {
        PhaseScope ph(ctx, kPhOrientScan, s);
        k_popc<<<grid_for(kw, 256, ns), 256, 0, s>>>(keep, kw, wpc);
        scan_i32_to_i64(wpc, kpre, kw, wtmp, wtb, s);
        // row offsets and d+
        cudaMemsetAsync(n_srows, 0, sizeof(unsigned), s);
        k_rows<<<grid_for(n + 1, 256, ns), 256, 0, s>>>(n, row_ptr, keep, kpre, o->rank, o->rpp, o->dplus, rd2, pd2,
                                                        &o->dc->max_dplus, tun.warp_max, srows, n_srows);
        ctx->launches += 5;
    }
    {
        PhaseScope ph(ctx, kPhOrientScatter, s);
        // padding (and the gaps between rows) of colr read as -1
        cudaMemsetAsync(o->colr, 0xff, sizeof(int32_t) * (std::max<int64_t>(m, 1) + 3 * n + 4), s);
        // the scatter also classifies each oriented edge for the partition (a-4)
        cudaMemsetAsync(pc, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), s);
        cudaMemsetAsync(umask, 0, sizeof(unsigned) * uw, s);
        cudaMemsetAsync(vmask, 0, sizeof(unsigned) * uw, s);
        if (nt1 > 0) {
            if (batch)
                k_orient_scatter<true><<<g1, kMpThreads, 0, s>>>(n, nt1, coord, row_ptr, col, rd2, o->row_graph, vtx_off, keep, kpre,
                                                                 o->rpp, tun.small_max, tun.merge_ratio, tun.merge_max,
                                                                 o->medge, o->medge_cap, o->colp, o->colr,
                                                                 umask, vmask, pc, o->dc);
            else
                k_orient_scatter<false><<<g1, kMpThreads, 0, s>>>(n, nt1, coord, row_ptr, col, rd2, nullptr, nullptr, keep, kpre,
                                                                  o->rpp, tun.small_max, tun.merge_ratio, tun.merge_max,
                                                                  o->medge, o->medge_cap, o->colp, o->colr,
                                                                  umask, vmask, pc, o->dc);
            TC_LAUNCH(ctx);
        }
    }
    // rank spans of the rows CTA tables are built from; level partition of the
    // rows whose lists the CTA kernel streams
    if (n > 0) {
        PhaseScope ph(ctx, kPhRowSort, s);
        const size_t sm = sizeof(int) * (kSortedMax + kRankLevels) * kSortWarps;
        cudaFuncSetAttribute(k_sort_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        // one listed row per warp, as many warps as fit
        const unsigned sg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kSortWarps - 1) / kSortWarps, (int64_t)ns * 8));
        k_sort_rows<<<sg, 32 * kSortWarps, sm, s>>>(n, o->rpp, o->dplus, srows, n_srows, o->colr, o->rspan);
        TC_LAUNCH(ctx);
    }
    // a-4: classify, group oriented edges by pivot
    {
        PhaseScope ph(ctx, kPhPivotCount, s);
        k_mp_coords<<<grid_for(nt2 + 1, 256, ns), 256, 0, s>>>(n, m, o->rpp, nt2, coord);
        TC_LAUNCH(ctx);
    }
    {
        PhaseScope ph(ctx, kPhPivotScan, s);
        // with no pivot edge (n_pivot_edges = 0) the masks and counts are all
        // zero: the scans return at once and prp is written as zeros
        const unsigned long long* np = &o->dc->n_pivot_edges;
        k_popc<<<grid_for(uw, 256, ns), 256, 0, s>>>(umask, uw, wpc);
        scan_i32_to_i64_unless_zero(wpc, upre, uw, wtmp, wtb, s, np);
        scan_i32_to_i64_unless_zero(pc, vpre, n, wtmp, wtb, s, np);
        k_pivot_offsets<<<grid_for(n + 1, 256, ns), 256, 0, s>>>(n, o->rpp, umask, upre, vpre, o->prp, vtop, np);
        ctx->launches += 8;
    }
    {
        PhaseScope ph(ctx, kPhPivotScatter, s);
        if (nt2 > 0) {
            k_pivot_scatter<<<g2, kMpThreads, 0, s>>>(n, nt2, coord, o->rpp, o->colp, umask, vmask, upre, vpre, vtop, o->pcol,
                                                      &o->dc->n_pivot_edges);
            TC_LAUNCH(ctx);
            // the partners' descriptors beside pcol, in one coalesced pass
            k_pdesc<<<grid_for(m, 256, ns), 256, 0, s>>>(&o->dc->n_pivot_edges, o->pcol, pd2, o->pdesc);
            TC_LAUNCH(ctx);
        }
    }
    dev_free(coord, s); dev_free(keep, s); dev_free(umask, s); dev_free(vmask, s); dev_free(wpc, s);
    dev_free(kpre, s); dev_free(upre, s); dev_free(vpre, s); dev_free(wtmp, s);
    dev_free(rd2, s); dev_free(pd2, s); dev_free(vtop, s); dev_free(srows, s); dev_free(n_srows, s);
    if (n > 0) {
        PhaseScope ph(ctx, kPhItems, s);
        k_items<<<grid_for(n, 256, ns), 256, 0, s>>>(n, o->perm, o->dplus, o->deg, tun.small_max, o->prp, tun.warp_max,
                                                     tun.table_cap, tun.chunk,
                                                     (int)chunk_c,
                                                     o->items_warp, o->items_warp_cap, o->items_cta, o->items_cta_cap, o->dc);
        TC_LAUNCH(ctx);
    }
    dev_free(pc, s);
   
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        tc_ocsr_free(o);
        return cuda_err(ctx, e, "build kernels");
    }
    *out = o;
    return TC_OK;
}

}  // namespace tc
