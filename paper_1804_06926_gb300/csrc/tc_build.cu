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
constexpr int kBigRow = 4096;     // rows longer than this are oriented chunk by chunk
constexpr int kBigChunk = 8192;   // entries per chunk of a long row
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

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                              long long* __restrict__ tile_sum) {
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
                                                    int64_t* __restrict__ out, int64_t n) {
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
                                                             int64_t* __restrict__ out) {
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

cudaError_t scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                            cudaStream_t s) {
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (tmp_bytes < scan_tmp_bytes(n)) return cudaErrorInvalidValue;
    long long* ts = (long long*)tmp;
    if (nt > 0) k_scan_reduce<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ts);
    k_scan_sums<<<1, 1024, 0, s>>>(ts, nt, out, n);
    if (nt > 0) k_scan_apply<<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, ts, out);
    return cudaGetLastError();
}

// ============================================================================
// a-1  degree: d(v) = row_ptr[v+1] - row_ptr[v]
// ============================================================================
__global__ void k_degree(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ deg) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        deg[v] = (int32_t)(rp[v + 1] - rp[v]);
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

__global__ void k_rank_from_sorted(int64_t n, const unsigned long long* __restrict__ sorted, int b,
                                   int32_t* __restrict__ rank, int32_t* __restrict__ perm) {
    const unsigned long long mask = (1ull << b) - 1ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(sorted[r] & mask);
        perm[r] = v;
        rank[v] = (int32_t)r;
    }
}

// colr[e] = rank[colp[e]]: the oriented lists renamed to rank ids
__global__ void k_relabel(int64_t m, const int32_t* __restrict__ colp, const int32_t* __restrict__ rank,
                          int32_t* __restrict__ colr) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        colr[e] = rank[colp[e]];
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
// a-2 / a-3  orientation filter and compaction.
// A group of GS lanes walks one row; neighbour v is kept iff
// rank(u) < rank(v), rank = (d, id).  The count pass writes d+(u); the
// scatter pass writes the kept neighbours at rpp[u] in their input order, so
// rows stay ascending.
// ============================================================================
template <int GS>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (GS == 32) {
        return 0xffffffffu;
    } else {
        const int g = (threadIdx.x & 31) / GS;
        return ((1u << GS) - 1u) << (g * GS);
    }
}

template <int GS, bool SCATTER, bool BATCH>
__global__ void __launch_bounds__(256) k_orient(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                const int32_t* __restrict__ deg, const int32_t* __restrict__ row_graph,
                                                const int64_t* __restrict__ vtx_off, int32_t* __restrict__ cnt,
                                                const int64_t* __restrict__ rpp, int32_t* __restrict__ colp,
                                                const int32_t* __restrict__ rank, int32_t* __restrict__ colr,
                                                int2* __restrict__ rspan) {
    const int lane = threadIdx.x & 31;
    const int sub = lane % GS;
    const int shift = (lane / GS) * GS;
    const unsigned gm = group_mask<GS>();
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / GS;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS; u < n; u += ngroups) {
        const int64_t b = rp[u], e = rp[u + 1];
        const int du = (int)(e - b);
        if (du > kBigRow) {  // long rows are cut into chunks for k_orient_big
            if (!SCATTER && sub == 0) {
                cnt[u] = 0;
                rspan[u] = make_int2(0x7fffffff, -1);
            }
            continue;
        }
        const int64_t base = BATCH ? vtx_off[row_graph[u]] : 0;
        int kept = 0;
        int64_t out = 0;
        int rmin = 0x7fffffff, rmax = -1;
        if (SCATTER) out = rpp[u];
        for (int64_t j0 = b; j0 < e; j0 += GS) {
            const int64_t i = j0 + sub;
            const bool valid = i < e;
            const int64_t v = valid ? (int64_t)col[i] + base : 0;
            const int dv = valid ? deg[v] : 0;
            const bool keep = valid && (du < dv || (du == dv && u < v));
            const unsigned bal = __ballot_sync(gm, keep);
            const unsigned mine = (GS == 32) ? bal : ((bal >> shift) & ((1u << (GS & 31)) - 1u));
            if (SCATTER && keep) {
                const int64_t pos = out + kept + __popc(mine & ((1u << sub) - 1u));
                const int r = rank[v];
                colp[pos] = (int32_t)v;
                colr[pos] = r;
                rmin = min(rmin, r);
                rmax = max(rmax, r);
            }
            kept += __popc(mine);
        }
        if (!SCATTER && sub == 0) cnt[u] = kept;
        if (SCATTER) {  // span of the row in rank ids
#pragma unroll
            for (int o = GS / 2; o; o >>= 1) {
                rmin = min(rmin, __shfl_xor_sync(gm, rmin, o));
                rmax = max(rmax, __shfl_xor_sync(gm, rmax, o));
            }
            if (sub == 0) rspan[u] = make_int2(rmin, rmax);
        }
    }
}

// Rows longer than kBigRow are cut into chunks of kBigChunk entries, each
// handled by one CTA, so that hub rows do not serialise on one warp.  The
// count pass sums each chunk's kept entries; the scatter pass places a
// chunk's kept entries after those of the row's earlier chunks.
struct BigChunk {
    int u, j, first, pad;
};

__global__ void k_big_chunks(int64_t n, const int64_t* __restrict__ rp, BigChunk* __restrict__ chunks,
                             int64_t cap, unsigned long long* __restrict__ n_chunks) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[u + 1] - rp[u];
        if (d <= kBigRow) continue;
        const int nch = (int)((d + kBigChunk - 1) / kBigChunk);
        const unsigned long long first = atomicAdd(n_chunks, (unsigned long long)nch);
        for (int j = 0; j < nch; ++j)
            if ((int64_t)(first + j) < cap) chunks[first + j] = BigChunk{(int)u, j, (int)first, 0};
    }
}

template <bool SCATTER, bool BATCH>
__global__ void __launch_bounds__(256) k_orient_big(const BigChunk* __restrict__ chunks,
                                                    const unsigned long long* __restrict__ n_chunks, int64_t cap,
                                                    const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                    const int32_t* __restrict__ deg, const int32_t* __restrict__ row_graph,
                                                    const int64_t* __restrict__ vtx_off, int32_t* __restrict__ cnt,
                                                    int32_t* __restrict__ chunk_cnt, const int64_t* __restrict__ rpp,
                                                    int32_t* __restrict__ colp, const int32_t* __restrict__ rank,
                                                    int32_t* __restrict__ colr, int2* __restrict__ rspan) {
    __shared__ int s_w[8];
    __shared__ long long s_off;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t nc = (int64_t)min(*n_chunks, (unsigned long long)cap);
    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const BigChunk ch = chunks[c];
        const int64_t u = ch.u;
        const int64_t rb = rp[u], re = rp[u + 1];
        const int du = (int)(re - rb);
        const int64_t b = rb + (int64_t)ch.j * kBigChunk, e = min(re, b + kBigChunk);
        const int64_t base = BATCH ? vtx_off[row_graph[u]] : 0;
        if (SCATTER && threadIdx.x == 0) {
            long long off = rpp[u];
            for (int64_t k = ch.first; k < c; ++k) off += chunk_cnt[k];
            s_off = off;
        }
        int run = 0;
        int rmin = 0x7fffffff, rmax = -1;
        for (int64_t r0 = b; r0 < e; r0 += blockDim.x) {
            const int64_t i = r0 + threadIdx.x;
            const bool valid = i < e;
            const int64_t v = valid ? (int64_t)col[i] + base : 0;
            const int dv = valid ? deg[v] : 0;
            const bool keep = valid && (du < dv || (du == dv && u < v));
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_w[w] = __popc(bal);
            __syncthreads();
            int before = 0, tot = 0;
            for (int k = 0; k < nw; ++k) {
                const int c2 = s_w[k];
                if (k < w) before += c2;
                tot += c2;
            }
            if (SCATTER && keep) {
                const int64_t pos = s_off + run + before + __popc(bal & ((1u << lane) - 1u));
                const int r = rank[v];
                colp[pos] = (int32_t)v;
                colr[pos] = r;
                rmin = min(rmin, r);
                rmax = max(rmax, r);
            }
            run += tot;
            __syncthreads();
        }
        if (SCATTER) {
            for (int o = 16; o; o >>= 1) {
                rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
                rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            }
            if (lane == 0 && rmax >= 0) {
                atomicMin(&rspan[u].x, rmin);
                atomicMax(&rspan[u].y, rmax);
            }
        }
        if (!SCATTER && threadIdx.x == 0) {
            chunk_cnt[c] = run;
            if (run) atomicAdd(&cnt[u], run);
        }
        __syncthreads();
    }
}

// ============================================================================
// a-4  partition (Alg. 2 Partition; Sec. 4.2.2 dynamic grouping).
// Every oriented edge (u, v) with a = d+(u), b = d+(v) falls in one class:
//   skip  : a <= 1 or b == 0 (N+(u) = {v} or N+(v) empty: no common vertex);
//   small : max(a, b) <= small_max -> one thread merges the two lists;
//   pivot : otherwise.  The endpoint with the longer list is the pivot p (u
//           on ties), the other is the partner q.  The pivot's list becomes a
//           shared-memory table and the partner's (shorter) list is streamed
//           against it: the "small x large" kernel the paper proposes in its
//           Sec. 5 discussion, applied to every non-small edge.
// ============================================================================
enum { kSkip = 0, kSmall = 1, kPivot = 2 };

__device__ __forceinline__ int edge_class(int a, int b, int small_max) {
    if (a <= 1 || b == 0) return kSkip;
    if (max(a, b) <= small_max) return kSmall;
    return kPivot;
}

template <int GS, bool SCATTER>
__global__ void __launch_bounds__(256) k_pivot(int64_t n, const int64_t* __restrict__ rpp, const int32_t* __restrict__ colp,
                                               const int32_t* __restrict__ dp, int small_max,
                                               int32_t* __restrict__ pc, const int64_t* __restrict__ prp,
                                               int32_t* __restrict__ pcol, DevCounters* __restrict__ dc) {
    __shared__ unsigned long long s_piv, s_small;
    if (!SCATTER && threadIdx.x == 0) { s_piv = 0; s_small = 0; }
    if (!SCATTER) __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane % GS;
    const int shift = (lane / GS) * GS;
    const unsigned gm = group_mask<GS>();
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / GS;
    unsigned long long my_piv = 0, my_small = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS; u < n; u += ngroups) {
        const int a = dp[u];
        if (a <= 1) continue;  // uniform within the group
        const int64_t b0 = rpp[u], e = rpp[u + 1];
        for (int64_t j0 = b0; j0 < e; j0 += GS) {
            const int64_t i = j0 + sub;
            const bool valid = i < e;
            const int v = valid ? colp[i] : 0;
            const int b = valid ? dp[v] : 0;
            const int cls = valid ? edge_class(a, b, small_max) : kSkip;
            const bool piv_u = cls == kPivot && a >= b;
            const bool piv_v = cls == kPivot && a < b;
            const unsigned bu = __ballot_sync(gm, piv_u);
            const unsigned mine = (GS == 32) ? bu : ((bu >> shift) & ((1u << (GS & 31)) - 1u));
            const int nu = __popc(mine);
            const int leader = __ffs(mine) - 1;  // lane within group
            if (!SCATTER) {
                if (piv_u && sub == leader) atomicAdd(&pc[u], nu);
                if (piv_v) atomicAdd(&pc[v], 1);
                my_piv += piv_u + piv_v;
                my_small += cls == kSmall;
            } else {
                int basepos = 0;
                if (piv_u && sub == leader) basepos = atomicAdd(&pc[u], nu);
                basepos = __shfl_sync(gm, basepos, shift + (leader < 0 ? 0 : leader));
                if (piv_u) pcol[prp[u] + basepos + __popc(mine & ((1u << sub) - 1u))] = v;
                if (piv_v) pcol[prp[v] + atomicAdd(&pc[v], 1)] = (int32_t)u;
            }
        }
    }
    if (!SCATTER) {
        // block-aggregate the class counters
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
}

// Work items per pivot.  Warp class (d+(p) <= warp_max): one item per chunk of
// partners.  CTA class: one item per (segment of the pivot list, chunk of
// partners); a segment holds at most table_cap keys.
__global__ void __launch_bounds__(256) k_items(int64_t n, const int32_t* __restrict__ dp, const int64_t* __restrict__ prp,
                                               int warp_max, int table_cap, int chunk,
                                               Item* __restrict__ iw, int64_t iw_cap,
                                               Item* __restrict__ ic, int64_t ic_cap,
                                               DevCounters* __restrict__ dc) {
    __shared__ long long sm[33];
    __shared__ unsigned long long s_bw, s_bc;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < n; t0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t0 + threadIdx.x;
        int pcnt = 0, d = 0;
        if (p < n) { pcnt = (int)(prp[p + 1] - prp[p]); d = dp[p]; }
        const int nch = (pcnt + chunk - 1) / chunk;
        const bool is_warp = d <= warp_max;
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
            if (bw + c < iw_cap) iw[bw + c] = Item{(int)p, 0, c * chunk, min(pcnt, (c + 1) * chunk)};
        }
        if (cc) {
            long long k = 0;
            for (int sg = 0; sg < nseg; ++sg)
                for (int c = 0; c < nch; ++c, ++k)
                    if (bc + k < ic_cap) ic[bc + k] = Item{(int)p, sg, c * chunk, min(pcnt, (c + 1) * chunk)};
        }
        __syncthreads();
    }
}

// ============================================================================
// host side
// ============================================================================
static int pick_group(int64_t n, int64_t entries, const char* env_name) {
    if (const char* v = std::getenv(env_name)) {  // tuning override: 4, 8, 16 or 32 lanes per row
        const int g = std::atoi(v);
        if (g == 4 || g == 8 || g == 16 || g == 32) return g;
    }
    double avg = n > 0 ? (double)entries / (double)n : 0.0;
    if (avg <= 4.0) return 4;
    if (avg <= 8.0) return 8;
    if (avg <= 16.0) return 16;
    return 32;
}

static unsigned grid_for(int64_t work, int threads, int num_sms, int per_sm = 8) {
    int64_t want = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

template <bool SCATTER, bool BATCH>
static void launch_orient(int gs, unsigned grid, cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* col,
                          const int32_t* deg, const int32_t* rg, const int64_t* vo, int32_t* cnt, const int64_t* rpp,
                          int32_t* colp, const int32_t* rank, int32_t* colr, int2* rspan) {
    switch (gs) {
        case 4: k_orient<4, SCATTER, BATCH><<<grid, 256, 0, s>>>(n, rp, col, deg, rg, vo, cnt, rpp, colp, rank, colr, rspan); break;
        case 8: k_orient<8, SCATTER, BATCH><<<grid, 256, 0, s>>>(n, rp, col, deg, rg, vo, cnt, rpp, colp, rank, colr, rspan); break;
        case 16: k_orient<16, SCATTER, BATCH><<<grid, 256, 0, s>>>(n, rp, col, deg, rg, vo, cnt, rpp, colp, rank, colr, rspan); break;
        default: k_orient<32, SCATTER, BATCH><<<grid, 256, 0, s>>>(n, rp, col, deg, rg, vo, cnt, rpp, colp, rank, colr, rspan); break;
    }
}

template <bool SCATTER>
static void launch_pivot(int gs, unsigned grid, cudaStream_t s, int64_t n, const int64_t* rpp, const int32_t* colp,
                         const int32_t* dp, int small_max, int32_t* pc, const int64_t* prp, int32_t* pcol,
                         DevCounters* dc) {
    switch (gs) {
        case 4: k_pivot<4, SCATTER><<<grid, 256, 0, s>>>(n, rpp, colp, dp, small_max, pc, prp, pcol, dc); break;
        case 8: k_pivot<8, SCATTER><<<grid, 256, 0, s>>>(n, rpp, colp, dp, small_max, pc, prp, pcol, dc); break;
        case 16: k_pivot<16, SCATTER><<<grid, 256, 0, s>>>(n, rpp, colp, dp, small_max, pc, prp, pcol, dc); break;
        default: k_pivot<32, SCATTER><<<grid, 256, 0, s>>>(n, rpp, colp, dp, small_max, pc, prp, pcol, dc); break;
    }
}

static int64_t isqrt_bound(int64_t x) {
    int64_t r = (int64_t)std::sqrt((double)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r + 1;
}

tc_status build_from_device_csr(tc_ctx* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                const int64_t* vtx_off, int64_t G, bool validate, tc_ocsr** out, cudaStream_t s) {
    const Tuning tun = ctx->tun;
    const bool batch = vtx_off != nullptr;
    const int64_t m = nnz / 2;
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
    auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
    // warp items: sum over warp pivots of ceil(pc/chunk) <= #pivots + m/chunk
    o->items_warp_cap = std::min<int64_t>(n, m) + cdiv(m, chunk) + 1;
    // CTA items: sum of ceil(d/cap)*ceil(pc/chunk) <= sum (d/cap+1)(pc/chunk+1); d+ <= sqrt(2m)
    // (each of the d+(u) out-neighbours has degree >= d(u) >= d+(u)), sum pc <= m, sum d <= m,
    // and a CTA pivot has d > warp_max.
    o->items_cta_cap = cdiv(dmax * m, cap * chunk) + cdiv(m, cap) + cdiv(m, chunk) + cdiv(m, tun.warp_max + 1) + 4;

    int32_t* deg = nullptr;
    int32_t* pc = nullptr;
    void* scan_tmp = nullptr;
    const size_t stb = scan_tmp_bytes(n);
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
    A((void**)&o->colr, sizeof(int32_t) * (std::max<int64_t>(m, 1) + 4));
    A((void**)&o->rspan, sizeof(int2) * std::max<int64_t>(n, 1));
    A((void**)&o->prp, sizeof(int64_t) * n1);
    A((void**)&o->pcol, sizeof(int32_t) * std::max<int64_t>(m, 1));
    A((void**)&o->items_warp, sizeof(Item) * o->items_warp_cap);
    A((void**)&o->items_cta, sizeof(Item) * o->items_cta_cap);
    A((void**)&o->dc, sizeof(DevCounters));
    if (batch) A((void**)&o->row_graph, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&o->deg, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&pc, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A(&scan_tmp, stb);
    if (e != cudaSuccess) {
        tc_ocsr_free(o);
        dev_free(pc, s); dev_free(scan_tmp, s);
        return set_err(ctx, TC_ERR_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    deg = o->deg;
    o->bytes = (int64_t)(sizeof(int64_t) * n1 * 2 + sizeof(int32_t) * (3 * m + 6 * n) + sizeof(Item) * (o->items_warp_cap + o->items_cta_cap)
                         + (batch ? sizeof(int32_t) * n : 0));
    cudaMemsetAsync(o->dc, 0, sizeof(DevCounters), s);

    const int ns = ctx->num_sms;
    {
        PhaseScope ph(ctx, kPhDegree, s);
        if (batch && G > 0) {
            k_row_graph<<<(unsigned)std::min<int64_t>(G, 65535), 256, 0, s>>>(G, vtx_off, o->row_graph);
            TC_LAUNCH(ctx);
        }
        if (n > 0) {
            k_degree<<<grid_for(n, 256, ns), 256, 0, s>>>(n, row_ptr, deg);
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
            dev_free(pc, s); dev_free(scan_tmp, s);
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
            radix_sort_u64(ka, kb, n, 2 * b, s, &sorted, &ctx->launches, b);
            k_rank_from_sorted<<<grid_for(n, 256, ns), 256, 0, s>>>(n, sorted, b, o->rank, o->perm);
            ctx->launches += 2;
        }
        dev_free(ka, s);
        dev_free(kb, s);
        if (e != cudaSuccess) {
            dev_free(pc, s); dev_free(scan_tmp, s);
            tc_ocsr_free(o);
            return set_err(ctx, TC_ERR_OOM, "rank: device allocation failed");
        }
    }
    const int gs = pick_group(n, nnz, "TC_ORIENT_GROUP");
    const unsigned og = grid_for(n * gs, 256, ns, 16);
    // long rows: chunk list (bounded by nnz/kBigChunk + nnz/kBigRow)
    const int64_t bc_cap = nnz / kBigChunk + nnz / kBigRow + 2;
    BigChunk* bchunks = nullptr;
    int32_t* bcnt = nullptr;
    unsigned long long* nbc = nullptr;
    e = dev_alloc((void**)&bchunks, sizeof(BigChunk) * bc_cap, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&bcnt, sizeof(int32_t) * bc_cap, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&nbc, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        dev_free(bchunks, s); dev_free(bcnt, s); dev_free(nbc, s);
        dev_free(pc, s); dev_free(scan_tmp, s);
        tc_ocsr_free(o);
        return set_err(ctx, TC_ERR_OOM, "orient: device allocation failed");
    }
    const unsigned bg = (unsigned)std::max(1, ns * 4);
    // a-2: kept count per row = d+(u)
    {
        PhaseScope ph(ctx, kPhOrientCount, s);
        cudaMemsetAsync(nbc, 0, sizeof(unsigned long long), s);
        if (n > 0) k_big_chunks<<<grid_for(n, 256, ns), 256, 0, s>>>(n, row_ptr, bchunks, bc_cap, nbc);
        if (batch) launch_orient<false, true>(gs, og, s, n, row_ptr, col, deg, o->row_graph, vtx_off, o->dplus, nullptr, nullptr, nullptr, nullptr, o->rspan);
        else launch_orient<false, false>(gs, og, s, n, row_ptr, col, deg, nullptr, nullptr, o->dplus, nullptr, nullptr, nullptr, nullptr, o->rspan);
        if (batch) k_orient_big<false, true><<<bg, 256, 0, s>>>(bchunks, nbc, bc_cap, row_ptr, col, deg, o->row_graph, vtx_off, o->dplus, bcnt, nullptr, nullptr, nullptr, nullptr, nullptr);
        else k_orient_big<false, false><<<bg, 256, 0, s>>>(bchunks, nbc, bc_cap, row_ptr, col, deg, nullptr, nullptr, o->dplus, bcnt, nullptr, nullptr, nullptr, nullptr, nullptr);
        ctx->launches += 3;
    }
    // a-3: row offsets of the oriented CSR, then the stable scatter
    {
        PhaseScope ph(ctx, kPhOrientScan, s);
        scan_i32_to_i64(o->dplus, o->rpp, n, scan_tmp, stb, s);
        ctx->launches += 3;
    }
    {
        PhaseScope ph(ctx, kPhOrientScatter, s);
        if (batch) launch_orient<true, true>(gs, og, s, n, row_ptr, col, deg, o->row_graph, vtx_off, nullptr, o->rpp, o->colp, o->rank, o->colr, o->rspan);
        else launch_orient<true, false>(gs, og, s, n, row_ptr, col, deg, nullptr, nullptr, nullptr, o->rpp, o->colp, o->rank, o->colr, o->rspan);
        if (batch) k_orient_big<true, true><<<bg, 256, 0, s>>>(bchunks, nbc, bc_cap, row_ptr, col, deg, o->row_graph, vtx_off, nullptr, bcnt, o->rpp, o->colp, o->rank, o->colr, o->rspan);
        else k_orient_big<true, false><<<bg, 256, 0, s>>>(bchunks, nbc, bc_cap, row_ptr, col, deg, nullptr, nullptr, nullptr, bcnt, o->rpp, o->colp, o->rank, o->colr, o->rspan);
        ctx->launches += 2;
    }
    dev_free(bchunks, s);
    dev_free(bcnt, s);
    dev_free(nbc, s);
    // a-4: classify, group oriented edges by pivot, cut work items
    const int gs2 = pick_group(n, m, "TC_PIVOT_GROUP");
    const unsigned pg = grid_for(n * gs2, 256, ns, 16);
    {
        PhaseScope ph(ctx, kPhPivotCount, s);
        cudaMemsetAsync(pc, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), s);
        launch_pivot<false>(gs2, pg, s, n, o->rpp, o->colp, o->dplus, tun.small_max, pc, nullptr, nullptr, o->dc);
        TC_LAUNCH(ctx);
    }
    {
        PhaseScope ph(ctx, kPhPivotScan, s);
        scan_i32_to_i64(pc, o->prp, n, scan_tmp, stb, s);
        ctx->launches += 3;
    }
    {
        PhaseScope ph(ctx, kPhPivotScatter, s);
        cudaMemsetAsync(pc, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), s);
        launch_pivot<true>(gs2, pg, s, n, o->rpp, o->colp, o->dplus, tun.small_max, pc, o->prp, o->pcol, o->dc);
        TC_LAUNCH(ctx);
    }
    if (n > 0) {
        PhaseScope ph(ctx, kPhItems, s);
        k_items<<<grid_for(n, 256, ns), 256, 0, s>>>(n, o->dplus, o->prp, tun.warp_max, tun.table_cap, tun.chunk,
                                                     o->items_warp, o->items_warp_cap, o->items_cta, o->items_cta_cap, o->dc);
        TC_LAUNCH(ctx);
    }
    dev_free(pc, s);
    dev_free(scan_tmp, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        tc_ocsr_free(o);
        return cuda_err(ctx, e, "build kernels");
    }
    *out = o;
    return TC_OK;
}

}  // namespace tc
