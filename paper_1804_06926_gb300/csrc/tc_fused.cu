// tc_fused.cu -- the whole method for one small graph in one kernel launch.
//
// A graph whose row offsets, oriented CSR and per-vertex counts fit in one
// CTA's shared memory is counted by one kernel launch: degrees and the (degree, id)
// order (Sec. 4.2.1), the orientation filter and its compaction into the
// oriented CSR N+ (Sec. 4.2.1, Alg. 2 Form_Filtered_Edge_List), the
// intersection of N+(u) and N+(v) for every oriented edge (Sec. 3.2, Alg. 2
// Compute_Intersection: a sorted merge, or for a pair of very unequal lengths
// a search of each element of the shorter list in the longer one) and the
// reduction to T and t(v) (Alg. 2 Reduce).  Such graphs are launch-bound on
// the general path (some thirty kernels for a few thousand edges); here they
// take one launch of ceil(m/1024) CTAs, each of which orients the whole graph
// in its shared memory and counts its share of the oriented edges.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

constexpr int kFusedThreads = 1024;

__device__ __forceinline__ int fused_block_excl_scan(int v, int* sm, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int t = lane < nw ? sm[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) sm[lane] = ti - t;
        if (lane == 31) sm[32] = ti;
    }
    __syncthreads();
    const int r = sm[w] + inc - v;
    *total = sm[32];
    __syncthreads();
    return r;
}

// One CTA of kFusedThreads threads.  Shared memory (32-bit words): srp[n+1]
// (row offsets, so d(v) = srp[v+1] - srp[v]), tv[n] (per-vertex counts),
// rpp[n+1], kw[W] (one keep bit per input entry, W = ceil(nnz/32)), wpre[W]
// (kept entries before each word), colp[m], scan scratch[33].
//   rp, col : the input CSR on the device (simple, rows ascending).
//   total   : T; per_vertex (nullable): t(v) for v < n.  Both zeroed by the
//             host before the launch; every CTA adds its share.
// Every CTA of the grid orients and compacts the whole graph into its own
// shared memory (cheap at these sizes, and it needs no grid-wide barrier),
// then takes its share of the oriented edges.  The orientation needs only the comparison (d(u), u) < (d(v), v), so no rank
// is formed.  The input entries are walked in coalesced runs (one warp = 32
// consecutive entries = one keep word), so the loads of the whole CSR are in
// flight at once; kept entries keep their input order, so an entry's place in
// N+ is the number of kept entries before it (wpre plus a popcount), as in
// the build.
constexpr int kFusedRun = 8;  // keep words per warp and step (loads in flight per lane)
__global__ void __launch_bounds__(kFusedThreads) k_count_fused(int n, int nnz, int m,
                                                               const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ col,
                                                               unsigned long long* __restrict__ total,
                                                               unsigned long long* __restrict__ per_vertex) {
    extern __shared__ __align__(16) unsigned fsm[];
    const int W = (nnz + 31) >> 5;
    int* srp = reinterpret_cast<int*>(fsm);
    int* tv = srp + n + 1;
    int* rpp = tv + n;
    unsigned* kw = reinterpret_cast<unsigned*>(rpp + n + 1);
    int* wpre = reinterpret_cast<int*>(kw + W);
    int* colp = wpre + W;
    int* scan = colp + m;
    __shared__ unsigned long long s_T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (tid == 0) s_T = 0;
    // every slot of N+ holds a vertex id even if the input is not a symmetric
    // simple CSR (then the counts are meaningless, but every index stays in range)
    for (int i = tid; i < m; i += nt) colp[i] = 0;
    for (int v = tid; v <= n; v += nt) srp[v] = (int)min(max(rp[v], (int64_t)0), (int64_t)nnz);
    __syncthreads();
    // orientation filter: entry j of row u is kept iff (d(u), u) < (d(v), v), v = col[j]
    for (int w0 = warp * kFusedRun; w0 < W; w0 += nw * kFusedRun) {
        int vv[kFusedRun];
#pragma unroll
        for (int q = 0; q < kFusedRun; ++q) {
            const int j = (w0 + q) * 32 + lane;
            vv[q] = (w0 + q < W && j < nnz) ? col[j] : -1;
        }
#pragma unroll
        for (int q = 0; q < kFusedRun; ++q) {
            if (w0 + q >= W) break;  // the same for the whole warp
            const int j = (w0 + q) * 32 + lane;
            bool kp = false;
            if (j < nnz && (unsigned)vv[q] < (unsigned)n) {
                int lo = 0, hi = n;  // the row u with srp[u] <= j < srp[u+1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (srp[mid] <= j) lo = mid;
                    else hi = mid;
                }
                const int v = vv[q];
                const int du = srp[lo + 1] - srp[lo], dv = srp[v + 1] - srp[v];
                kp = dv > du || (dv == du && v > lo);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) kw[w0 + q] = bal;
        }
    }
    __syncthreads();
    // wpre = exclusive prefix of the kept entries per keep word
    {
        const int per = (W + nt - 1) / nt;
        const int w0 = min(W, tid * per), w1 = min(W, w0 + per);
        int c = 0;
        for (int w = w0; w < w1; ++w) c += __popc(kw[w]);
        int tot;
        int run = fused_block_excl_scan(c, scan, &tot);
        for (int w = w0; w < w1; ++w) {
            wpre[w] = run;
            run += __popc(kw[w]);
        }
    }
    __syncthreads();
    // rpp[u] = kept entries before row u (a symmetric simple CSR keeps exactly
    // m entries; the clamp keeps any other input inside the arrays)
    for (int u = tid; u <= n; u += nt) {
        const int x = srp[u];
        const int w = x >> 5;
        const int before = w < W ? wpre[w] + __popc(kw[w] & ((1u << (x & 31)) - 1u))
                                 : (W > 0 ? wpre[W - 1] + __popc(kw[W - 1]) : 0);
        rpp[u] = min(before, m);
        if (u < n) tv[u] = 0;
    }
    // compaction: each kept entry to its place in N+ (rows stay ascending)
    for (int w0 = warp * kFusedRun; w0 < W; w0 += nw * kFusedRun) {
#pragma unroll
        for (int q = 0; q < kFusedRun; ++q) {
            const int w = w0 + q;
            if (w >= W) break;
            const unsigned bits = kw[w];
            if ((bits >> lane) & 1u) {
                const int pos = wpre[w] + __popc(bits & ((1u << lane) - 1u));
                if (pos < m) colp[pos] = col[w * 32 + lane];
            }
        }
    }
    __syncthreads();
    // intersection: one thread per oriented edge (u, v), a sorted merge of
    // N+(u) and N+(v); every common w closes the triangle (u, v, w).  The
    // CTAs of the grid share the edges (each has built the same N+ above).
    unsigned long long acc = 0;
    const int me = rpp[n];
    for (int e = blockIdx.x * nt + tid; e < me; e += gridDim.x * nt) {
        int lo = 0, hi = n;  // the row u with rpp[u] <= e < rpp[u+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rpp[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int u = lo, v = colp[e];
        int a = rpp[u], ae = rpp[u + 1], b = rpp[v], be = rpp[v + 1];
        if (ae - a > be - b) {  // [a, ae) the shorter list, [b, be) the longer
            const int t0 = a, t1 = ae;
            a = b;
            ae = be;
            b = t0;
            be = t1;
        }
        unsigned c = 0;
        if (8 * (ae - a) < be - b) {
            // skewed pair: each element of the shorter list is searched in the
            // rest of the longer one (both ascending)
            for (; a < ae && b < be; ++a) {
                const int x = colp[a];
                int l = b, h = be;
                while (l < h) {
                    const int mid = (l + h) >> 1;
                    if (colp[mid] < x) l = mid + 1;
                    else h = mid;
                }
                if (l < be && colp[l] == x) {
                    atomicAdd(reinterpret_cast<unsigned*>(&tv[x]), 1u);
                    ++c;
                    ++l;
                }
                b = l;
            }
        } else {
            while (a < ae && b < be) {
                const int x = colp[a], y = colp[b];
                if (x == y) {
                    atomicAdd(reinterpret_cast<unsigned*>(&tv[x]), 1u);
                    ++c;
                    ++a;
                    ++b;
                } else if (x < y) {
                    ++a;
                } else {
                    ++b;
                }
            }
        }
        if (c) {
            atomicAdd(reinterpret_cast<unsigned*>(&tv[u]), c);
            atomicAdd(reinterpret_cast<unsigned*>(&tv[v]), c);
            acc += c;
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&s_T, acc);
    __syncthreads();
    // this CTA's share of T and t(v), added to the outputs the host zeroed
    if (tid == 0 && s_T) atomicAdd(total, s_T);
    if (per_vertex)
        for (int u = tid; u < n; u += nt) {
            const unsigned c = (unsigned)tv[u];
            if (c) atomicAdd(&per_vertex[u], (unsigned long long)c);
        }
}

// Shared-memory bytes of the fused kernel for n vertices and m oriented edges
// (-1 when the graph is outside its limits).
static int64_t fused_smem_bytes(int64_t n, int64_t m) {
    if (n < 0 || n > kFusedMaxN || m < 0) return -1;
    const int64_t W = (2 * m + 31) / 32;
    const int64_t words = (n + 1) + n + (n + 1) + 2 * W + m + 33;
    return 4 * words;
}

bool fused_fits(int64_t n, int64_t nnz) {
    const int64_t b = fused_smem_bytes(n, nnz / 2);
    return b >= 0 && b <= kFusedMaxSmem;
}

cudaError_t launch_fused(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col, unsigned long long* total,
                         unsigned long long* per_vertex, cudaStream_t s) {
    const int64_t m = nnz / 2;
    const int64_t bytes = fused_smem_bytes(n, m);
    if (bytes < 0 || bytes > kFusedMaxSmem) return cudaErrorInvalidValue;
    int dev = 0, num_sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    // one CTA (one SM) per 1024 oriented edges: each CTA then merges about
    // one edge per thread
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(num_sms, 1), (m + kFusedThreads - 1) / kFusedThreads));
    cudaError_t e = cudaFuncSetAttribute(k_count_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && per_vertex && n > 0)
        e = cudaMemsetAsync(per_vertex, 0, sizeof(unsigned long long) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    k_count_fused<<<ctas, kFusedThreads, (size_t)bytes, s>>>((int)n, (int)nnz, (int)m, rp, col, total, per_vertex);
    return cudaGetLastError();
}

}  // namespace tc
