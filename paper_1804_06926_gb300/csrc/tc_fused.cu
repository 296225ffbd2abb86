// tc_fused.cu -- the whole method for one small graph in one kernel launch.
//
// A graph whose degree keys, ranks, oriented CSR and per-vertex counts fit in
// one CTA's shared memory is counted by a single CTA: degrees and the
// (degree, id) rank (Sec. 4.2.1), the orientation filter and its compaction
// into the oriented CSR N+ (Sec. 4.2.1, Alg. 2 Form_Filtered_Edge_List), the
// sorted-merge intersection of N+(u) and N+(v) for every oriented edge
// (Sec. 3.2, Alg. 2 Compute_Intersection) and the reduction to T and t(v)
// (Alg. 2 Reduce).  Such graphs are launch-bound on the general path (some
// thirty kernels for a few thousand edges); here they take one launch.
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
// (row offsets), key[N2] (N2 = n rounded up to a power of two, at least 1),
// rnk[n], tv[n] (per-vertex counts), rpp[n+1], kw[W] (one keep bit per input
// entry, W = ceil(nnz/32)), wpre[W] (kept entries before each word), colp[m],
// scan scratch[33].
//   rp, col : the input CSR on the device (simple, rows ascending, n <= 2^13
//             so that (degree << idbits) | id fits 32 bits).
//   total   : T; per_vertex (nullable): t(v) for v < n.  Both overwritten.
// The input entries are walked in coalesced runs (one warp = 32 consecutive
// entries = one keep word), so the loads of the whole CSR are in flight at
// once; kept entries keep their input order, so an entry's place in N+ is the
// number of kept entries before it (wpre plus a popcount), as in the build.
constexpr int kFusedRun = 8;  // keep words per warp and step (loads in flight per lane)
__global__ void __launch_bounds__(kFusedThreads) k_count_fused(int n, int N2, int idbits, int nnz, int m,
                                                               const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ col,
                                                               unsigned long long* __restrict__ total,
                                                               unsigned long long* __restrict__ per_vertex) {
    extern __shared__ __align__(16) unsigned fsm[];
    const int W = (nnz + 31) >> 5;
    int* srp = reinterpret_cast<int*>(fsm);
    unsigned* key = reinterpret_cast<unsigned*>(srp + n + 1);
    int* rnk = reinterpret_cast<int*>(key + N2);
    int* tv = rnk + n;
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
    // degrees and (degree, id) keys; padding sorts last
    for (int v = tid; v < N2; v += nt)
        key[v] = v < n ? ((unsigned)(srp[v + 1] - srp[v]) << idbits) | (unsigned)v : 0xffffffffu;
    __syncthreads();
    // bitonic sort of the keys, ascending: key[i] = the vertex of rank i
    for (int k = 2; k <= N2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < N2; i += nt) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned a = key[i], b = key[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    const unsigned idmask = (1u << idbits) - 1u;
    for (int i = tid; i < n; i += nt) rnk[key[i] & idmask] = i;
    __syncthreads();
    // orientation filter: entry j of row u is kept iff rank(u) < rank(col[j])
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
                kp = rnk[vv[q]] > rnk[lo];
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
    // N+(u) and N+(v); every common w closes the triangle (u, v, w)
    unsigned long long acc = 0;
    const int me = rpp[n];
    for (int e = tid; e < me; e += nt) {
        int lo = 0, hi = n;  // the row u with rpp[u] <= e < rpp[u+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rpp[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int u = lo, v = colp[e];
        int a = rpp[u], ae = rpp[u + 1], b = rpp[v], be = rpp[v + 1];
        unsigned c = 0;
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
        if (c) {
            atomicAdd(reinterpret_cast<unsigned*>(&tv[u]), c);
            atomicAdd(reinterpret_cast<unsigned*>(&tv[v]), c);
            acc += c;
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&s_T, acc);
    __syncthreads();
    if (tid == 0) *total = s_T;
    if (per_vertex)
        for (int u = tid; u < n; u += nt) per_vertex[u] = (unsigned long long)(unsigned)tv[u];
}

static int fused_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Shared-memory bytes of the fused kernel for n vertices and m oriented edges
// (-1 when the graph is outside its limits).
static int64_t fused_smem_bytes(int64_t n, int64_t m) {
    if (n < 0 || n > kFusedMaxN || m < 0) return -1;
    const int64_t N2 = fused_pow2((int)std::max<int64_t>(n, 1));
    const int64_t W = (2 * m + 31) / 32;
    const int64_t words = (n + 1) + N2 + 2 * n + (n + 1) + 2 * W + m + 33;
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
    const int N2 = fused_pow2((int)std::max<int64_t>(n, 1));
    int idbits = 1;
    while ((int64_t(1) << idbits) < n) ++idbits;
    cudaError_t e = cudaFuncSetAttribute(k_count_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_count_fused<<<1, kFusedThreads, (size_t)bytes, s>>>((int)n, N2, idbits, (int)nnz, (int)m, rp, col, total,
                                                           per_vertex);
    return cudaGetLastError();
}

}  // namespace tc
