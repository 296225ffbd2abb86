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

// One CTA of kFusedThreads threads.  Shared memory (32-bit words): key[N2]
// (N2 = n rounded up to a power of two, at least 1), rnk[n], dpl[n] (d+, then
// the per-vertex counts), rpp[n+1], colp[m], scan scratch[33].
//   rp, col : the input CSR on the device (simple, rows ascending, n <= 2^13
//             so that (degree << idbits) | id fits 32 bits).
//   total   : T; per_vertex (nullable): t(v) for v < n.  Both overwritten.
__global__ void __launch_bounds__(kFusedThreads) k_count_fused(int n, int N2, int idbits, int m,
                                                               const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ col,
                                                               unsigned long long* __restrict__ total,
                                                               unsigned long long* __restrict__ per_vertex) {
    extern __shared__ __align__(16) unsigned fsm[];
    unsigned* key = fsm;
    int* rnk = reinterpret_cast<int*>(key + N2);
    int* dpl = rnk + n;
    int* rpp = dpl + n;
    int* colp = rpp + n + 1;
    int* scan = colp + m;
    __shared__ unsigned long long s_T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (tid == 0) s_T = 0;
    // every slot of N+ holds a vertex id even if the input is not a symmetric
    // simple CSR (then the counts are meaningless, but every index stays in range)
    for (int i = tid; i < m; i += nt) colp[i] = 0;
    // degrees and (degree, id) keys; padding sorts last
    for (int v = tid; v < N2; v += nt)
        key[v] = v < n ? ((unsigned)(rp[v + 1] - rp[v]) << idbits) | (unsigned)v : 0xffffffffu;
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
    // orientation filter: d+(u) = neighbours of higher rank (one warp per row)
    for (int u = warp; u < n; u += nw) {
        const int ru = rnk[u];
        const int64_t b = rp[u], e = rp[u + 1];
        int c = 0;
        for (int64_t j = b + lane; j < e; j += 32) {
            const unsigned v = (unsigned)col[j];
            c += v < (unsigned)n && rnk[v] > ru;  // an id out of range is never kept
        }
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) dpl[u] = c;
    }
    __syncthreads();
    // rpp = exclusive prefix of d+ (each thread scans a contiguous run of rows)
    {
        const int per = (n + nt - 1) / nt;
        const int u0 = min(n, tid * per), u1 = min(n, u0 + per);
        int s = 0;
        for (int u = u0; u < u1; ++u) s += dpl[u];
        int tot;
        int run = fused_block_excl_scan(s, scan, &tot);
        // a symmetric simple CSR keeps exactly m entries; the clamp keeps any
        // other input inside the arrays
        for (int u = u0; u < u1; ++u) {
            rpp[u] = min(run, m);
            run += dpl[u];
        }
        if (tid == 0) rpp[n] = min(tot, m);
    }
    __syncthreads();
    // compaction: the kept neighbours of u in input (id) order, so that every
    // N+(u) is ascending; dpl becomes the per-vertex triangle counts
    for (int u = warp; u < n; u += nw) {
        const int ru = rnk[u];
        const int64_t b = rp[u], e = rp[u + 1];
        int o = rpp[u];
        for (int64_t j0 = b; j0 < e; j0 += 32) {
            const int64_t j = j0 + lane;
            int v = 0;
            bool kp = false;
            if (j < e) {
                v = col[j];
                kp = (unsigned)v < (unsigned)n && rnk[v] > ru;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, kp);
            const int pos = o + __popc(bal & ((1u << lane) - 1u));
            if (kp && pos < m) colp[pos] = v;
            o += __popc(bal);
        }
    }
    __syncthreads();
    for (int u = tid; u < n; u += nt) dpl[u] = 0;
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
                atomicAdd(reinterpret_cast<unsigned*>(&dpl[x]), 1u);
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
            atomicAdd(reinterpret_cast<unsigned*>(&dpl[u]), c);
            atomicAdd(reinterpret_cast<unsigned*>(&dpl[v]), c);
            acc += c;
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&s_T, acc);
    __syncthreads();
    if (tid == 0) *total = s_T;
    if (per_vertex)
        for (int u = tid; u < n; u += nt) per_vertex[u] = (unsigned long long)(unsigned)dpl[u];
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
    const int64_t words = N2 + 3 * n + 1 + m + 33;
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
    k_count_fused<<<1, kFusedThreads, (size_t)bytes, s>>>((int)n, N2, idbits, (int)m, rp, col, total, per_vertex);
    return cudaGetLastError();
}

}  // namespace tc
