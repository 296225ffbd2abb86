// tc_sort.cu -- edge list -> simple undirected CSR on the device.
//
// The paper's datasets are de-duplicated and counted in both directions
// (Table 1 caption); an edge-list input is brought to that form here:
// self-loops dropped, both directions emitted, an LSD radix sort of the
// (u, v) keys, duplicates dropped, row offsets from the run boundaries.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// key = u * 2^b + v; a self-loop becomes the all-ones sentinel (sorts last)
__global__ void k_make_keys(int64_t np, const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t n,
                            int b, unsigned long long sentinel, unsigned long long* __restrict__ keys,
                            int* __restrict__ err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = src[i], v = dst[i];
        unsigned long long k0 = sentinel, k1 = sentinel;
        if (u < 0 || u >= n || v < 0 || v >= n) atomicOr(err, 1);
        else if (u != v) {
            k0 = ((unsigned long long)u << b) | (unsigned long long)v;
            k1 = ((unsigned long long)v << b) | (unsigned long long)u;
        }
        keys[2 * i] = k0;
        keys[2 * i + 1] = k1;
    }
}

// A pass is trivial when every key's digit is 0: with maxv given, digit
// bits [shift, shift+8) of a key are bits [shift-vbase, ...) of a value that
// is at most *maxv.  A trivial pass is the identity and does nothing.  The
// trivial passes are the last ones (a digit above the highest set bit of
// *maxv), so the keys end in the buffer that the last real pass wrote.
__device__ __forceinline__ bool rs_trivial(const int* maxv, int vbase, int shift) {
    return maxv && shift >= vbase && ((unsigned)*maxv >> (shift - vbase)) == 0u;
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const unsigned long long* __restrict__ keys, int64_t K, int shift,
                                                        int32_t* __restrict__ hist, int64_t ntiles,
                                                        const int* __restrict__ maxv, int vbase) {
    if (rs_trivial(maxv, vbase, shift)) return;
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + r * kRsThreads + threadIdx.x;
        if (i < K) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of a tile keep their order within each digit.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const unsigned long long* __restrict__ in,
                                                           unsigned long long* __restrict__ out, int64_t K, int shift,
                                                           const int64_t* __restrict__ off, int64_t ntiles,
                                                           const int* __restrict__ maxv, int vbase) {
    __shared__ int wcnt[kRsWarps][256];
    __shared__ int run[256];
    __shared__ long long base[256];
    const int tid = threadIdx.x, warp = tid >> 5;
    if (rs_trivial(maxv, vbase, shift)) return;
    run[tid] = 0;
    base[tid] = off[(int64_t)tid * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = t0 + r * kRsThreads + tid;
        const bool valid = i < K;
        const unsigned long long key = valid ? in[i] : 0ull;
        const int d = valid ? (int)((key >> shift) & 255u) : 256;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int acc = run[tid];
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {
                const int c = wcnt[w][tid];
                wcnt[w][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) out[base[d] + wcnt[warp][d] + rank] = key;
        __syncthreads();
    }
}

// LSD radix sort of K keys on bits [low_bit, key_bits) (8 bits per pass,
// stable).  ka holds the input, kb is scratch of the same size.  Without
// maxv, *sorted receives whichever of the two holds the result.  With maxv,
// the passes made trivial by it do nothing, so the result is in ka after an
// even number of real passes and in kb after an odd one, which only the
// device knows: *sorted receives ka, and the consumer counts the real passes
// from *maxv to pick the buffer (k_rank_from_sorted in tc_build.cu).
cudaError_t radix_sort_u64(unsigned long long* ka, unsigned long long* kb, int64_t K, int key_bits, cudaStream_t s,
                           unsigned long long** sorted, long long* launches, int low_bit, const int* maxv, int vbase) {
    *sorted = ka;
    if (K <= 0) return cudaSuccess;
    const int64_t ntiles = (K + kRsTile - 1) / kRsTile;
    const int64_t nh = 256 * ntiles;
    int32_t* hist = nullptr;
    int64_t* hoff = nullptr;
    void* stmp = nullptr;
    const size_t stb = scan_tmp_bytes(nh);
    cudaError_t e = dev_alloc((void**)&hist, sizeof(int32_t) * nh, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&hoff, sizeof(int64_t) * (nh + 1), s);
    if (e == cudaSuccess) e = dev_alloc(&stmp, stb, s);
    if (e == cudaSuccess) {
        for (int shift = low_bit; shift < key_bits; shift += 8) {
            k_rs_hist<<<(unsigned)ntiles, kRsThreads, 0, s>>>(ka, K, shift, hist, ntiles, maxv, vbase);
            scan_i32_to_i64(hist, hoff, nh, stmp, stb, s);
            k_rs_scatter<<<(unsigned)ntiles, kRsThreads, 0, s>>>(ka, kb, K, shift, hoff, ntiles, maxv, vbase);
            std::swap(ka, kb);
            if (launches) *launches += 5;
        }
        *sorted = ka;
        e = cudaGetLastError();
    }
    dev_free(hist, s);
    dev_free(hoff, s);
    dev_free(stmp, s);
    return e;
}

// flag[i] = 1 for the first copy of a non-sentinel key
__global__ void k_mark_unique(const unsigned long long* __restrict__ keys, int64_t K, unsigned long long sentinel,
                              int32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        flag[i] = (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

__global__ void k_compact(const unsigned long long* __restrict__ keys, int64_t K, const int32_t* __restrict__ flag,
                          const int64_t* __restrict__ pos, int b, unsigned long long* __restrict__ ckeys,
                          int32_t* __restrict__ col) {
    const unsigned long long vmask = (1ull << b) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            ckeys[pos[i]] = keys[i];
            col[pos[i]] = (int32_t)(keys[i] & vmask);
        }
    }
}

// run boundaries of u in the compacted keys -> degree per row
__global__ void k_row_bounds(const unsigned long long* __restrict__ ck, const int64_t* __restrict__ nnz_p, int b,
                             int32_t* __restrict__ deg) {
    const int64_t nnz = *nnz_p;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long u = ck[p] >> b;
        if (p == nnz - 1 || (ck[p + 1] >> b) != u) {
            // last entry of row u: its degree is p+1 minus the first position of the run
            int64_t lo = 0, hi = p;  // first index with key>>b == u
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((ck[mid] >> b) < u) lo = mid + 1; else hi = mid;
            }
            deg[u] = (int32_t)(p + 1 - lo);
        }
    }
}

tc_status edges_to_csr(tc_ctx* ctx, int64_t n, int64_t np, const int32_t* src, const int32_t* dst, int64_t** row_ptr,
                       int32_t** col, int64_t* nnz_out, cudaStream_t s) {
    int b = 1;
    while (((int64_t)1 << b) < n) ++b;
    const int key_bits = 2 * b;
    const unsigned long long sentinel = key_bits >= 64 ? ~0ull : ((1ull << key_bits) - 1ull);
    const int64_t K = 2 * np;
    const int64_t ntiles = (K + kRsTile - 1) / kRsTile;
    const int64_t nh = 256 * std::max<int64_t>(ntiles, 1);
    unsigned long long *ka = nullptr, *kb = nullptr;
    int32_t* hist = nullptr;
    int64_t* hoff = nullptr;
    int32_t* flag = nullptr;
    int64_t* pos = nullptr;
    int32_t* deg = nullptr;
    int* err = nullptr;
    void* stmp = nullptr;
    const size_t stb = scan_tmp_bytes(std::max<int64_t>(std::max(nh, K), n));
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = dev_alloc(p, bytes, s);
    };
    A((void**)&ka, sizeof(unsigned long long) * std::max<int64_t>(K, 1));
    A((void**)&kb, sizeof(unsigned long long) * std::max<int64_t>(K, 1));
    A((void**)&hist, sizeof(int32_t) * nh);
    A((void**)&hoff, sizeof(int64_t) * (nh + 1));
    A((void**)&flag, sizeof(int32_t) * std::max<int64_t>(K, 1));
    A((void**)&pos, sizeof(int64_t) * (K + 1));
    A((void**)&deg, sizeof(int32_t) * std::max<int64_t>(n, 1));
    A((void**)&err, sizeof(int));
    A(&stmp, stb);
    A((void**)row_ptr, sizeof(int64_t) * (n + 1));
    A((void**)col, sizeof(int32_t) * std::max<int64_t>(K, 1));
    auto cleanup = [&]() {
        dev_free(ka, s); dev_free(kb, s); dev_free(hist, s); dev_free(hoff, s); dev_free(flag, s);
        dev_free(pos, s); dev_free(deg, s); dev_free(err, s); dev_free(stmp, s);
    };
    if (e != cudaSuccess) {
        cleanup();
        dev_free(*row_ptr, s); dev_free(*col, s);
        *row_ptr = nullptr; *col = nullptr;
        return set_err(ctx, TC_ERR_OOM, "edge list: device allocation failed");
    }
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((std::max(K, n) + 255) / 256, (int64_t)ctx->num_sms * 16));
    int64_t nnz = 0;
    int herr = 0;
    {
    PhaseScope ph(ctx, kPhEdgeSort, s);
    ctx->launches += 8 + 5 * ((key_bits + 7) / 8);  // includes the radix-sort passes
    cudaMemsetAsync(err, 0, sizeof(int), s);
    if (np > 0) k_make_keys<<<grid, 256, 0, s>>>(np, src, dst, n, b, sentinel, ka, err);
    {
        unsigned long long* sorted = ka;
        radix_sort_u64(ka, kb, K, key_bits, s, &sorted, nullptr, 0);
        if (sorted != ka) std::swap(ka, kb);
    }
    if (K > 0) k_mark_unique<<<grid, 256, 0, s>>>(ka, K, sentinel, flag);
    scan_i32_to_i64(flag, pos, K, stmp, stb, s);
    if (K > 0) k_compact<<<grid, 256, 0, s>>>(ka, K, flag, pos, b, kb, *col);
    cudaMemsetAsync(deg, 0, sizeof(int32_t) * std::max<int64_t>(n, 1), s);
    if (K > 0) k_row_bounds<<<grid, 256, 0, s>>>(kb, pos + K, b, deg);
    scan_i32_to_i64(deg, *row_ptr, n, stmp, stb, s);
    }
    cudaMemcpyAsync(&nnz, pos + K, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cleanup();
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || herr) {
        dev_free(*row_ptr, s); dev_free(*col, s);
        *row_ptr = nullptr; *col = nullptr;
        if (e != cudaSuccess) return cuda_err(ctx, e, "edge list");
        return set_err(ctx, TC_ERR_INVALID_GRAPH, "edge list: vertex id outside [0, n)");
    }
    *nnz_out = nnz;
    return TC_OK;
}

}  // namespace tc
