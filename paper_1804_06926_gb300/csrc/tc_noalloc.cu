// tc_noalloc.cu -- tc_orient_noalloc: the orientation filter and compaction
// into caller-owned buffers, without allocating any device memory.
//
// Some callers cannot allocate device memory once they are running: serving
// loops with a latency budget (cudaMalloc and cudaFree may synchronise the
// device) and processes whose HBM is already fully reserved by another
// allocator.  This entry point lets them build the oriented CSR with buffers
// they own.
//
// Its only scratch is the tile-sum array of the exclusive scan over the
// per-row kept counts.  It lives in a file-scope __device__ array of fixed
// size (64 KiB + padding), so every GPU that loads the library holds it until
// the process exits.  All calls share that array and it keeps the contents of
// the last call; the scan writes every tile sum it reads, so nothing needs
// clearing.  Calls whose work overlaps on the GPU (on different streams, or
// from different host threads) race on the array: serialise them.
#include <algorithm>
#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr int64_t kNoallocMaxN = TC_NOALLOC_MAX_VERTICES;
constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr int kNaTile = kNaThreads * kNaItems;
constexpr int64_t kNaMaxTiles = (kNoallocMaxN + kNaTile - 1) / kNaTile + 1;

// Scan scratch: one int64 sum per tile of kNaTile rows.
static __device__ __align__(256) long long g_noalloc_tile_sums[kNaMaxTiles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
long long* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current and kept for the life of the process
// (a cudaDeviceReset of the device would move the array; the header says so).
cudaError_t scratch_ptr(int dev, long long** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tile_sums);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<long long*>(p);
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

__device__ __forceinline__ long long na_warp_incl_scan(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ long long na_block_excl_scan(long long v, long long* sm, long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long inc = na_warp_incl_scan(v);
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        const long long t = lane < nw ? sm[lane] : 0;
        const long long ti = na_warp_incl_scan(t);
        if (lane < nw) sm[lane] = ti - t;
        if (lane == 31) sm[32] = ti;
    }
    __syncthreads();
    const long long r = sm[w] + inc - v;
    *total = sm[32];
    __syncthreads();
    return r;
}

// rank(v) = (d(v), v) with d read from the row offsets
__device__ __forceinline__ bool na_keep(int64_t du, int64_t u, int64_t dv, int64_t v) {
    return du < dv || (du == dv && u < v);
}

// Pass 1: kept entries of row u (one warp per row) -> rpp[u].
__global__ void k_na_orient_count(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  int64_t* __restrict__ rpp) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < n; u += nw) {
        const int64_t b = rp[u], e = rp[u + 1], du = e - b;
        int kept = 0;
        for (int64_t i = b + lane; i - lane < e; i += 32) {
            bool keep = false;
            if (i < e) {
                const int64_t v = col[i];
                keep = na_keep(du, u, rp[v + 1] - rp[v], v);
            }
            kept += __popc(__ballot_sync(0xffffffffu, keep));
        }
        if (lane == 0) rpp[u] = kept;
    }
}

// Pass 2: in-place exclusive scan of rpp[0..n), rpp[n] = total.
__global__ void __launch_bounds__(kNaThreads) k_na_scan_reduce(const int64_t* __restrict__ x, int64_t n,
                                                               long long* __restrict__ tile_sum) {
    __shared__ long long sm[33];
    const int64_t base = (int64_t)blockIdx.x * kNaTile;
    long long s = 0;
    for (int j = 0; j < kNaItems; ++j) {
        const int64_t i = base + j * kNaThreads + threadIdx.x;
        if (i < n) s += x[i];
    }
    long long tot;
    na_block_excl_scan(s, sm, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_na_scan_sums(long long* __restrict__ tile_sum, int64_t ntiles,
                                                       int64_t* __restrict__ x, int64_t n) {
    __shared__ long long sm[33];
    long long carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const long long v = i < ntiles ? tile_sum[i] : 0;
        long long tot;
        const long long ex = na_block_excl_scan(v, sm, &tot);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) x[n] = carry;
}

__global__ void __launch_bounds__(kNaThreads) k_na_scan_apply(int64_t* __restrict__ x, int64_t n,
                                                              const long long* __restrict__ tile_off) {
    __shared__ long long sm[33];
    const int64_t base = (int64_t)blockIdx.x * kNaTile + (int64_t)threadIdx.x * kNaItems;
    long long v[kNaItems];
    long long s = 0;
    for (int j = 0; j < kNaItems; ++j) {
        v[j] = (base + j < n) ? x[base + j] : 0;
        s += v[j];
    }
    long long tot;
    long long run = tile_off[blockIdx.x] + na_block_excl_scan(s, sm, &tot);
    for (int j = 0; j < kNaItems; ++j) {
        if (base + j < n) x[base + j] = run;
        run += v[j];
    }
}

// Pass 3: kept neighbours of row u at rpp[u], in input (ascending) order.
__global__ void k_na_orient_scatter(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const int64_t* __restrict__ rpp, int32_t* __restrict__ colp) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < n; u += nw) {
        const int64_t b = rp[u], e = rp[u + 1], du = e - b;
        int64_t out = rpp[u];
        for (int64_t i = b + lane; i - lane < e; i += 32) {
            bool keep = false;
            int32_t v = 0;
            if (i < e) {
                v = col[i];
                keep = na_keep(du, u, rp[(int64_t)v + 1] - rp[v], v);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) colp[out + __popc(bal & ((1u << lane) - 1u))] = v;
            out += __popc(bal);
        }
    }
}

}  // namespace

extern "C" tc_status tc_orient_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                       int64_t* rpp_out, int32_t* colp_out, void* stream) {
    if (n < 0 || nnz < 0 || nnz % 2 || !row_ptr || !rpp_out || (nnz > 0 && (!col || !colp_out)))
        return TC_ERR_INVALID_ARG;
    if (n > kNoallocMaxN) return TC_ERR_INVALID_ARG;  // beyond the fixed scratch: use tc_build_oriented_csr
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    long long* tile_sums = nullptr;
    e = scratch_ptr(dev, &tile_sums);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ntiles = (n + kNaTile - 1) / kNaTile;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sms * 16));
    if (n > 0) k_na_orient_count<<<grid, 256, 0, s>>>(n, row_ptr, col, rpp_out);
    if (ntiles > 0) k_na_scan_reduce<<<(unsigned)ntiles, kNaThreads, 0, s>>>(rpp_out, n, tile_sums);
    k_na_scan_sums<<<1, 1024, 0, s>>>(tile_sums, ntiles, rpp_out, n);
    if (ntiles > 0) k_na_scan_apply<<<(unsigned)ntiles, kNaThreads, 0, s>>>(rpp_out, n, tile_sums);
    if (n > 0) k_na_orient_scatter<<<grid, 256, 0, s>>>(n, row_ptr, col, rpp_out, colp_out);
    e = cudaGetLastError();
    return e == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
