// tc_metrics.cu -- triangle-derived metrics on the device: local clustering
// coefficients and transitivity (the paper names them as the immediate use
// of the counts, Sec. 5: "clustering coefficient and transitivity metrics").
//
//   wedges(v)  = d(v) (d(v) - 1) / 2   (paths of length two centred at v)
//   c(v)       = t(v) / wedges(v), 0 when d(v) < 2
//   W          = sum_v wedges(v)
//   transitivity = 3 T / W, 0 when W = 0
// Each ratio is one IEEE division of two exact integers (< 2^53), so the
// result is the correctly rounded quotient.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

__global__ void k_local_clustering(int64_t n, const int32_t* __restrict__ deg, const unsigned long long* __restrict__ t,
                                   double* __restrict__ coeff, unsigned long long* __restrict__ wedges) {
    __shared__ unsigned long long s_w;
    if (threadIdx.x == 0) s_w = 0;
    __syncthreads();
    unsigned long long wsum = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const long long d = deg[v];
        const unsigned long long w = (unsigned long long)(d * (d - 1) / 2);
        wsum += w;
        if (coeff) coeff[v] = w ? (double)t[v] / (double)w : 0.0;
    }
    for (int o = 16; o; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&s_w, wsum);
    __syncthreads();
    if (threadIdx.x == 0 && s_w) atomicAdd(wedges, s_w);
}

__global__ void k_transitivity(const unsigned long long* __restrict__ total, const unsigned long long* __restrict__ wedges,
                               double* __restrict__ out) {
    const unsigned long long w = *wedges;
    *out = w ? (double)(3ull * *total) / (double)w : 0.0;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_clustering(tc_ctx* ctx, const tc_ocsr* o, const int64_t* total, const int64_t* per_vertex,
                                   double* local, double* transitivity, int64_t* wedges, void* stream) {
    if (!ctx || !o || !per_vertex || (transitivity && !total))
        return set_err(ctx, TC_ERR_INVALID_ARG, "clustering: per_vertex (and total for transitivity) required");
    if (o->G > 0) return set_err(ctx, TC_ERR_INVALID_ARG, "clustering: batch handles are not supported");
    cudaSetDevice(o->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* dw = nullptr;
    double* dtr = nullptr;
    cudaError_t e = dev_alloc((void**)&dw, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = dev_alloc((void**)&dtr, sizeof(double), s);
    if (e != cudaSuccess) {
        dev_free(dw, s);
        return set_err(ctx, TC_ERR_OOM, "clustering: scratch allocation failed");
    }
    // a host `local` goes through device scratch
    double* dl = local;
    cudaPointerAttributes at;
    const bool host_local = local && (cudaPointerGetAttributes(&at, local) != cudaSuccess ||
                                      at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered);
    cudaGetLastError();
    if (host_local && dev_alloc((void**)&dl, sizeof(double) * (size_t)std::max<int64_t>(o->n, 1), s) != cudaSuccess) {
        dev_free(dw, s);
        dev_free(dtr, s);
        return set_err(ctx, TC_ERR_OOM, "clustering: scratch allocation failed");
    }
    cudaMemsetAsync(dw, 0, sizeof(unsigned long long), s);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((o->n + 255) / 256, (int64_t)ctx->num_sms * 8));
    k_local_clustering<<<grid, 256, 0, s>>>(o->n, o->deg, (const unsigned long long*)per_vertex, dl, dw);
    if (host_local && o->n > 0) e = cudaMemcpyAsync(local, dl, sizeof(double) * (size_t)o->n, cudaMemcpyDeviceToHost, s);
    if (host_local) dev_free(dl, s);
    TC_LAUNCH(ctx);
    if (e == cudaSuccess && transitivity) {
        k_transitivity<<<1, 1, 0, s>>>((const unsigned long long*)total, dw, dtr);
        TC_LAUNCH(ctx);
        e = cudaMemcpyAsync(transitivity, dtr, sizeof(double), cudaMemcpyDefault, s);
    }
    if (e == cudaSuccess && wedges) e = cudaMemcpyAsync(wedges, dw, sizeof(int64_t), cudaMemcpyDefault, s);
    dev_free(dw, s);
    dev_free(dtr, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "clustering");
    return TC_OK;
}
