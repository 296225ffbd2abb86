// tc_support.cu -- per-edge triangle support and triangle listing.
//
// The paper notes that the methods it compares enumerate the triangles as
// well as count them, and that enumeration is the subroutine of k-truss
// (Sec. 1; Sec. 3.1 for subgraph matching).  For every oriented edge (u, v) the sorted
// lists N+(u) and N+(v) are merged (Sec. 3.2); each common w closes the
// triangle {u, v, w}, listed as (u, v, w) with rank(u) < rank(v) < rank(w),
// and adds one to the support of its three edges: (u, v) itself, (u, w) at
// w's position in N+(u) and (v, w) at w's position in N+(v) -- the merge
// yields both positions.  Support is indexed like the oriented CSR's col
// array (tc_ocsr_copy).
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

// SUP: support of all three edges; LIST: write the triangles; LOWER: only the
// per-edge count c(u, v) = |N+(u) & N+(v)| into sup[e] (the masked product).
template <bool SUP, bool LIST, bool LOWER = false>
__global__ void __launch_bounds__(256) k_support_list(int64_t n, const int64_t* __restrict__ rpp,
                                                      const int32_t* __restrict__ colp,
                                                      unsigned long long* __restrict__ sup, int32_t* __restrict__ tri,
                                                      long long cap, unsigned long long* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    unsigned long long found = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < n; u += nw) {
        const int64_t ub = rpp[u], ue = rpp[u + 1];
        for (int64_t e = ub + lane; e < ue; e += 32) {
            const int32_t v = colp[e];
            int64_t i = ub, k = rpp[v];
            const int64_t ke = rpp[(int64_t)v + 1];
            unsigned long long c = 0;
            while (i < ue && k < ke) {
                const int32_t x = colp[i], y = colp[k];
                if (x < y) ++i;
                else if (x > y) ++k;
                else {
                    ++c;
                    if (SUP) {
                        atomicAdd(&sup[i], 1ull);
                        atomicAdd(&sup[k], 1ull);
                    }
                    if (LIST) {
                        const unsigned long long slot = atomicAdd(count, 1ull);
                        if ((long long)slot < cap) {
                            tri[3 * slot + 0] = (int32_t)u;
                            tri[3 * slot + 1] = v;
                            tri[3 * slot + 2] = x;
                        }
                    }
                    ++i;
                    ++k;
                }
            }
            if (SUP && c) atomicAdd(&sup[e], c);
            if (LOWER) sup[e] = c;
            found += c;
        }
    }
    if (!LIST) {
        for (int o = 16; o; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
        if (lane == 0 && found) atomicAdd(count, found);
    }
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_edge_support(tc_ctx* ctx, const tc_ocsr* o, int64_t* support, int32_t* triangles,
                                     int64_t capacity, int64_t* count, void* stream) {
    if (!ctx || !o || !count || capacity < 0) return set_err(ctx, TC_ERR_INVALID_ARG, "edge support: bad arguments");
    if (o->G > 0) return set_err(ctx, TC_ERR_INVALID_ARG, "edge support: batch handles are not supported");
    cudaSetDevice(o->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* dcount = nullptr;
    cudaError_t e = dev_alloc((void**)&dcount, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_err(ctx, TC_ERR_OOM, "edge support: scratch allocation failed");
    // host outputs go through device scratch
    auto is_host = [](const void* p) {
        cudaPointerAttributes at;
        const bool h = cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type == cudaMemoryTypeHost ||
                       at.type == cudaMemoryTypeUnregistered;
        cudaGetLastError();
        return h;
    };
    unsigned long long* sup = (unsigned long long*)support;
    int32_t* tri = triangles;
    const bool h_sup = support && is_host(support), h_tri = triangles && capacity > 0 && is_host(triangles);
    if (h_sup) e = dev_alloc((void**)&sup, sizeof(int64_t) * (size_t)std::max<int64_t>(o->m, 1), s);
    if (e == cudaSuccess && h_tri) e = dev_alloc((void**)&tri, sizeof(int32_t) * 3 * (size_t)capacity, s);
    if (e != cudaSuccess) {
        if (h_sup) dev_free(sup, s);
        dev_free(dcount, s);
        return set_err(ctx, TC_ERR_OOM, "edge support: scratch allocation failed");
    }
    cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s);
    if (sup && o->m > 0) cudaMemsetAsync(sup, 0, sizeof(int64_t) * (size_t)o->m, s);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((o->n * 32 + 255) / 256, (int64_t)ctx->num_sms * 16));
    const bool list = tri != nullptr;
    if (o->n > 0) {
        if (sup && list) k_support_list<true, true><<<grid, 256, 0, s>>>(o->n, o->rpp, o->colp, sup, tri, capacity, dcount);
        else if (sup) k_support_list<true, false><<<grid, 256, 0, s>>>(o->n, o->rpp, o->colp, sup, nullptr, 0, dcount);
        else if (list) k_support_list<false, true><<<grid, 256, 0, s>>>(o->n, o->rpp, o->colp, nullptr, tri, capacity, dcount);
        else k_support_list<false, false><<<grid, 256, 0, s>>>(o->n, o->rpp, o->colp, nullptr, nullptr, 0, dcount);
        TC_LAUNCH(ctx);
    }
    if (h_sup && o->m > 0) cudaMemcpyAsync(support, sup, sizeof(int64_t) * (size_t)o->m, cudaMemcpyDeviceToHost, s);
    if (h_tri) cudaMemcpyAsync(triangles, tri, sizeof(int32_t) * 3 * (size_t)capacity, cudaMemcpyDeviceToHost, s);
    if (h_sup) dev_free(sup, s);
    if (h_tri) dev_free(tri, s);
    e = cudaMemcpyAsync(count, dcount, sizeof(int64_t), cudaMemcpyDefault, s);
    dev_free(dcount, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "edge support");
    return TC_OK;
}

// Alg. 3 of the paper (Sec. 3.3) with the TC-specific masking it proposes as
// future work (Sec. 5: compute only the upper triangle, only where A is
// nonzero, and never write B = LU to memory): with the vertices in decreasing
// rank order, C = A o (LU) is nonzero only at edges, and for the oriented
// edge e = (u, v) its upper-triangle entry is |N+(u) & N+(v)|.  c[e] receives
// it for every oriented edge (order of tc_ocsr_copy); sum c = T.
extern "C" tc_status tc_masked_product(tc_ctx* ctx, const tc_ocsr* o, int64_t* c, int64_t* total, void* stream) {
    if (!ctx || !o || !c) return set_err(ctx, TC_ERR_INVALID_ARG, "masked product: c is required");
    if (o->G > 0) return set_err(ctx, TC_ERR_INVALID_ARG, "masked product: batch handles are not supported");
    cudaSetDevice(o->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaPointerAttributes at;
    const bool h_c = cudaPointerGetAttributes(&at, c) != cudaSuccess || at.type == cudaMemoryTypeHost ||
                     at.type == cudaMemoryTypeUnregistered;
    cudaGetLastError();
    unsigned long long* dc = (unsigned long long*)c;
    unsigned long long* dcount = nullptr;
    cudaError_t e = dev_alloc((void**)&dcount, sizeof(unsigned long long), s);
    if (e == cudaSuccess && h_c) e = dev_alloc((void**)&dc, sizeof(int64_t) * (size_t)std::max<int64_t>(o->m, 1), s);
    if (e != cudaSuccess) {
        dev_free(dcount, s);
        return set_err(ctx, TC_ERR_OOM, "masked product: scratch allocation failed");
    }
    cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s);
    const unsigned grid =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((o->n * 32 + 255) / 256, (int64_t)ctx->num_sms * 16));
    if (o->n > 0) {
        k_support_list<false, false, true><<<grid, 256, 0, s>>>(o->n, o->rpp, o->colp, dc, nullptr, 0, dcount);
        TC_LAUNCH(ctx);
    }
    if (h_c && o->m > 0) cudaMemcpyAsync(c, dc, sizeof(int64_t) * (size_t)o->m, cudaMemcpyDeviceToHost, s);
    if (total) cudaMemcpyAsync(total, dcount, sizeof(int64_t), cudaMemcpyDefault, s);
    if (h_c) dev_free(dc, s);
    dev_free(dcount, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "masked product");
    return TC_OK;
}
