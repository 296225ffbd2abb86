// tc_labels.cu -- counting a labelled triangle by subgraph matching (Alg. 1,
// Sec. 3.1 "TC using Subgraph Matching").
//
// The query is a triangle whose vertices carry labels {l0, l1, l2}.  As in
// Alg. 1, candidate edges are filtered first: an edge {u, v} of the data
// graph is kept iff the unordered label pair {lab(u), lab(v)} is the label
// pair of some query edge (a vertex whose label is not in the query loses all
// its edges, the candidate-set pruning of Alg. 1).  The join is the
// set-intersection count on the filtered graph: every triangle left has
// three candidate edges.  When the query labels are all distinct or all
// equal, exactly the matching triangles survive.  For a query {a, a, b} the
// filtered graph also keeps triangles labelled {a, a, a} (all three edges are
// a-a pairs); they are counted on the a-a subgraph and subtracted.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

// bit (i, j) of the allowed-pair mask: the query has an edge labelled {q_i, q_j}
__device__ __forceinline__ bool pair_allowed(int a, int b, const int q[3], int npairs_mode) {
    // npairs_mode 0: all query edges; 1: only {q0, q0} pairs (the a-a subgraph)
    if (npairs_mode == 1) return a == q[0] && b == q[0];
    return (a == q[0] && b == q[1]) || (a == q[1] && b == q[0]) || (a == q[1] && b == q[2]) ||
           (a == q[2] && b == q[1]) || (a == q[0] && b == q[2]) || (a == q[2] && b == q[0]);
}

template <bool SCATTER>
__global__ void k_label_filter(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ lab, int q0, int q1, int q2, int mode,
                               int32_t* __restrict__ cnt, const int64_t* __restrict__ orp, int32_t* __restrict__ ocol) {
    const int q[3] = {q0, q1, q2};
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < n; u += nw) {
        const int64_t b = rp[u], e = rp[u + 1];
        const int lu = lab[u];
        int kept = 0;
        const int64_t out = SCATTER ? orp[u] : 0;
        for (int64_t i = b + lane; i - lane < e; i += 32) {
            bool keep = false;
            int32_t v = 0;
            if (i < e) {
                v = col[i];
                keep = pair_allowed(lu, lab[v], q, mode);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (SCATTER && keep) ocol[out + kept + __popc(bal & ((1u << lane) - 1u))] = v;
            kept += __popc(bal);
        }
        if (!SCATTER && lane == 0) cnt[u] = kept;
    }
}

// Filter to the candidate-edge CSR (device buffers owned here) and count it.
static tc_status filtered_count(tc_ctx* ctx, int64_t n, const int64_t* rp, const int32_t* col, const int32_t* lab,
                                const int q[3], int mode, unsigned long long* total, cudaStream_t s) {
    int32_t* cnt = nullptr;
    int64_t* orp = nullptr;
    int32_t* ocol = nullptr;
    void* stmp = nullptr;
    const size_t stb = scan_tmp_bytes(n);
    cudaError_t e = dev_alloc((void**)&cnt, sizeof(int32_t) * std::max<int64_t>(n, 1), s);
    if (e == cudaSuccess) e = dev_alloc((void**)&orp, sizeof(int64_t) * (n + 1), s);
    if (e == cudaSuccess) e = dev_alloc(&stmp, stb, s);
    if (e != cudaSuccess) {
        dev_free(cnt, s); dev_free(orp, s); dev_free(stmp, s);
        return set_err(ctx, TC_ERR_OOM, "labelled count: allocation failed");
    }
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, (int64_t)ctx->num_sms * 16));
    if (n > 0) k_label_filter<false><<<grid, 256, 0, s>>>(n, rp, col, lab, q[0], q[1], q[2], mode, cnt, nullptr, nullptr);
    scan_i32_to_i64(cnt, orp, n, stmp, stb, s);
    int64_t nnz = 0;
    cudaMemcpyAsync(&nnz, orp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ocol, sizeof(int32_t) * std::max<int64_t>(nnz, 1), s);
    if (e != cudaSuccess) {
        dev_free(cnt, s); dev_free(orp, s); dev_free(stmp, s);
        return cuda_err(ctx, e, "labelled count: filter");
    }
    if (n > 0) k_label_filter<true><<<grid, 256, 0, s>>>(n, rp, col, lab, q[0], q[1], q[2], mode, nullptr, orp, ocol);
    ctx->launches += 5;
    tc_ocsr* o = nullptr;
    tc_status st = build_from_device_csr(ctx, n, nnz, orp, ocol, nullptr, 0, false, &o, s);
    if (st == TC_OK) st = count_device(ctx, o, total, nullptr, s);
    if (o) tc_ocsr_release(o, s);
    dev_free(cnt, s); dev_free(orp, s); dev_free(ocol, s); dev_free(stmp, s);
    return st;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_count_labelled(tc_ctx* ctx, const tc_graph* g, const int32_t* labels, const int32_t* query,
                                       int64_t* total, void* stream) {
    if (!ctx || !g || !labels || !query || !total || !g->row_ptr || (g->flags & TC_IN_HOST))
        return set_err(ctx, TC_ERR_INVALID_ARG, "labelled count: device CSR, labels, query[3] and total required");
    if (g->n < 0 || g->n > 0x7fffffffLL || g->nnz < 0 || (g->nnz > 0 && !g->col))
        return set_err(ctx, TC_ERR_INVALID_ARG, "labelled count: bad sizes");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int q[3] = {query[0], query[1], query[2]};
    std::sort(q, q + 3);
    // {a, a, b} / {a, b, b}: the repeated label first, the other last
    int rep = -1;
    if (q[0] == q[1] && q[1] != q[2]) rep = q[0];
    else if (q[1] == q[2] && q[0] != q[1]) { rep = q[1]; std::swap(q[0], q[2]); }
    unsigned long long* dt = nullptr;
    cudaError_t e = dev_alloc((void**)&dt, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_err(ctx, TC_ERR_OOM, "labelled count: allocation failed");
    tc_status st = filtered_count(ctx, g->n, g->row_ptr, g->col, labels, q, 0, dt, s);
    if (st == TC_OK && rep >= 0) st = filtered_count(ctx, g->n, g->row_ptr, g->col, labels, q, 1, dt + 1, s);
    unsigned long long h[2] = {0, 0};
    if (st == TC_OK) {
        cudaMemcpyAsync(h, dt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_err(ctx, e, "labelled count");
    }
    dev_free(dt, s);
    if (st != TC_OK) return st;
    const int64_t T = (int64_t)h[0] - (rep >= 0 ? (int64_t)h[1] : 0);
    e = cudaMemcpy(total, &T, sizeof(int64_t), cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_err(ctx, e, "labelled count: result");
    return TC_OK;
}
