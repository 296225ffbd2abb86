// tc_count.cu -- steps 3-4 of the method on the device: intersect N+(u) with
// N+(v) for every oriented edge and reduce to the total and t(v).
//
// Paper: Sec. 3.2 (the common neighbours w of an oriented edge (u, v) each
// close one triangle), Alg. 2 Compute_Intersection / Reduce, Sec. 4.2.2
// (TwoSmall: one thread per pair; TwoLarge: CTA-cooperative intersection of
// long lists), and the small x large kernel proposed in Sec. 5 (walk the
// shorter list, search the longer one).
//
// Three kernels share the work that the partition (tc_build.cu) cut:
//   k_count_small : one thread per source row u with d+(u) <= small_max;
//                   sorted merge of N+(u) with each short N+(v).
//   k_count_warp  : one warp per work item of a pivot with d+(p) <= warp_max;
//                   N+(p) goes into a warp-private shared-memory table.
//   k_count_cta   : one CTA per work item of a longer pivot list; the table
//                   (one segment of N+(p)) is shared by all warps of the CTA.
// In the table kernels every warp streams the lists of 32 partners q at a
// time, flattened into one coalesced sequence of (partner, element) pairs,
// and probes each element w of N+(q) in the table of N+(p).
//
// Per-vertex counts: triangle {p, q, w} with w in N+(p) and N+(q) is found
// exactly once.  w is a key of the pivot's table, so its count accumulates in
// the table slot and is flushed once per item; q gets one atomic per partner
// with a non-zero count; p one atomic per item.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {

struct CountArgs {
    const int64_t* rpp;
    const int32_t* colp;
    const int32_t* dp;
    const int64_t* prp;
    const int32_t* pcol;
    const Item* items;
    const unsigned long long* n_items;
    unsigned long long items_cap;   // allocated items (n_items never exceeds it; clamped anyway)
    unsigned int* queue;
    unsigned long long* totals;   // [G] (batch) or [1]
    unsigned long long* t;        // per-vertex counts or nullptr
    const int32_t* row_graph;     // batch: graph of each vertex, else nullptr
    int64_t n;
    int cap;                      // keys per table segment
    int small_max;
};

constexpr int kProbeHash = 1;
constexpr int kProbeBsearch = 2;

__device__ __forceinline__ unsigned hslot(int x, int logS) {
    return ((unsigned)x * 0x9E3779B1u) >> (32 - logS);
}

__device__ __forceinline__ void table_insert(int* keys, int logS, int x) {
    const unsigned mask = (1u << logS) - 1u;
    unsigned h = hslot(x, logS);
    while (true) {
        const int prev = atomicCAS(&keys[h], -1, x);
        if (prev == -1) return;
        h = (h + 1u) & mask;
    }
}

// slot of x, or -1
template <int PROBE>
__device__ __forceinline__ int table_find(const int* keys, int logS, int len, int x) {
    if (PROBE == kProbeHash) {
        const unsigned mask = (1u << logS) - 1u;
        unsigned h = hslot(x, logS);
        while (true) {
            const int k = keys[h];
            if (k == x) return (int)h;
            if (k == -1) return -1;
            h = (h + 1u) & mask;
        }
    } else {
        int lo = 0, hi = len;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keys[mid] < x) lo = mid + 1; else hi = mid;
        }
        return (lo < len && keys[lo] == x) ? lo : -1;
    }
}

__device__ __forceinline__ int warp_incl_scan_i(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One warp intersects the partners pb+first, pb+first+stride, ... (in groups
// of 32) with the table.  pcnt: this warp's 32 shared counters.
template <bool PV, int PROBE>
__device__ __forceinline__ unsigned long long warp_partners(const CountArgs& a, int* keys, int* cnts, int logS,
                                                            int len, int64_t pbase, int pb, int pe, int first,
                                                            int stride, int* pcnt) {
    const int lane = threadIdx.x & 31;
    unsigned long long acc = 0;
    for (int g0 = pb + first; g0 < pe; g0 += stride) {
        const int i = g0 + lane;
        const bool valid = i < pe;
        const int q = valid ? a.pcol[pbase + i] : 0;
        const int64_t qb = valid ? a.rpp[q] : 0;
        const int dq = valid ? a.dp[q] : 0;
        const int incl = warp_incl_scan_i(dq);
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - dq;
        pcnt[lane] = 0;
        __syncwarp();
        for (int k0 = 0; k0 < tot; k0 += 32) {
            const int k = k0 + lane;
            // owner partner j of flattened element k: the last lane with excl_j <= k
            int j = 0;
#pragma unroll
            for (int s = 16; s; s >>= 1) {
                const int ej = __shfl_sync(0xffffffffu, excl, j + s);
                if (ej <= k) j += s;
            }
            const int64_t qbj = __shfl_sync(0xffffffffu, qb, j);
            const int ej = __shfl_sync(0xffffffffu, excl, j);
            if (k < tot) {
                const int w = a.colp[qbj + (k - ej)];
                const int h = table_find<PROBE>(keys, logS, len, w);
                if (h >= 0) {
                    if (PV) atomicAdd(&cnts[h], 1);
                    atomicAdd(&pcnt[j], 1);
                }
            }
        }
        __syncwarp();
        const int c = pcnt[lane];
        if (valid && c) {
            acc += (unsigned long long)c;
            if (PV) atomicAdd(&a.t[q], (unsigned long long)c);
        }
        __syncwarp();
    }
    return acc;
}

// ---------------------------------------------------------------------------
// CTA-table kernel (persistent; items from a global queue)
// ---------------------------------------------------------------------------
template <bool PV, int PROBE>
__global__ void __launch_bounds__(1024) k_count_cta(CountArgs a) {
    extern __shared__ int smem[];
    int* keys = smem;
    int* cnts = smem + 2 * a.cap;
    __shared__ int s_pcnt[32][32];
    __shared__ unsigned s_item;
    __shared__ unsigned long long s_acc;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long n_items = min(*a.n_items, a.items_cap);
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(a.queue, 1u);
            s_acc = 0;
        }
        __syncthreads();
        const unsigned it = s_item;
        if (it >= n_items) break;
        const Item item = a.items[it];
        const int p = item.p;
        const int64_t lb = a.rpp[p] + (int64_t)item.seg * a.cap;
        const int len = (int)min((int64_t)a.cap, a.rpp[p + 1] - lb);
        int logS, S;
        if (PROBE == kProbeHash) {
            logS = max(5, 32 - __clz(2 * len - 1));
            S = 1 << logS;
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                keys[i] = -1;
                if (PV) cnts[i] = 0;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += blockDim.x) table_insert(keys, logS, a.colp[lb + i]);
        } else {
            logS = 0;
            S = len;
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                keys[i] = a.colp[lb + i];
                if (PV) cnts[i] = 0;
            }
        }
        __syncthreads();
        unsigned long long acc = warp_partners<PV, PROBE>(a, keys, cnts, logS, len, a.prp[p], item.pb, item.pe,
                                                          warp * 32, nw * 32, s_pcnt[warp]);
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) atomicAdd(&s_acc, acc);
        __syncthreads();
        if (PV) {
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                const int c = cnts[i];
                if (c) atomicAdd(&a.t[keys[i]], (unsigned long long)c);
            }
        }
        if (threadIdx.x == 0 && s_acc) {
            const int g = a.row_graph ? a.row_graph[p] : 0;
            atomicAdd(&a.totals[g], s_acc);
            if (PV) atomicAdd(&a.t[p], s_acc);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// warp-table kernel: each warp owns a table of 2*wcap slots
// ---------------------------------------------------------------------------
template <bool PV, int PROBE>
__global__ void __launch_bounds__(256) k_count_warp(CountArgs a, int wcap) {
    extern __shared__ int smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_warp = 4 * wcap + 32;
    int* keys = smem + warp * per_warp;
    int* cnts = keys + 2 * wcap;
    int* pcnt = cnts + 2 * wcap;
    const unsigned long long n_items = min(*a.n_items, a.items_cap);
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(a.queue, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const Item item = a.items[it];
        const int p = item.p;
        const int64_t lb = a.rpp[p];
        const int len = (int)(a.rpp[p + 1] - lb);
        int logS, S;
        if (PROBE == kProbeHash) {
            logS = max(5, 32 - __clz(2 * len - 1));
            S = 1 << logS;
            for (int i = lane; i < S; i += 32) {
                keys[i] = -1;
                if (PV) cnts[i] = 0;
            }
            __syncwarp();
            for (int i = lane; i < len; i += 32) table_insert(keys, logS, a.colp[lb + i]);
        } else {
            logS = 0;
            S = len;
            for (int i = lane; i < len; i += 32) {
                keys[i] = a.colp[lb + i];
                if (PV) cnts[i] = 0;
            }
        }
        __syncwarp();
        unsigned long long acc =
            warp_partners<PV, PROBE>(a, keys, cnts, logS, len, a.prp[p], item.pb, item.pe, 0, 32, pcnt);
        __syncwarp();
        if (PV) {
            for (int i = lane; i < S; i += 32) {
                const int c = cnts[i];
                if (c) atomicAdd(&a.t[keys[i]], (unsigned long long)c);
            }
        }
        acc = warp_sum_u64(acc);
        if (lane == 0 && acc) {
            const int g = a.row_graph ? a.row_graph[p] : 0;
            atomicAdd(&a.totals[g], acc);
            if (PV) atomicAdd(&a.t[p], acc);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// TwoSmall: one thread per source row, sorted merge of short lists
// ---------------------------------------------------------------------------
template <bool PV>
__global__ void __launch_bounds__(256) k_count_small(CountArgs a) {
    __shared__ unsigned long long s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    unsigned long long acc = 0;
    const int sm = a.small_max;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < a.n; u += (int64_t)gridDim.x * blockDim.x) {
        const int du = a.dp[u];
        if (du < 2 || du > sm) continue;
        const int64_t ub = a.rpp[u];
        unsigned long long cu = 0;
        for (int i = 0; i < du; ++i) {
            const int v = a.colp[ub + i];
            const int dv = a.dp[v];
            if (dv == 0 || dv > sm) continue;
            const int64_t vb = a.rpp[v];
            int x = 0, y = 0, c = 0;
            while (x < du && y < dv) {
                const int xa = a.colp[ub + x], yb = a.colp[vb + y];
                if (xa < yb) ++x;
                else if (xa > yb) ++y;
                else {
                    ++c;
                    if (PV) atomicAdd(&a.t[xa], 1ull);
                    ++x;
                    ++y;
                }
            }
            if (c) {
                cu += (unsigned long long)c;
                if (PV) atomicAdd(&a.t[v], (unsigned long long)c);
            }
        }
        if (cu) {
            if (PV) atomicAdd(&a.t[u], cu);
            if (a.row_graph) atomicAdd(&a.totals[a.row_graph[u]], cu);
            else acc += cu;
        }
    }
    if (!a.row_graph) {
        acc = warp_sum_u64(acc);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&s_acc, acc);
        __syncthreads();
        if (threadIdx.x == 0 && s_acc) atomicAdd(&a.totals[0], s_acc);
    }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
static int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <bool PV, int PROBE>
static cudaError_t launch_tables(tc_ctx* ctx, const CountArgs& base, const tc_ocsr* o, unsigned* queues, int num_sms,
                                 const Tuning& tun, cudaStream_t s) {
    // warp-table items
    {
        PhaseScope ph(ctx, kPhCountWarp, s);
        TC_LAUNCH(ctx);
        CountArgs a = base;
        a.items = o->items_warp;
        a.n_items = &o->dc->n_items_warp;
        a.items_cap = (unsigned long long)o->items_warp_cap;
        a.queue = queues + 0;
        const int wcap = std::max(16, pow2ceil(tun.warp_max));
        const size_t smem = (size_t)8 * (4 * wcap + 32) * sizeof(int);
        auto kern = k_count_warp<PV, PROBE>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        kern<<<(unsigned)(num_sms * std::max(per_sm, 1)), 256, smem, s>>>(a, wcap);
    }
    // CTA-table items
    {
        PhaseScope ph(ctx, kPhCountCta, s);
        TC_LAUNCH(ctx);
        CountArgs a = base;
        a.items = o->items_cta;
        a.n_items = &o->dc->n_items_cta;
        a.items_cap = (unsigned long long)o->items_cta_cap;
        a.queue = queues + 1;
        const size_t smem = (size_t)4 * a.cap * sizeof(int);
        auto kern = k_count_cta<PV, PROBE>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tun.cta_threads, smem);
        kern<<<(unsigned)(num_sms * std::max(per_sm, 1)), tun.cta_threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

tc_status count_device(tc_ctx* ctx, const tc_ocsr* o, unsigned long long* totals, unsigned long long* per_vertex,
                       cudaStream_t s) {
    const Tuning& tun = o->tun;
    const int64_t G = o->G > 0 ? o->G : 1;
    unsigned* queues = nullptr;
    {
        PhaseScope ph(ctx, kPhCountInit, s);
        cudaError_t e = cudaMemsetAsync(totals, 0, sizeof(unsigned long long) * G, s);
        if (e == cudaSuccess && per_vertex && o->n > 0)
            e = cudaMemsetAsync(per_vertex, 0, sizeof(unsigned long long) * o->n, s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "count: memset");
        if (o->n == 0 || o->m == 0) return TC_OK;
        e = dev_alloc((void**)&queues, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return set_err(ctx, TC_ERR_OOM, "count: queue allocation failed");
        cudaMemsetAsync(queues, 0, 2 * sizeof(unsigned), s);
    }
    cudaError_t e = cudaSuccess;

    CountArgs a{};
    a.rpp = o->rpp;
    a.colp = o->colp;
    a.dp = o->dplus;
    a.prp = o->prp;
    a.pcol = o->pcol;
    a.totals = totals;
    a.t = per_vertex;
    a.row_graph = o->row_graph;
    a.n = o->n;
    a.cap = tun.table_cap;
    a.small_max = tun.small_max;
    const int ns = ctx->num_sms;

    if (tun.small_max >= 2) {
        PhaseScope ph(ctx, kPhCountSmall, s);
        TC_LAUNCH(ctx);
        int per_sm = 0;
        if (per_vertex) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_small<true>, 256, 0);
            k_count_small<true><<<(unsigned)(ns * std::max(per_sm, 1)), 256, 0, s>>>(a);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_small<false>, 256, 0);
            k_count_small<false><<<(unsigned)(ns * std::max(per_sm, 1)), 256, 0, s>>>(a);
        }
    }
    if (tun.probe == kProbeBsearch) {
        e = per_vertex ? launch_tables<true, kProbeBsearch>(ctx, a, o, queues, ns, tun, s)
                       : launch_tables<false, kProbeBsearch>(ctx, a, o, queues, ns, tun, s);
    } else {
        e = per_vertex ? launch_tables<true, kProbeHash>(ctx, a, o, queues, ns, tun, s)
                       : launch_tables<false, kProbeHash>(ctx, a, o, queues, ns, tun, s);
    }
    dev_free(queues, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "count kernels");
    return TC_OK;
}

}  // namespace tc
