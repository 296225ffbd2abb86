// tc_api.cu -- the C ABI (include/tc.h): contexts, oriented-CSR handles,
// single-graph and batched counting, CUDA-graph batch plans.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "tc_internal.cuh"

namespace tc {

tc_status set_err(tc_ctx* ctx, tc_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

tc_status cuda_err(tc_ctx* ctx, cudaError_t e, const char* where) {
    cudaGetLastError();  // clear a sticky launch error so the context stays usable
    return set_err(ctx, e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    return cudaMallocAsync(p, std::max<size_t>(bytes, 16), s);
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

static cudaEvent_t get_event(tc_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// NVTX range names of the phases (host-side ranges around each phase's
// launches; a profiler that records NVTX shows them beside the kernels)
static const char* const kPhaseNames[kNumPhases] = {
    "tc.degree",        "tc.validate",   "tc.orient_count", "tc.orient_scan", "tc.orient_scatter", "tc.pivot_count",
    "tc.pivot_scan",    "tc.pivot_scatter", "tc.items",     "tc.count_small", "tc.count_warp",     "tc.count_cta",
    "tc.edge_sort",     "tc.count_init", "tc.rank",         "tc.row_sort",    "tc.count_merge",
    "tc.fused"};

PhaseScope::PhaseScope(tc_ctx* c_, int id_, cudaStream_t s_) : c(c_), id(id_), s(s_) {
    nvtxRangePushA(id >= 0 && id < kNumPhases ? kPhaseNames[id] : "tc.phase");
    if (c && c->trace) {
        a = get_event(c);
        cudaEventRecord(a, s);
    }
}

PhaseScope::~PhaseScope() {
    if (a) {
        cudaEvent_t b = get_event(c);
        cudaEventRecord(b, s);
        c->recs.push_back({id, a, b});
    }
    nvtxRangePop();
}

// Defaults, then TC_SMALL_MAX / TC_WARP_MAX / TC_TABLE_CAP / TC_PROBE /
// TC_CTA_THREADS / TC_CHUNK / ... from the environment, then non-zero fields of c.
static void apply_config(Tuning& t, const tc_config* c) {
    Tuning d;
    t = d;
    auto env = [](const char* name, int& field) {
        const char* v = std::getenv(name);
        if (v && *v) field = std::atoi(v);
    };
    env("TC_SMALL_MAX", t.small_max);
    env("TC_WARP_MAX", t.warp_max);
    env("TC_TABLE_CAP", t.table_cap);
    env("TC_PROBE", t.probe);
    env("TC_CTA_THREADS", t.cta_threads);
    env("TC_CHUNK", t.chunk);
    env("TC_BITMAP_BITS", t.bitmap_bits);
    env("TC_DIRECT_SPAN", t.direct_span);
    env("TC_MERGE_RATIO", t.merge_ratio);
    env("TC_MERGE_MAX", t.merge_max);
    env("TC_STAGE", t.stage);
    env("TC_SMALL_LANES", t.small_lanes);
    if (!c) return;
    if (c->small_max > 0) t.small_max = c->small_max;
    if (c->small_max < 0) t.small_max = 0;  // negative disables the thread-per-edge class
    if (c->warp_max > 0) t.warp_max = c->warp_max;
    if (c->table_cap > 0) t.table_cap = c->table_cap;
    if (c->probe > 0) t.probe = c->probe;
    if (c->cta_threads > 0) t.cta_threads = c->cta_threads;
    if (c->chunk > 0) t.chunk = c->chunk;
    if (c->bitmap_bits > 0) t.bitmap_bits = c->bitmap_bits;
    if (c->bitmap_bits < 0) t.bitmap_bits = 0;
    if (c->direct_span > 0) t.direct_span = c->direct_span;
    if (c->direct_span < 0) t.direct_span = 0;
    if (c->merge_ratio > 0) t.merge_ratio = c->merge_ratio;
    if (c->merge_ratio < 0) t.merge_ratio = 0;
    if (c->merge_max > 0) t.merge_max = c->merge_max;
    if (c->stage != 0) t.stage = c->stage > 0 ? 1 : 0;
    if (c->small_lanes > 0) t.small_lanes = c->small_lanes;
}

static bool config_ok(const Tuning& t) {
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    return t.small_max >= 0 && t.small_max <= 64 && t.warp_max >= 2 && t.warp_max <= 1024 &&
           pow2(t.table_cap) && t.table_cap >= 16 && t.table_cap <= 4096 &&
           (t.probe == 1 || t.probe == 2) && t.cta_threads >= 64 && t.cta_threads <= 1024 &&
           t.cta_threads % 32 == 0 && t.chunk >= 1 && t.chunk <= 32768 && t.bitmap_bits >= 0 &&
           t.bitmap_bits <= 262144 && t.bitmap_bits % 32 == 0 && t.direct_span >= 0 && t.direct_span <= 16384 &&
           (t.merge_ratio == 0 || (t.merge_ratio >= 100 && t.merge_ratio <= 1000000)) && t.merge_max >= 16 &&
           t.merge_max <= 4096 && t.stage >= 0 && t.stage <= 1 && pow2(t.small_lanes) && t.small_lanes <= 32;
}

static bool is_host_ptr(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Copy `bytes` of a host array into a fresh stream-ordered device buffer.
template <typename T>
static cudaError_t upload(const T* h, int64_t count, T** d, cudaStream_t s) {
    cudaError_t e = dev_alloc((void**)d, sizeof(T) * (size_t)std::max<int64_t>(count, 1), s);
    if (e != cudaSuccess) return e;
    if (count > 0) e = cudaMemcpyAsync(*d, h, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice, s);
    return e;
}

// Count with outputs anywhere: device outputs are written in place; host
// outputs go through device scratch, a copy back and a stream synchronise.
static tc_status count_any(tc_ctx* ctx, const tc_ocsr* o, int64_t* totals, int64_t nt, int64_t* pv,
                           cudaStream_t s, int shard = 0, int nshards = 1) {
    const bool h_tot = is_host_ptr(totals);
    const bool h_pv = pv && is_host_ptr(pv);
    if (!h_tot && !h_pv)
        return count_device(ctx, o, (unsigned long long*)totals, (unsigned long long*)pv, s, shard, nshards);
    unsigned long long* dt = (unsigned long long*)totals;
    unsigned long long* dpv = (unsigned long long*)pv;
    cudaError_t e = cudaSuccess;
    if (h_tot) e = dev_alloc((void**)&dt, sizeof(int64_t) * (size_t)nt, s);
    if (e == cudaSuccess && h_pv) e = dev_alloc((void**)&dpv, sizeof(int64_t) * (size_t)std::max<int64_t>(o->n, 1), s);
    if (e != cudaSuccess) {
        if (h_tot) dev_free(dt, s);
        return set_err(ctx, TC_ERR_OOM, "count: output scratch allocation failed");
    }
    tc_status st = count_device(ctx, o, dt, dpv, s, shard, nshards);
    if (st == TC_OK) {
        if (h_tot) cudaMemcpyAsync(totals, dt, sizeof(int64_t) * (size_t)nt, cudaMemcpyDeviceToHost, s);
        if (h_pv && o->n > 0) cudaMemcpyAsync(pv, dpv, sizeof(int64_t) * (size_t)o->n, cudaMemcpyDeviceToHost, s);
    }
    if (h_tot) dev_free(dt, s);
    if (h_pv) dev_free(dpv, s);
    unsigned bits = 0u;
    e = take_device_error(s, &bits);  // synchronises s
    if (st == TC_OK && e != cudaSuccess) st = cuda_err(ctx, e, "count: synchronise");
    if (st == TC_OK && bits)
        st = set_err(ctx, TC_ERR_DEVICE, "count: a device-side check failed (check word " + std::to_string(bits) + ")");
    return st;
}

static void release_ocsr(tc_ocsr* o, cudaStream_t s, bool async) {
    if (!o) return;
    void* ptrs[] = {o->rpp,  o->colp, o->dplus,      o->deg, o->rank,      o->perm, o->colr,     o->rspan,
                    o->prp, o->pcol, o->items_warp, o->items_cta, o->dc,   o->row_graph, o->medge, o->pdesc};
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o->device);
    for (void* p : ptrs) {
        if (!p) continue;
        if (async) cudaFreeAsync(p, s);
        else cudaFree(p);
    }
    cudaSetDevice(prev);
    delete o;
}

}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_ctx_create(int device, const tc_config* cfg, tc_ctx** out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    tc_ctx* c = new tc_ctx();
    c->device = device;
    apply_config(c->tun, cfg);
    if (!config_ok(c->tun)) {
        delete c;
        return TC_ERR_INVALID_ARG;
    }
    cudaSetDevice(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    // keep freed pool memory cached in this process (stream-ordered reuse)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return TC_OK;
}

void tc_ctx_destroy(tc_ctx* ctx) {
    if (!ctx) return;
    for (auto& r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
}

tc_status tc_ctx_set_trace(tc_ctx* ctx, int enable) {
    if (!ctx) return TC_ERR_INVALID_ARG;
    ctx->trace = enable != 0;
    return TC_OK;
}

tc_status tc_ctx_read_trace(tc_ctx* ctx, tc_trace* out) {
    if (!ctx || !out) return TC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->launches = ctx->launches;
    ctx->launches = 0;
    tc_status st = TC_OK;
    for (auto& r : ctx->recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) st = cuda_err(ctx, e, "read trace");
        if (r.phase >= 0 && r.phase < TC_TRACE_PHASES) {
            out->phase_ms[r.phase] += ms;
            out->phase_calls[r.phase] += 1;
        }
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->recs.clear();
    return st;
}

const char* tc_last_error(const tc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tc_status tc_ctx_set_config(tc_ctx* ctx, const tc_config* cfg) {
    if (!ctx) return TC_ERR_INVALID_ARG;
    Tuning t;
    apply_config(t, cfg);
    if (!config_ok(t)) return set_err(ctx, TC_ERR_INVALID_ARG, "tc_config out of range");
    ctx->tun = t;
    return TC_OK;
}

tc_status tc_ctx_get_config(const tc_ctx* ctx, tc_config* out) {
    if (!ctx || !out) return TC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->small_max = ctx->tun.small_max;
    out->warp_max = ctx->tun.warp_max;
    out->table_cap = ctx->tun.table_cap;
    out->probe = ctx->tun.probe;
    out->cta_threads = ctx->tun.cta_threads;
    out->chunk = ctx->tun.chunk;
    out->bitmap_bits = ctx->tun.bitmap_bits;
    out->direct_span = ctx->tun.direct_span;
    out->merge_ratio = ctx->tun.merge_ratio;
    out->merge_max = ctx->tun.merge_max;
    out->stage = ctx->tun.stage;
    out->small_lanes = ctx->tun.small_lanes;
    return TC_OK;
}

tc_status tc_build_oriented_csr(tc_ctx* ctx, const tc_graph* g, tc_ocsr** out, void* stream) {
    if (!ctx || !g || !out) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (g->n < 0 || g->n > 0x7fffffffLL || g->nnz < 0)
        return set_err(ctx, TC_ERR_INVALID_ARG, "n must be in [0, 2^31) and nnz >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    const bool host = (g->flags & TC_IN_HOST) != 0;
    const bool validate = (g->flags & TC_VALIDATE) != 0;
    if (g->row_ptr) {
        if (g->nnz > 0 && !g->col) return set_err(ctx, TC_ERR_INVALID_ARG, "col is NULL");
        if (g->nnz % 2) return set_err(ctx, TC_ERR_INVALID_GRAPH, "a symmetric CSR has an even number of entries");
        const int64_t* rp = g->row_ptr;
        const int32_t* col = g->col;
        int64_t* drp = nullptr;
        int32_t* dcol = nullptr;
        const int32_t* col_src = nullptr;
        if (host) {
            if (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->nnz)
                return set_err(ctx, TC_ERR_INVALID_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] must be nnz");
            cudaError_t e = upload(g->row_ptr, g->n + 1, &drp, s);
            // A pinned, mapped col (cudaHostAlloc, or registered and mapped)
            // is read by the orientation's first pass straight from host
            // memory, which leaves the device copy: the transfer (host to
            // device runs at the same rate either way) overlaps that pass
            // instead of preceding it.  Pageable memory, and validation
            // (which reads col before that pass), take the plain upload.
            if (e == cudaSuccess && g->nnz > 0 && !validate) {
                cudaPointerAttributes at;
                if (cudaPointerGetAttributes(&at, g->col) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                    at.devicePointer)
                    col_src = static_cast<const int32_t*>(at.devicePointer);
                else
                    cudaGetLastError();
            }
            if (e == cudaSuccess) {
                if (col_src) e = dev_alloc((void**)&dcol, sizeof(int32_t) * (size_t)g->nnz, s);
                else e = upload(g->col, g->nnz, &dcol, s);
            }
            if (e != cudaSuccess) {
                dev_free(drp, s);
                dev_free(dcol, s);
                return cuda_err(ctx, e, "upload");
            }
            rp = drp;
            col = dcol;
        }
        tc_status st = build_from_device_csr(ctx, g->n, g->nnz, rp, col, nullptr, 0, validate, out, s, col_src);
        dev_free(drp, s);
        dev_free(dcol, s);
        return st;
    }
    // edge list
    if (g->nnz > 0 && (!g->src || !g->dst)) return set_err(ctx, TC_ERR_INVALID_ARG, "src/dst is NULL");
    const int32_t* src = g->src;
    const int32_t* dst = g->dst;
    int32_t* dsrc = nullptr;
    int32_t* ddst = nullptr;
    if (host) {
        cudaError_t e = upload(g->src, g->nnz, &dsrc, s);
        if (e == cudaSuccess) e = upload(g->dst, g->nnz, &ddst, s);
        if (e != cudaSuccess) {
            dev_free(dsrc, s);
            dev_free(ddst, s);
            return cuda_err(ctx, e, "upload");
        }
        src = dsrc;
        dst = ddst;
    }
    int64_t* rp = nullptr;
    int32_t* col = nullptr;
    int64_t nnz = 0;
    tc_status st = edges_to_csr(ctx, g->n, g->nnz, src, dst, &rp, &col, &nnz, s);
    dev_free(dsrc, s);
    dev_free(ddst, s);
    if (st != TC_OK) return st;
    st = build_from_device_csr(ctx, g->n, nnz, rp, col, nullptr, 0, false, out, s);
    dev_free(rp, s);
    dev_free(col, s);
    return st;
}

tc_status tc_count(tc_ctx* ctx, const tc_ocsr* o, int64_t* total, int64_t* per_vertex, void* stream) {
    if (!ctx || !o || !total) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    if (o->G > 0) return set_err(ctx, TC_ERR_INVALID_ARG, "batch handle: use tc_count_batch");
    cudaSetDevice(o->device);
    return count_any(ctx, o, total, 1, per_vertex, (cudaStream_t)stream);
}

tc_status tc_count_shard(tc_ctx* ctx, const tc_ocsr* o, int32_t shard, int32_t nshards, int64_t* total,
                         int64_t* per_vertex, void* stream) {
    if (!ctx || !o || !total) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    if (nshards < 1 || shard < 0 || shard >= nshards)
        return set_err(ctx, TC_ERR_INVALID_ARG, "shard must be in [0, nshards)");
    if (o->G > 0) return set_err(ctx, TC_ERR_INVALID_ARG, "batch handle: use tc_count_batch");
    cudaSetDevice(o->device);
    return count_any(ctx, o, total, 1, per_vertex, (cudaStream_t)stream, shard, nshards);
}

tc_status tc_count_graph(tc_ctx* ctx, const tc_graph* g, int64_t* total, int64_t* per_vertex, void* stream) {
    if (!ctx || !g || !total) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    if (g->n < 0 || g->n > 0x7fffffffLL || g->nnz < 0)
        return set_err(ctx, TC_ERR_INVALID_ARG, "n must be in [0, 2^31) and nnz >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    const bool fused = g->row_ptr && !(g->flags & TC_VALIDATE) && g->nnz % 2 == 0 && fused_fits(g->n, g->nnz);
    if (!fused) {  // build, count, release the handle in stream order
        tc_ocsr* o = nullptr;
        tc_status st = tc_build_oriented_csr(ctx, g, &o, stream);
        if (st != TC_OK) return st;
        st = tc_count(ctx, o, total, per_vertex, stream);
        release_ocsr(o, s, true);
        return st;
    }
    if (g->nnz > 0 && !g->col) return set_err(ctx, TC_ERR_INVALID_ARG, "col is NULL");
    const int64_t n = g->n;
    const int64_t* rp = g->row_ptr;
    const int32_t* col = g->col;
    int64_t* drp = nullptr;
    int32_t* dcol = nullptr;
    cudaError_t e = cudaSuccess;
    if (g->flags & TC_IN_HOST) {
        if (g->row_ptr[0] != 0 || g->row_ptr[n] != g->nnz)
            return set_err(ctx, TC_ERR_INVALID_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] must be nnz");
        e = upload(g->row_ptr, n + 1, &drp, s);
        if (e == cudaSuccess) e = upload(g->col, g->nnz, &dcol, s);
        rp = drp;
        col = dcol;
    }
    const bool h_tot = is_host_ptr(total);
    const bool h_pv = per_vertex && is_host_ptr(per_vertex);
    unsigned long long* dt = (unsigned long long*)total;
    unsigned long long* dpv = (unsigned long long*)per_vertex;
    if (e == cudaSuccess && h_tot) e = dev_alloc((void**)&dt, sizeof(int64_t), s);
    if (e == cudaSuccess && h_pv) e = dev_alloc((void**)&dpv, sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1), s);
    if (e == cudaSuccess) {
        PhaseScope ph(ctx, kPhFused, s);
        e = launch_fused(n, g->nnz, rp, col, dt, dpv, s);
        TC_LAUNCH(ctx);
    }
    if (e == cudaSuccess && h_tot) e = cudaMemcpyAsync(total, dt, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_pv && n > 0)
        e = cudaMemcpyAsync(per_vertex, dpv, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (h_tot) dev_free(dt, s);
    if (h_pv) dev_free(dpv, s);
    dev_free(drp, s);
    dev_free(dcol, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "fused count");
    if (h_tot || h_pv) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "fused count: synchronise");
    }
    return TC_OK;
}

tc_status tc_ocsr_get_view(const tc_ocsr* o, tc_ocsr_view* out) {
    if (!o || !out) return TC_ERR_INVALID_ARG;
    out->n = o->n;
    out->m = o->m;
    out->row_ptr = o->rpp;
    out->col = o->colp;
    out->bytes = o->bytes;
    return TC_OK;
}

tc_status tc_ocsr_copy(const tc_ocsr* o, int64_t* row_ptr, int32_t* col, void* stream) {
    if (!o || !row_ptr || (!col && o->m > 0)) return TC_ERR_INVALID_ARG;
    cudaSetDevice(o->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(row_ptr, o->rpp, sizeof(int64_t) * (size_t)(o->n + 1), cudaMemcpyDefault, s);
    if (e == cudaSuccess && o->m > 0) e = cudaMemcpyAsync(col, o->colp, sizeof(int32_t) * (size_t)o->m, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    return TC_OK;
}

void tc_ocsr_free(tc_ocsr* o) { release_ocsr(o, nullptr, false); }

void tc_ocsr_release(tc_ocsr* o, void* stream) { release_ocsr(o, (cudaStream_t)stream, true); }

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct BatchDev {
    int64_t G = 0, n = 0, nnz = 0;
    const int64_t* vtx_off = nullptr;
    const int64_t* row_ptr = nullptr;
    const int32_t* col = nullptr;
    int64_t* own_vo = nullptr;
    int64_t* own_rp = nullptr;
    int32_t* own_col = nullptr;
};

static tc_status batch_to_device(tc_ctx* ctx, const tc_batch* b, BatchDev& d, cudaStream_t s) {
    if (!b || b->G < 1 || !b->vtx_off || !b->edge_off || !b->row_ptr)
        return set_err(ctx, TC_ERR_INVALID_ARG, "batch: G >= 1 and offset arrays required");
    d.G = b->G;
    const bool host = (b->flags & TC_IN_HOST) != 0;
    if (host) {
        d.n = b->vtx_off[b->G];
        d.nnz = b->edge_off[b->G];
    } else {
        cudaError_t e = cudaMemcpyAsync(&d.n, b->vtx_off + b->G, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&d.nnz, b->edge_off + b->G, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "batch: reading sizes");
    }
    if (d.n < 0 || d.n > 0x7fffffffLL || d.nnz < 0 || d.nnz % 2)
        return set_err(ctx, TC_ERR_INVALID_GRAPH, "batch: bad total sizes");
    if (d.nnz > 0 && !b->col) return set_err(ctx, TC_ERR_INVALID_ARG, "batch: col is NULL");
    if (host) {
        cudaError_t e = upload(b->vtx_off, b->G + 1, &d.own_vo, s);
        if (e == cudaSuccess) e = upload(b->row_ptr, d.n + 1, &d.own_rp, s);
        if (e == cudaSuccess) e = upload(b->col, d.nnz, &d.own_col, s);
        if (e != cudaSuccess) {
            dev_free(d.own_vo, s); dev_free(d.own_rp, s); dev_free(d.own_col, s);
            return cuda_err(ctx, e, "batch: upload");
        }
        d.vtx_off = d.own_vo;
        d.row_ptr = d.own_rp;
        d.col = d.own_col;
    } else {
        d.vtx_off = b->vtx_off;
        d.row_ptr = b->row_ptr;
        d.col = b->col;
    }
    return TC_OK;
}

static void batch_release(BatchDev& d, cudaStream_t s) {
    dev_free(d.own_vo, s);
    dev_free(d.own_rp, s);
    dev_free(d.own_col, s);
    d.own_vo = d.own_rp = nullptr;
    d.own_col = nullptr;
}

tc_status tc_count_batch(tc_ctx* ctx, const tc_batch* b, int64_t* totals, int64_t* per_vertex, void* stream) {
    if (!ctx || !b || !totals) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    BatchDev d;
    tc_status st = batch_to_device(ctx, b, d, s);
    if (st != TC_OK) return st;
    tc_ocsr* o = nullptr;
    st = build_from_device_csr(ctx, d.n, d.nnz, d.row_ptr, d.col, d.vtx_off, d.G, (b->flags & TC_VALIDATE) != 0, &o, s);
    batch_release(d, s);
    if (st != TC_OK) return st;
    st = count_any(ctx, o, totals, d.G, per_vertex, s);
    release_ocsr(o, s, true);
    return st;
}

}  // extern "C"

struct tc_batch_plan {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

tc_status tc_batch_plan_create(tc_ctx* ctx, const tc_batch* b, int64_t* totals, int64_t* per_vertex, void* stream,
                               tc_batch_plan** out) {
    if (!ctx || !b || !totals || !out) return set_err(ctx, TC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (b->flags & TC_IN_HOST) return set_err(ctx, TC_ERR_INVALID_ARG, "plan: inputs must be device memory");
    if (is_host_ptr(totals) || (per_vertex && is_host_ptr(per_vertex)))
        return set_err(ctx, TC_ERR_INVALID_ARG, "plan: outputs must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    BatchDev d;
    tc_status st = batch_to_device(ctx, b, d, s);  // reads the sizes (synchronises once)
    if (st != TC_OK) return st;
    // one eager pass validates (when asked) and warms up kernel attributes
    {
        tc_ocsr* o = nullptr;
        st = build_from_device_csr(ctx, d.n, d.nnz, d.row_ptr, d.col, d.vtx_off, d.G, (b->flags & TC_VALIDATE) != 0, &o, s);
        if (st != TC_OK) return st;
        st = count_device(ctx, o, (unsigned long long*)totals, (unsigned long long*)per_vertex, s);
        release_ocsr(o, s, true);
        if (st != TC_OK) return st;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "plan: eager pass");
    }
    // capture on a private stream (the legacy default stream cannot be captured)
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(ctx, e, "plan: capture stream");
    const bool trace_was = ctx->trace;
    ctx->trace = false;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        ctx->trace = trace_was;
        cudaStreamDestroy(cs);
        return cuda_err(ctx, e, "plan: begin capture");
    }
    tc_ocsr* o = nullptr;
    st = build_from_device_csr(ctx, d.n, d.nnz, d.row_ptr, d.col, d.vtx_off, d.G, false, &o, cs);
    if (st == TC_OK) st = count_device(ctx, o, (unsigned long long*)totals, (unsigned long long*)per_vertex, cs);
    if (o) release_ocsr(o, cs, true);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    ctx->trace = trace_was;
    cudaStreamDestroy(cs);
    if (st != TC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "plan: end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_err(ctx, e, "plan: instantiate");
    }
    tc_batch_plan* p = new tc_batch_plan();
    p->device = ctx->device;
    p->graph = graph;
    p->exec = exec;
    *out = p;
    return TC_OK;
}

tc_status tc_batch_plan_launch(tc_batch_plan* plan, void* stream) {
    if (!plan) return TC_ERR_INVALID_ARG;
    cudaSetDevice(plan->device);
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TC_ERR_CUDA;
    }
    return TC_OK;
}

void tc_batch_plan_destroy(tc_batch_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
}

}  // extern "C"
