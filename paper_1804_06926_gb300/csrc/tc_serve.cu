// tc_serve.cu -- continuous-batching request loop for count requests.
//
// No counterpart in the paper (it counts one graph per run); each request is
// the paper's problem (Sec. 3) solved by the same build + count path.
//
// One request thread owns `slots` CUDA streams.  It admits queued requests in
// arrival order whenever a slot is free and the HBM budget holds the resident
// oriented CSRs plus every in-flight request's estimate; it retires a request
// when the slot's completion event has fired.  Requests on different slots
// overlap on the device.  Small requests waiting together at the head of the
// queue are fused: their CSRs are concatenated (vertex offsets + local ids)
// and run through the batched build + count of tc_count_batch on one slot, so
// one launch sequence serves them all; each request still receives its own
// exact total and per-vertex counts.  Oriented CSRs built for a non-zero
// graph_key stay resident (LRU eviction under the budget) so a repeated key
// skips the build.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tc_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    uint64_t key = 0;
    int64_t n = 0, nnz = 0;
    uint32_t flags = 0;
    bool csr = true;
    // pinned host copies of the inputs
    int64_t* h_rp = nullptr;
    int32_t* h_a = nullptr;  // col, or src
    int32_t* h_b = nullptr;  // dst (edge list)
    int64_t est_bytes = 0;
    Clock::time_point t_submit, t_admit, t_done;
    // results (pinned host)
    int64_t* h_total = nullptr;
    int64_t* h_pv = nullptr;
    std::vector<int64_t> pv;
    int64_t total = 0;
    tc_status status = TC_PENDING;
    bool cache_hit = false;
    bool done = false;
};

// A fused batch of small requests on one slot: pinned offsets and outputs,
// and device outputs (stream-ordered allocations).  The requests' own pinned
// inputs are copied straight into the concatenated device arrays.
struct BatchJob {
    std::vector<Request*> reqs;
    int64_t G = 0, N = 0, NNZ = 0;
    int64_t* h_off = nullptr;    // [2(G+1)]: vertex offsets, then edge offsets
    int64_t* h_tot = nullptr;
    int64_t* h_pv = nullptr;
    unsigned long long* d_tot = nullptr;
    unsigned long long* d_pv = nullptr;
};

// The row offsets of graph g were copied as its own (starting at 0): shift
// them by the graph's first edge, and close the concatenated array.
__global__ void k_shift_rows(int64_t G, const int64_t* __restrict__ off, int64_t* __restrict__ rp) {
    const int64_t* vo = off;
    const int64_t* eo = off + G + 1;
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x)
        for (int64_t v = vo[g] + threadIdx.x; v < vo[g + 1]; v += blockDim.x) rp[v] += eo[g];
    if (blockIdx.x == 0 && threadIdx.x == 0) rp[vo[G]] = eo[G];
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Request* req = nullptr;
    BatchJob job;                // job.reqs non-empty: the slot runs a fused batch
    tc_ocsr* o = nullptr;
    bool o_cached = false;       // o belongs to the resident cache
    unsigned long long* d_total = nullptr;
    unsigned long long* d_pv = nullptr;
    int64_t d_pv_cap = 0;
    unsigned* h_err = nullptr;   // pinned copy of the device check word, read at retire
};

struct CacheEntry {
    tc_ocsr* o = nullptr;
    int64_t bytes = 0;
    int in_use = 0;
    std::list<uint64_t>::iterator lru_it;
};

int64_t estimate_bytes(int64_t n, int64_t nnz, const tc::Tuning& t) {
    const int64_t m = nnz / 2;
    const int64_t dmax = std::max<int64_t>(1, (int64_t)std::sqrt((double)(2 * m)) + 1);
    const int64_t iw = std::min(n, m) + m / t.chunk + 2;
    const int64_t ic = dmax * m / ((int64_t)t.table_cap * t.chunk) + m / t.table_cap + m / t.chunk + m / (t.warp_max + 1) + 6;
    const int64_t ocsr = 16 * (n + 1) + 4 * (5 * m + 9 * n) + 16 * (iw + ic) + (t.merge_ratio > 0 ? 8 * m : 0);
    const int64_t input = 8 * (n + 1) + 4 * nnz;
    const int64_t scratch = 8 * n + 64 * 1024 + 8 * (n + 1);  // deg, pc, scan tiles, outputs
    return ocsr + input + scratch + (1 << 20);
}

}  // namespace

struct tc_server {
    tc_server_config cfg{};
    tc_ctx* ctx = nullptr;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    std::unordered_map<uint64_t, CacheEntry> cache;
    std::list<uint64_t> lru;  // front = most recent
    int64_t resident = 0, inflight = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    tc_server_stats stats{};
    // pinned staging buffers, reused by size class
    std::multimap<size_t, void*> pinned_free;
    std::mutex pin_mu;

    void* pin_alloc(size_t bytes) {
        size_t cls = 4096;
        while (cls < bytes) cls <<= 1;
        {
            std::lock_guard<std::mutex> g(pin_mu);
            auto it = pinned_free.find(cls);
            if (it != pinned_free.end()) {
                void* p = it->second;
                pinned_free.erase(it);
                return p;
            }
        }
        void* p = nullptr;
        if (cudaHostAlloc(&p, cls, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void pin_free(void* p, size_t bytes) {
        if (!p) return;
        size_t cls = 4096;
        while (cls < bytes) cls <<= 1;
        std::lock_guard<std::mutex> g(pin_mu);
        pinned_free.emplace(cls, p);
    }
    void free_inputs(Request* r) {
        if (r->csr) {
            pin_free(r->h_rp, sizeof(int64_t) * (r->n + 1));
            pin_free(r->h_a, sizeof(int32_t) * std::max<int64_t>(r->nnz, 1));
        } else {
            pin_free(r->h_a, sizeof(int32_t) * std::max<int64_t>(r->nnz, 1));
            pin_free(r->h_b, sizeof(int32_t) * std::max<int64_t>(r->nnz, 1));
        }
        r->h_rp = nullptr;
        r->h_a = r->h_b = nullptr;
    }

    void evict_until(int64_t need) {
        // drop least-recently-used resident oriented CSRs not in use
        auto it = lru.end();
        while (resident + inflight + need > cfg.hbm_budget_bytes && it != lru.begin()) {
            --it;
            auto ce = cache.find(*it);
            if (ce == cache.end() || ce->second.in_use) continue;
            tc_ocsr_release(ce->second.o, slots[0].stream);  // stream-ordered; slot 0 is idle or ordered after
            resident -= ce->second.bytes;
            stats.evictions++;
            cache.erase(ce);
            it = lru.erase(it);
        }
    }

    void finish(Request* r, tc_status st) {
        r->status = st;
        r->t_done = Clock::now();
        r->done = true;
        stats.finished++;
    }

    bool launch(Slot& sl, Request* r) {
        cudaStream_t s = sl.stream;
        tc_ctx* c = ctx;
        tc_ocsr* o = nullptr;
        bool hit = false;
        if (r->key) {
            auto ce = cache.find(r->key);
            if (ce != cache.end()) {
                o = ce->second.o;
                ce->second.in_use++;
                lru.erase(ce->second.lru_it);
                lru.push_front(r->key);
                ce->second.lru_it = lru.begin();
                hit = true;
            }
        }
        tc_status st = TC_OK;
        if (!o) {
            // blocks that evictions released on slot 0's stream are reused here only
            // after that release: the stream-ordered pool tracks the dependency
            tc_graph g{};
            g.n = r->n;
            g.nnz = r->nnz;
            g.flags = TC_IN_HOST | (r->flags & TC_VALIDATE);
            if (r->csr) { g.row_ptr = r->h_rp; g.col = r->h_a; }
            else { g.src = r->h_a; g.dst = r->h_b; }
            st = tc_build_oriented_csr(c, &g, &o, s);
        }
        if (st == TC_OK) {
            if (sl.d_pv_cap < r->n && cfg.per_vertex) {
                if (sl.d_pv) cudaFreeAsync(sl.d_pv, s);
                sl.d_pv = nullptr;
                sl.d_pv_cap = 0;
                if (cudaMallocAsync((void**)&sl.d_pv, sizeof(int64_t) * std::max<int64_t>(r->n, 1), s) == cudaSuccess)
                    sl.d_pv_cap = r->n;
                else st = TC_ERR_OOM;
            }
        }
        if (st == TC_OK) st = tc::count_device(c, o, sl.d_total, cfg.per_vertex ? sl.d_pv : nullptr, s);
        if (st == TC_OK) {
            cudaMemcpyAsync(r->h_total, sl.d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (cfg.per_vertex && r->n > 0)
                cudaMemcpyAsync(r->h_pv, sl.d_pv, sizeof(int64_t) * r->n, cudaMemcpyDeviceToHost, s);
            tc::peek_device_error_async(sl.h_err, s);
            cudaEventRecord(sl.ev, s);
        }
        if (st != TC_OK) {
            if (o && !hit) tc_ocsr_release(o, s);
            if (hit) cache[r->key].in_use--;
            inflight -= r->est_bytes;
            free_inputs(r);
            finish(r, st);
            return false;
        }
        sl.req = r;
        sl.o = o;
        sl.o_cached = hit;
        r->cache_hit = hit;
        if (hit) stats.cache_hits++;
        return true;
    }

    bool fusable(const Request* r) const {
        // small in edges and in vertices (a fused batch stays far below 2^31 vertices)
        return r->csr && !(r->flags & TC_VALIDATE) && r->nnz <= cfg.batch_nnz && r->n <= cfg.batch_nnz &&
               r->h_rp[0] == 0 && r->h_rp[r->n] == r->nnz;
    }

    void free_job(BatchJob& b, cudaStream_t s) {
        pin_free(b.h_off, sizeof(int64_t) * 2 * (b.G + 1));
        pin_free(b.h_tot, sizeof(int64_t) * std::max<int64_t>(b.G, 1));
        if (b.h_pv) pin_free(b.h_pv, sizeof(int64_t) * std::max<int64_t>(b.N, 1));
        tc::dev_free(b.d_tot, s);
        tc::dev_free(b.d_pv, s);
        b = BatchJob();
    }

    // Concatenate the requests' CSRs on the device and run the batched build + count.
    bool launch_batch(Slot& sl, std::vector<Request*>& B) {
        cudaStream_t s = sl.stream;
        BatchJob& b = sl.job;
        b.G = (int64_t)B.size();
        for (Request* r : B) {
            b.N += r->n;
            b.NNZ += r->nnz;
        }
        b.h_off = (int64_t*)pin_alloc(sizeof(int64_t) * 2 * (b.G + 1));
        b.h_tot = (int64_t*)pin_alloc(sizeof(int64_t) * std::max<int64_t>(b.G, 1));
        if (cfg.per_vertex) b.h_pv = (int64_t*)pin_alloc(sizeof(int64_t) * std::max<int64_t>(b.N, 1));
        tc_status st = (b.h_off && b.h_tot && (!cfg.per_vertex || b.h_pv)) ? TC_OK : TC_ERR_OOM;
        int64_t *d_off = nullptr, *d_rp = nullptr;
        int32_t* d_col = nullptr;
        tc_ocsr* o = nullptr;
        if (st == TC_OK) {
            int64_t* vo = b.h_off;
            int64_t* eo = b.h_off + b.G + 1;
            vo[0] = eo[0] = 0;
            for (int64_t i = 0; i < b.G; ++i) {
                vo[i + 1] = vo[i] + B[i]->n;
                eo[i + 1] = eo[i] + B[i]->nnz;
            }
            cudaError_t e = tc::dev_alloc((void**)&d_off, sizeof(int64_t) * 2 * (b.G + 1), s);
            if (e == cudaSuccess) e = tc::dev_alloc((void**)&d_rp, sizeof(int64_t) * (b.N + 1), s);
            if (e == cudaSuccess) e = tc::dev_alloc((void**)&d_col, sizeof(int32_t) * std::max<int64_t>(b.NNZ, 1), s);
            if (e == cudaSuccess) e = tc::dev_alloc((void**)&b.d_tot, sizeof(int64_t) * b.G, s);
            if (e == cudaSuccess && cfg.per_vertex)
                e = tc::dev_alloc((void**)&b.d_pv, sizeof(int64_t) * std::max<int64_t>(b.N, 1), s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_off, b.h_off, sizeof(int64_t) * 2 * (b.G + 1), cudaMemcpyHostToDevice, s);
            for (int64_t i = 0; i < b.G && e == cudaSuccess; ++i) {
                const Request* r = B[i];
                if (r->n) e = cudaMemcpyAsync(d_rp + vo[i], r->h_rp, sizeof(int64_t) * r->n, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess && r->nnz)
                    e = cudaMemcpyAsync(d_col + eo[i], r->h_a, sizeof(int32_t) * r->nnz, cudaMemcpyHostToDevice, s);
            }
            if (e == cudaSuccess) {
                k_shift_rows<<<(unsigned)std::min<int64_t>(b.G, 1024), 256, 0, s>>>(b.G, d_off, d_rp);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) st = TC_ERR_OOM;
        }
        int64_t* d_vo = d_off;  // the vertex offsets lead the offset array
        if (st == TC_OK) st = tc::build_from_device_csr(ctx, b.N, b.NNZ, d_rp, d_col, d_vo, b.G, false, &o, s);
        tc::dev_free(d_off, s);
        tc::dev_free(d_rp, s);
        tc::dev_free(d_col, s);
        if (st == TC_OK) st = tc::count_device(ctx, o, b.d_tot, cfg.per_vertex ? b.d_pv : nullptr, s);
        if (st == TC_OK) {
            cudaMemcpyAsync(b.h_tot, b.d_tot, sizeof(int64_t) * b.G, cudaMemcpyDeviceToHost, s);
            if (cfg.per_vertex && b.N > 0)
                cudaMemcpyAsync(b.h_pv, b.d_pv, sizeof(int64_t) * b.N, cudaMemcpyDeviceToHost, s);
            tc::peek_device_error_async(sl.h_err, s);
            cudaEventRecord(sl.ev, s);
        }
        if (st != TC_OK) {
            if (o) tc_ocsr_release(o, s);
            free_job(b, s);
            for (Request* r : B) {
                inflight -= r->est_bytes;
                free_inputs(r);
                finish(r, st);
            }
            return false;
        }
        b.reqs = B;
        sl.o = o;
        stats.batches++;
        stats.batched_requests += b.G;
        return true;
    }

    void retire_batch(Slot& sl) {
        BatchJob& b = sl.job;
        for (int64_t i = 0; i < b.G; ++i) {
            Request* r = b.reqs[i];
            r->total = b.h_tot[i];
            if (cfg.per_vertex) r->pv.assign(b.h_pv + b.h_off[i], b.h_pv + b.h_off[i + 1]);
            pin_free(r->h_total, sizeof(int64_t));
            if (r->h_pv) pin_free(r->h_pv, sizeof(int64_t) * std::max<int64_t>(r->n, 1));
            r->h_total = nullptr;
            r->h_pv = nullptr;
            free_inputs(r);
            inflight -= r->est_bytes;
            finish(r, *sl.h_err ? TC_ERR_DEVICE : TC_OK);
        }
        tc_ocsr_release(sl.o, sl.stream);
        sl.o = nullptr;
        free_job(b, sl.stream);
    }

    void retire(Slot& sl) {
        Request* r = sl.req;
        r->total = *r->h_total;
        if (cfg.per_vertex) r->pv.assign(r->h_pv, r->h_pv + r->n);
        pin_free(r->h_total, sizeof(int64_t));
        if (r->h_pv) pin_free(r->h_pv, sizeof(int64_t) * std::max<int64_t>(r->n, 1));
        r->h_total = nullptr;
        r->h_pv = nullptr;
        free_inputs(r);
        inflight -= r->est_bytes;
        if (sl.o_cached) {
            cache[r->key].in_use--;
        } else if (r->key && !cache.count(r->key)) {
            CacheEntry ce;
            ce.o = sl.o;
            tc_ocsr_view v;
            tc_ocsr_get_view(sl.o, &v);
            ce.bytes = v.bytes;
            lru.push_front(r->key);
            ce.lru_it = lru.begin();
            cache[r->key] = ce;
            resident += ce.bytes;
        } else {
            tc_ocsr_release(sl.o, sl.stream);
        }
        sl.req = nullptr;
        sl.o = nullptr;
        finish(r, *sl.h_err ? TC_ERR_DEVICE : TC_OK);
    }

    void loop() {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progressed = false;
            for (auto& sl : slots) {
                const bool busy = sl.req || !sl.job.reqs.empty();
                if (busy && cudaEventQuery(sl.ev) == cudaSuccess) {
                    if (sl.req) retire(sl);
                    else retire_batch(sl);
                    progressed = true;
                }
            }
            // admit in arrival order
            while (!queue.empty()) {
                Slot* free_slot = nullptr;
                for (auto& sl : slots)
                    if (!sl.req && sl.job.reqs.empty()) { free_slot = &sl; break; }
                if (!free_slot) break;
                Request* r = queue.front();
                const bool hit = r->key && cache.count(r->key);
                // fuse the small requests waiting together at the head of the queue
                if (!hit && cfg.batch_graphs > 1 && queue.size() >= 2 && fusable(r)) {
                    std::vector<Request*> B;
                    int64_t need = 0, nnz = 0, nv = 0;
                    for (Request* q : queue) {
                        if ((int)B.size() >= cfg.batch_graphs || !fusable(q) || (q->key && cache.count(q->key)) ||
                            nnz + q->nnz > 8 * cfg.batch_nnz || nv + q->n > (int64_t(1) << 30))
                            break;
                        B.push_back(q);
                        need += q->est_bytes;
                        nnz += q->nnz;
                        nv += q->n;
                    }
                    if (B.size() >= 2) {
                        if (resident + inflight + need > cfg.hbm_budget_bytes) evict_until(need);
                        if (resident + inflight + need <= cfg.hbm_budget_bytes) {
                            const auto now = Clock::now();
                            for (Request* q : B) {
                                queue.pop_front();
                                q->t_admit = now;
                            }
                            inflight += need;
                            stats.admitted += (int64_t)B.size();
                            stats.peak_inflight_bytes = std::max(stats.peak_inflight_bytes, inflight);
                            launch_batch(*free_slot, B);
                            int busy = 0;
                            for (auto& sl : slots) busy += (sl.req || !sl.job.reqs.empty()) ? 1 : 0;
                            stats.peak_inflight = std::max(stats.peak_inflight, busy);
                            progressed = true;
                            continue;
                        }
                    }
                }
                const int64_t need = hit ? 0 : r->est_bytes;
                if (resident + inflight + need > cfg.hbm_budget_bytes) evict_until(need);
                if (resident + inflight + need > cfg.hbm_budget_bytes) {
                    if (inflight == 0 && need > cfg.hbm_budget_bytes) {
                        queue.pop_front();
                        free_inputs(r);
                        finish(r, TC_ERR_BUDGET);
                        progressed = true;
                        continue;
                    }
                    break;  // wait for in-flight work to retire
                }
                queue.pop_front();
                r->est_bytes = need;
                r->t_admit = Clock::now();
                inflight += need;
                stats.admitted++;
                stats.peak_inflight_bytes = std::max(stats.peak_inflight_bytes, inflight);
                launch(*free_slot, r);
                int busy = 0;
                for (auto& sl : slots) busy += (sl.req || !sl.job.reqs.empty()) ? 1 : 0;
                stats.peak_inflight = std::max(stats.peak_inflight, busy);
                progressed = true;
            }
            stats.resident_bytes = resident;
            if (progressed) cv_done.notify_all();
            bool any_busy = false;
            for (auto& sl : slots) any_busy |= sl.req != nullptr || !sl.job.reqs.empty();
            if (stop && queue.empty() && !any_busy) break;
            if (!progressed) {
                if (any_busy) cv_work.wait_for(lk, std::chrono::microseconds(20));
                else cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
};

extern "C" {

tc_status tc_server_create(const tc_server_config* cfg, const tc_config* tuning, tc_server** out) {
    if (!out) return TC_ERR_INVALID_ARG;
    *out = nullptr;
    tc_server* s = new tc_server();
    if (cfg) s->cfg = *cfg;
    if (s->cfg.slots <= 0) s->cfg.slots = 8;
    if (s->cfg.slots > 64) s->cfg.slots = 64;
    if (s->cfg.hbm_budget_bytes <= 0) s->cfg.hbm_budget_bytes = 40ll << 30;
    if (s->cfg.batch_graphs <= 0) s->cfg.batch_graphs = 32;
    if (s->cfg.batch_nnz <= 0) s->cfg.batch_nnz = 1ll << 20;
    tc_status st = tc_ctx_create(s->cfg.device, tuning, &s->ctx);
    if (st != TC_OK) {
        delete s;
        return st;
    }
    cudaSetDevice(s->cfg.device);
    s->slots.resize(s->cfg.slots);
    for (auto& sl : s->slots) {
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        cudaMalloc((void**)&sl.d_total, sizeof(int64_t));
        if (cudaHostAlloc((void**)&sl.h_err, sizeof(unsigned), cudaHostAllocPortable) == cudaSuccess) *sl.h_err = 0u;
    }
    bool pinned = true;
    for (auto& sl : s->slots) pinned = pinned && sl.h_err;
    if (cudaGetLastError() != cudaSuccess || !pinned) {
        tc_server_destroy(s);
        return TC_ERR_CUDA;
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return TC_OK;
}

void tc_server_destroy(tc_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->cfg.device);
    cudaDeviceSynchronize();
    for (auto& kv : s->cache) tc_ocsr_free(kv.second.o);
    for (auto& sl : s->slots) {
        if (sl.d_total) cudaFree(sl.d_total);
        if (sl.d_pv) cudaFree(sl.d_pv);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.h_err) cudaFreeHost(sl.h_err);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : s->reqs) {
        s->free_inputs(kv.second);
        delete kv.second;
    }
    for (auto& kv : s->pinned_free) cudaFreeHost(kv.second);
    if (s->ctx) tc_ctx_destroy(s->ctx);
    delete s;
}

tc_status tc_submit(tc_server* s, const tc_graph* g, uint64_t graph_key, uint64_t* ticket) {
    if (!s || !g || !ticket) return TC_ERR_INVALID_ARG;
    if (g->n < 0 || g->n > 0x7fffffffLL || g->nnz < 0) return TC_ERR_INVALID_ARG;
    Request* r = new Request();
    r->key = graph_key;
    r->n = g->n;
    r->nnz = g->nnz;
    r->flags = g->flags;
    r->csr = g->row_ptr != nullptr;
    r->t_submit = Clock::now();
    bool ok = true;
    if (r->csr) {
        if (g->nnz > 0 && !g->col) ok = false;
        r->h_rp = (int64_t*)s->pin_alloc(sizeof(int64_t) * (g->n + 1));
        r->h_a = (int32_t*)s->pin_alloc(sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
        ok = ok && r->h_rp && r->h_a;
        if (ok) {
            std::memcpy(r->h_rp, g->row_ptr, sizeof(int64_t) * (g->n + 1));
            if (g->nnz) std::memcpy(r->h_a, g->col, sizeof(int32_t) * g->nnz);
        }
    } else {
        if (g->nnz > 0 && (!g->src || !g->dst)) ok = false;
        r->h_a = (int32_t*)s->pin_alloc(sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
        r->h_b = (int32_t*)s->pin_alloc(sizeof(int32_t) * std::max<int64_t>(g->nnz, 1));
        ok = ok && r->h_a && r->h_b;
        if (ok && g->nnz) {
            std::memcpy(r->h_a, g->src, sizeof(int32_t) * g->nnz);
            std::memcpy(r->h_b, g->dst, sizeof(int32_t) * g->nnz);
        }
    }
    r->h_total = (int64_t*)s->pin_alloc(sizeof(int64_t));
    if (s->cfg.per_vertex) r->h_pv = (int64_t*)s->pin_alloc(sizeof(int64_t) * std::max<int64_t>(g->n, 1));
    ok = ok && r->h_total && (!s->cfg.per_vertex || r->h_pv);
    if (!ok) {
        s->free_inputs(r);
        if (r->h_total) s->pin_free(r->h_total, sizeof(int64_t));
        if (r->h_pv) s->pin_free(r->h_pv, sizeof(int64_t) * std::max<int64_t>(g->n, 1));
        delete r;
        return TC_ERR_INVALID_ARG;
    }
    // edge lists are estimated as CSRs of twice the pair count
    r->est_bytes = estimate_bytes(r->n, r->csr ? r->nnz : 2 * r->nnz, s->ctx->tun) + (r->csr ? 0 : 24 * r->nnz);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        s->stats.submitted++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return TC_OK;
}

static void fill_result(const Request* r, tc_result* out) {
    out->status = r->status;
    out->total = r->total;
    out->n = r->n;
    out->per_vertex = r->pv.empty() ? nullptr : r->pv.data();
    out->submit_to_done_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    out->queue_ms = r->status == TC_ERR_BUDGET ? out->submit_to_done_ms
                                               : std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
    out->cache_hit = r->cache_hit ? 1 : 0;
}

tc_status tc_poll(tc_server* s, uint64_t ticket, tc_result* out) {
    if (!s || !out) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TC_ERR_NOT_FOUND;
    if (!it->second->done) {
        out->status = TC_PENDING;
        return TC_PENDING;
    }
    fill_result(it->second, out);
    return it->second->status;
}

tc_status tc_wait(tc_server* s, uint64_t ticket, int64_t timeout_ms, tc_result* out) {
    if (!s || !out) return TC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TC_ERR_NOT_FOUND;
    Request* r = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0));
    while (!r->done) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) {
            out->status = TC_ERR_TIMEOUT;
            return TC_ERR_TIMEOUT;
        }
    }
    fill_result(r, out);
    return r->status;
}

tc_status tc_release(tc_server* s, uint64_t ticket) {
    if (!s) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TC_ERR_NOT_FOUND;
    if (!it->second->done) return TC_PENDING;
    delete it->second;
    s->reqs.erase(it);
    return TC_OK;
}

tc_status tc_server_get_stats(const tc_server* s, tc_server_stats* out) {
    if (!s || !out) return TC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(const_cast<tc_server*>(s)->mu);
    *out = s->stats;
    out->resident_bytes = s->resident;
    return TC_OK;
}

}  // extern "C"
