// lco_serve.cu -- device memory pool and the served-contraction runtime.
//
// The pool is host bookkeeping over one device allocation: first fit in
// address order, 256-byte blocks, freed neighbours merged.
//
// The server keeps operands, workspaces and results in its pool.  A worker
// thread admits queued requests in arrival order into stream slots and runs
// each one as the two phases of Sec. 5.2 -- phase 1 gives f, the product
// count; phase 2 multiplies into an output of f entries -- with an
// asynchronous read of the workspace header between them.  Operands are
// immutable while resident, so the plan and f of an (operand pair, modes)
// combination are kept after its first request: a repeated request is
// admitted with its whole output and workspace and runs both phases back
// to back, with one completion read.  Completion is observed with CUDA
// events, so requests overlap on the device and none waits for another's
// host round trip.  The arithmetic of a request is exactly that of
// lco_contract (same plan, same kernels).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lco_host.h"

// ---------------------------------------------------------------------------
// Pool
// ---------------------------------------------------------------------------

struct lco_pool {
    uintptr_t base = 0;
    size_t bytes = 0;
    std::map<size_t, size_t> free_blocks;        // offset -> size, address order
    std::unordered_map<size_t, size_t> used;     // offset -> size
    size_t in_use = 0, peak = 0;
    mutable std::mutex mu;
};

namespace {

constexpr size_t kPoolAlign = 256;

size_t round_up(size_t x) { return (x + kPoolAlign - 1) / kPoolAlign * kPoolAlign; }

}  // namespace

extern "C" {

int32_t lco_pool_create(void *base, size_t bytes, lco_pool **pool) {
    if (!pool) return LCO_ERR_INVALID;
    *pool = nullptr;
    if (!base) return LCO_ERR_INVALID;
    // usable range: aligned start, whole blocks
    const uintptr_t b = reinterpret_cast<uintptr_t>(base);
    const uintptr_t start = (b + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
    if (bytes < kPoolAlign || start - b >= bytes) return LCO_ERR_INVALID;
    const size_t usable = (bytes - (start - b)) / kPoolAlign * kPoolAlign;
    if (usable < kPoolAlign) return LCO_ERR_INVALID;
    lco_pool *p = new (std::nothrow) lco_pool();
    if (!p) return LCO_ERR_OOM;
    p->base = start;
    p->bytes = usable;
    p->free_blocks[0] = usable;
    *pool = p;
    return LCO_OK;
}

int32_t lco_pool_destroy(lco_pool *pool) {
    delete pool;
    return LCO_OK;
}

int32_t lco_pool_alloc(lco_pool *pool, size_t bytes, void **ptr) {
    if (!pool || !ptr) return LCO_ERR_INVALID;
    *ptr = nullptr;
    const size_t need = round_up(bytes ? bytes : 1);
    std::lock_guard<std::mutex> g(pool->mu);
    for (auto it = pool->free_blocks.begin(); it != pool->free_blocks.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, sz = it->second;
        pool->free_blocks.erase(it);
        if (sz > need) pool->free_blocks[off + need] = sz - need;
        pool->used[off] = need;
        pool->in_use += need;
        pool->peak = std::max(pool->peak, pool->in_use);
        *ptr = reinterpret_cast<void *>(pool->base + off);
        return LCO_OK;
    }
    return LCO_ERR_OOM;
}

int32_t lco_pool_free(lco_pool *pool, void *ptr) {
    if (!pool || !ptr) return LCO_ERR_INVALID;
    const uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    if (a < pool->base || a >= pool->base + pool->bytes) return LCO_ERR_INVALID;
    const size_t off = a - pool->base;
    std::lock_guard<std::mutex> g(pool->mu);
    auto u = pool->used.find(off);
    if (u == pool->used.end()) return LCO_ERR_INVALID;
    size_t start = off, sz = u->second;
    pool->used.erase(u);
    pool->in_use -= sz;
    auto next = pool->free_blocks.lower_bound(start);
    if (next != pool->free_blocks.end() && next->first == start + sz) {   // merge with the next block
        sz += next->second;
        next = pool->free_blocks.erase(next);
    }
    if (next != pool->free_blocks.begin()) {                               // and with the previous one
        auto prev = std::prev(next);
        if (prev->first + prev->second == start) {
            start = prev->first;
            sz += prev->second;
            pool->free_blocks.erase(prev);
        }
    }
    pool->free_blocks[start] = sz;
    return LCO_OK;
}

int32_t lco_pool_stats(const lco_pool *pool, size_t *used, size_t *peak, size_t *largest_free) {
    if (!pool) return LCO_ERR_INVALID;
    std::lock_guard<std::mutex> g(pool->mu);
    size_t lf = 0;
    for (const auto &kv : pool->free_blocks) lf = std::max(lf, kv.second);
    if (used) *used = pool->in_use;
    if (peak) *peak = pool->peak;
    if (largest_free) *largest_free = lf;
    return LCO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------

namespace {

using Clock = std::chrono::steady_clock;

struct Operand {
    lco_shape shape{};
    int64_t *liv = nullptr;
    double *val = nullptr;
    void *block = nullptr;
    int refs = 0;          // requests holding it
    bool dropped = false;
};

enum ReqState { kQueued = 0, kPhase1 = 1, kPhase2 = 2, kDone = 3 };

// The plan of an (operand pair, modes) combination, shared by its requests,
// and its product count once a request has computed it.
struct PlanEntry {
    lco_plan *plan = nullptr;
    lco_plan_info info{};
    std::atomic<int64_t> f{-1};
    ~PlanEntry() {
        if (plan) lco_plan_destroy(plan);
    }
};

struct PlanKey {
    int64_t ha, hb;
    int32_t nc;
    int32_t ma[LCO_MAX_ORDER], mb[LCO_MAX_ORDER];
    bool operator<(const PlanKey &o) const {
        if (ha != o.ha) return ha < o.ha;
        if (hb != o.hb) return hb < o.hb;
        if (nc != o.nc) return nc < o.nc;
        for (int i = 0; i < nc; ++i) {
            if (ma[i] != o.ma[i]) return ma[i] < o.ma[i];
            if (mb[i] != o.mb[i]) return mb[i] < o.mb[i];
        }
        return false;
    }
};

struct Request {
    uint64_t id = 0;
    std::shared_ptr<Operand> a, b;
    std::shared_ptr<PlanEntry> pe;
    lco_plan *plan = nullptr;  // pe->plan
    lco_plan_info info{};
    std::atomic<int> state{kQueued};
    int slot = -1;
    void *ws = nullptr;        // workspace (phase 1, and phase 2 when f fits)
    int64_t ws_cap = 0;        // output capacity the workspace is sized for
    void *ws2 = nullptr;       // larger workspace when f exceeded ws_cap
    void *cbuf = nullptr;      // C: liv[cap] then val[cap]
    int64_t cap = 0;
    int32_t status = LCO_OK, alg = 0;
    int64_t f = 0, nnz_c = 0;
    double t_submit = 0, t_done = 0;
    Clock::time_point t_wait_mem{};
    bool waiting_mem = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    lco::WsHeader *hdr = nullptr;   // pinned host copy of the request's header
    Request *req = nullptr;
};

// A request that cannot get pool memory for this long fails with
// LCO_ERR_ADMISSION (memory is freed only by completions and releases).
constexpr double kAdmissionWaitUs = 2e6;

}  // namespace

struct lco_server {
    int device = 0;
    void *pool_mem = nullptr;
    bool own_pool = false;
    lco_pool *pool = nullptr;
    std::vector<Slot> slots;
    cudaStream_t put_stream = nullptr;       // operand uploads
    std::mutex mu;                           // everything below
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::unordered_map<int64_t, std::shared_ptr<Operand>> operands;
    std::map<PlanKey, std::shared_ptr<PlanEntry>> plans;   // dropped with either operand
    uint64_t next_req = 1;
    int64_t next_handle = 1;
    uint64_t submitted = 0, completed = 0, failed = 0;
    int64_t in_flight = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    int nworkers = 1;
    Clock::time_point epoch;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - epoch).count();
    }
    void pfree(void *&p) {
        if (p) lco_pool_free(pool, p);
        p = nullptr;
    }
    void finish(Request *r, int32_t status);
    void finish_locked(Request *r, int32_t status);
    bool admit(Request *r, Slot &sl, int si);
    void advance(Slot &sl);
    void run(int w);
};

void lco_server::finish(Request *r, int32_t status) {
    std::lock_guard<std::mutex> g(mu);
    finish_locked(r, status);
}

void lco_server::finish_locked(Request *r, int32_t status) {
    // caller holds mu; the request's device work has completed (or never ran)
    if (status != LCO_OK) r->status = status;
    pfree(r->ws);
    pfree(r->ws2);
    if (r->status != LCO_OK) pfree(r->cbuf);
    if (r->a) r->a->refs--;
    if (r->b) r->b->refs--;
    for (auto *op : {r->a.get(), r->b.get()}) {
        if (op && op->dropped && op->refs == 0 && op->block) {
            lco_pool_free(pool, op->block);
            op->block = nullptr;
        }
    }
    r->a.reset();
    r->b.reset();
    if (r->pe && r->status == LCO_OK && r->f >= 0) r->pe->f.store(r->f);
    r->pe.reset();
    r->plan = nullptr;
    r->state = kDone;
    r->t_done = now_us();
    if (r->slot >= 0) {
        slots[r->slot].req = nullptr;
        r->slot = -1;
        in_flight--;
    }
    if (r->status == LCO_OK) completed++; else failed++;
    cv_done.notify_all();
}

// Phase 1 of a queued request on slot `si`; false when the pool cannot hold
// its workspace yet (the request stays queued).
bool lco_server::admit(Request *r, Slot &sl, int si) {
    const int64_t na = r->a->shape.nnz, nb = r->b->shape.nnz;
    const int64_t fk = r->pe->f.load();
    if (fk >= 0) {
        // the product count is known: output and workspace at once, both
        // phases back to back, one completion read
        const int64_t cap = fk > 0 ? fk : 1;
        size_t wb = 0;
        if (lco_contract_workspace(r->plan, cap, &wb) != LCO_OK) {
            finish(r, LCO_ERR_INVALID);
            return true;
        }
        if (lco_pool_alloc(pool, wb, &r->ws) != LCO_OK) return false;
        if (lco_pool_alloc(pool, (size_t)cap * 16, &r->cbuf) != LCO_OK) {
            pfree(r->ws);
            return false;
        }
        r->ws_cap = cap;
        r->cap = cap;
        r->f = fk;
        r->slot = si;
        sl.req = r;
        {
            std::lock_guard<std::mutex> g(mu);
            in_flight++;
        }
        r->state = kPhase2;
        cudaStream_t s = sl.stream;
        int64_t *c_liv = reinterpret_cast<int64_t *>(r->cbuf);
        double *c_val = reinterpret_cast<double *>(c_liv + cap);
        int32_t rc = LCO_OK;
        if (lco::contract_ws_init(r->plan, r->ws, cap, s) != cudaSuccess) rc = LCO_ERR_CUDA;
        if (rc == LCO_OK)
            rc = lco_contract(r->plan, r->a->liv, r->a->val, r->b->liv, r->b->val, c_liv, c_val, cap, r->ws, wb, s);
        if (rc == LCO_OK &&
            cudaMemcpyAsync(sl.hdr, r->ws, sizeof(lco::WsHeader), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = LCO_ERR_CUDA;
        if (rc == LCO_OK && cudaEventRecord(sl.ev, s) != cudaSuccess) rc = LCO_ERR_CUDA;
        if (rc != LCO_OK) {
            cudaStreamSynchronize(s);
            finish(r, rc);
        }
        return true;
    }
    // room for phase 2 too when f turns out to be at most this guess
    r->ws_cap = 4 * (na + nb) + 1024;
    size_t wb = 0;
    if (lco_contract_workspace(r->plan, r->ws_cap, &wb) != LCO_OK) {
        finish(r, LCO_ERR_INVALID);
        return true;
    }
    if (lco_pool_alloc(pool, wb, &r->ws) != LCO_OK) {
        // fall back to a phase-1-only workspace
        r->ws_cap = 0;
        lco_contract_workspace(r->plan, 0, &wb);
        if (lco_pool_alloc(pool, wb, &r->ws) != LCO_OK) return false;
    }
    r->slot = si;
    sl.req = r;
    {
        std::lock_guard<std::mutex> g(mu);
        in_flight++;
    }
    r->state = kPhase1;
    cudaStream_t s = sl.stream;
    int32_t rc = LCO_OK;
    if (lco::contract_ws_init(r->plan, r->ws, -1, s) != cudaSuccess) rc = LCO_ERR_CUDA;
    if (rc == LCO_OK)
        rc = lco_contract_symbolic(r->plan, r->a->liv, r->a->val, r->b->liv, r->b->val, r->ws, wb, s);
    if (rc == LCO_OK && cudaMemcpyAsync(sl.hdr, r->ws, sizeof(lco::WsHeader), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = LCO_ERR_CUDA;
    if (rc == LCO_OK && cudaEventRecord(sl.ev, s) != cudaSuccess) rc = LCO_ERR_CUDA;
    if (rc != LCO_OK) {
        cudaStreamSynchronize(s);
        finish(r, rc);
    }
    return true;
}

// The slot's event has completed: move its request on.
void lco_server::advance(Slot &sl) {
    Request *r = sl.req;
    cudaStream_t s = sl.stream;
    const lco::WsHeader h = *sl.hdr;
    if (h.status != 0) {
        finish(r, h.status);
        return;
    }
    if (r->state == kPhase1) {
        r->f = h.f;
        r->alg = h.alg;
        const int64_t cap = h.f > 0 ? h.f : 1;
        if (!r->cbuf) {
            if (lco_pool_alloc(pool, (size_t)cap * 16, &r->cbuf) != LCO_OK) {
                if (!r->waiting_mem) {
                    r->waiting_mem = true;
                    r->t_wait_mem = Clock::now();
                }
                return;                                  // retried on the next sweep
            }
            r->cap = cap;
        }
        void *ws = r->ws;
        size_t wb = 0;
        lco_contract_workspace(r->plan, cap, &wb);
        if (h.f > r->ws_cap) {
            // phase 2 needs a larger workspace: carry phase 1's region over
            if (!r->ws2 && lco_pool_alloc(pool, wb, &r->ws2) != LCO_OK) {
                if (!r->waiting_mem) {
                    r->waiting_mem = true;
                    r->t_wait_mem = Clock::now();
                }
                return;
            }
            ws = r->ws2;
            if (cudaMemcpyAsync(ws, r->ws, lco::contract_phase1_bytes(r->plan), cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess) {
                cudaStreamSynchronize(s);
                finish(r, LCO_ERR_CUDA);
                return;
            }
        }
        // SOP's sort state sits at an offset that depends on the capacity
        if (r->info.alg == LCO_ALG_SOP && lco::contract_ws_init(r->plan, ws, cap, s) != cudaSuccess) {
            cudaStreamSynchronize(s);
            finish(r, LCO_ERR_CUDA);
            return;
        }
        r->waiting_mem = false;
        int64_t *c_liv = reinterpret_cast<int64_t *>(r->cbuf);
        double *c_val = reinterpret_cast<double *>(c_liv + cap);
        int32_t rc = lco_contract_numeric(r->plan, r->a->liv, r->a->val, r->b->liv, r->b->val, c_liv, c_val, cap,
                                          ws, wb, s);
        if (rc == LCO_OK &&
            cudaMemcpyAsync(sl.hdr, ws, sizeof(lco::WsHeader), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = LCO_ERR_CUDA;
        if (rc == LCO_OK && cudaEventRecord(sl.ev, s) != cudaSuccess) rc = LCO_ERR_CUDA;
        if (rc != LCO_OK) {
            cudaStreamSynchronize(s);
            finish(r, rc);
            return;
        }
        r->state = kPhase2;
        return;
    }
    // phase 2 done
    r->nnz_c = h.nnz_c;
    r->alg = h.alg;
    finish(r, LCO_OK);
}

// Worker w owns the slots i with i % nworkers == w.  The server mutex is
// held only to take requests from the queue and to publish results; CUDA
// calls run without it, so the workers' host work overlaps.
void lco_server::run(int w) {
    cudaSetDevice(device);
    std::vector<int> mine;
    for (int i = w; i < (int)slots.size(); i += nworkers) mine.push_back(i);
    while (true) {
        bool progressed = false;
        // 1. this worker's requests in flight
        for (int si : mine) {
            Slot &sl = slots[si];
            Request *r = sl.req;
            if (!r) continue;
            if (r->waiting_mem) {
                // phase 1 is done; waiting for pool memory for phase 2
                if (std::chrono::duration<double, std::micro>(Clock::now() - r->t_wait_mem).count() >
                    kAdmissionWaitUs) {
                    finish(r, LCO_ERR_ADMISSION);
                    progressed = true;
                    continue;
                }
                advance(sl);
                progressed = progressed || !r->waiting_mem;
                continue;
            }
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            if (q != cudaSuccess) {
                finish(r, LCO_ERR_CUDA);
                continue;
            }
            advance(sl);
        }
        // 2. admissions into free slots, in arrival order
        for (int si : mine) {
            Slot &sl = slots[si];
            if (sl.req) continue;
            Request *r = nullptr;
            {
                std::lock_guard<std::mutex> g(mu);
                if (queue.empty()) break;
                r = queue.front();
                queue.pop_front();
                if (stop) {
                    finish_locked(r, LCO_ERR_ADMISSION);
                    progressed = true;
                    continue;
                }
            }
            if (admit(r, sl, si)) {
                r->waiting_mem = false;
                progressed = true;
                continue;
            }
            // no memory yet: back to the head of the queue (or fail once the
            // wait has lasted too long)
            std::lock_guard<std::mutex> g(mu);
            if (!r->waiting_mem) {
                r->waiting_mem = true;
                r->t_wait_mem = Clock::now();
            } else if (std::chrono::duration<double, std::micro>(Clock::now() - r->t_wait_mem).count() >
                       kAdmissionWaitUs) {
                r->waiting_mem = false;
                finish_locked(r, LCO_ERR_ADMISSION);
                progressed = true;
                continue;
            }
            queue.push_front(r);
            break;
        }
        bool busy = false;
        for (int si : mine) busy = busy || slots[si].req != nullptr;
        if (!progressed) {
            std::unique_lock<std::mutex> lk(mu);
            if (stop && queue.empty() && !busy) break;
            if (!busy && queue.empty()) {
                cv_work.wait(lk);                        // idle: sleep until a submit or stop
            } else {
                lk.unlock();                             // work on the device: poll again shortly
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            }
        }
    }
}

namespace {

int32_t fill_result(const lco_server *srv, const Request *r, lco_serve_result *out) {
    std::memset(out, 0, sizeof(*out));
    out->done = r->state == kDone;
    out->status = r->status;
    out->alg = r->alg;
    out->f = r->f;
    out->submit_us = r->t_submit;
    out->done_us = r->t_done;
    out->c = r->info.c_shape;
    out->c.nnz = out->done ? r->nnz_c : 0;
    if (out->done && r->status == LCO_OK && r->cbuf) {
        out->c_liv = reinterpret_cast<const int64_t *>(r->cbuf);
        out->c_val = reinterpret_cast<const double *>(out->c_liv + r->cap);
    }
    (void)srv;
    return LCO_OK;
}

}  // namespace

extern "C" {

int32_t lco_serve_create(const lco_serve_config *cfg, lco_server **out) {
    if (!cfg || !out) return LCO_ERR_INVALID;
    *out = nullptr;
    if (cfg->nslots < 1 || cfg->nslots > 256 || cfg->pool_bytes < 4096) return LCO_ERR_INVALID;
    std::unique_ptr<lco_server> s(new (std::nothrow) lco_server());
    if (!s) return LCO_ERR_OOM;
    if (cfg->device >= 0) {
        if (cudaSetDevice(cfg->device) != cudaSuccess) return LCO_ERR_CUDA;
        s->device = cfg->device;
    } else if (cudaGetDevice(&s->device) != cudaSuccess) {
        return LCO_ERR_CUDA;
    }
    if (cfg->pool) {
        s->pool_mem = cfg->pool;
    } else {
        if (cudaMalloc(&s->pool_mem, cfg->pool_bytes) != cudaSuccess) return LCO_ERR_OOM;
        s->own_pool = true;
    }
    int32_t rc = lco_pool_create(s->pool_mem, cfg->pool_bytes, &s->pool);
    if (rc != LCO_OK) {
        if (s->own_pool) cudaFree(s->pool_mem);
        return rc;
    }
    s->slots.resize(cfg->nslots);
    if (cudaStreamCreateWithFlags(&s->put_stream, cudaStreamNonBlocking) != cudaSuccess) {
        lco_server *raw = s.release();
        raw->stop = true;
        lco_serve_destroy(raw);
        return LCO_ERR_CUDA;
    }
    for (auto &sl : s->slots) {
        void *h = nullptr;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&h, sizeof(lco::WsHeader)) != cudaSuccess) {
            lco_server *raw = s.release();
            raw->stop = true;
            lco_serve_destroy(raw);
            return LCO_ERR_CUDA;
        }
        sl.hdr = reinterpret_cast<lco::WsHeader *>(h);
    }
    s->epoch = Clock::now();
    s->nworkers = cfg->nworkers > 0 ? cfg->nworkers : 4;
    if (s->nworkers > cfg->nslots) s->nworkers = cfg->nslots;
    lco_server *raw = s.release();
    for (int w = 0; w < raw->nworkers; ++w) raw->workers.emplace_back([raw, w] { raw->run(w); });
    *out = raw;
    return LCO_OK;
}

int32_t lco_serve_destroy(lco_server *srv) {
    if (!srv) return LCO_ERR_INVALID;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    for (auto &t : srv->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(srv->device);
    for (auto &sl : srv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.hdr) cudaFreeHost(sl.hdr);
    }
    if (srv->put_stream) cudaStreamDestroy(srv->put_stream);
    srv->reqs.clear();
    srv->plans.clear();
    srv->operands.clear();
    lco_pool_destroy(srv->pool);
    if (srv->own_pool) cudaFree(srv->pool_mem);
    delete srv;
    return LCO_OK;
}

int32_t lco_serve_put(lco_server *srv, const lco_shape *t, const int64_t *liv, const double *val, int64_t *handle) {
    if (!srv || !t || !handle) return LCO_ERR_INVALID;
    int64_t total = 0;
    int32_t rc = lco::check_shape(t, &total);
    if (rc != LCO_OK) return rc;
    if (t->nnz < 0 || (t->nnz > 0 && (!liv || !val))) return LCO_ERR_INVALID;
    auto op = std::make_shared<Operand>();
    op->shape = *t;
    const size_t n = (size_t)(t->nnz > 0 ? t->nnz : 1);
    if (lco_pool_alloc(srv->pool, n * 16, &op->block) != LCO_OK) return LCO_ERR_ADMISSION;
    op->liv = reinterpret_cast<int64_t *>(op->block);
    op->val = reinterpret_cast<double *>(op->liv + n);
    cudaSetDevice(srv->device);
    if (t->nnz > 0) {
        cudaStream_t s = srv->put_stream;
        if (cudaMemcpyAsync(op->liv, liv, (size_t)t->nnz * 8, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaMemcpyAsync(op->val, val, (size_t)t->nnz * 8, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            lco_pool_free(srv->pool, op->block);
            return LCO_ERR_CUDA;
        }
    }
    std::lock_guard<std::mutex> g(srv->mu);
    *handle = srv->next_handle++;
    srv->operands[*handle] = op;
    return LCO_OK;
}

int32_t lco_serve_drop(lco_server *srv, int64_t handle) {
    if (!srv) return LCO_ERR_INVALID;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->operands.find(handle);
    if (it == srv->operands.end()) return LCO_ERR_INVALID;
    auto op = it->second;
    srv->operands.erase(it);
    for (auto pit = srv->plans.begin(); pit != srv->plans.end();) {
        if (pit->first.ha == handle || pit->first.hb == handle) pit = srv->plans.erase(pit);
        else ++pit;
    }
    op->dropped = true;
    if (op->refs == 0 && op->block) {
        lco_pool_free(srv->pool, op->block);
        op->block = nullptr;
    }
    return LCO_OK;
}

int32_t lco_serve_submit(lco_server *srv, int64_t ha, int64_t hb, int32_t ncontract, const int32_t *modes_a,
                         const int32_t *modes_b, uint64_t *req) {
    if (!srv || !req) return LCO_ERR_INVALID;
    if (ncontract < 0 || ncontract > LCO_MAX_ORDER || (ncontract > 0 && (!modes_a || !modes_b)))
        return LCO_ERR_INVALID;
    std::shared_ptr<Operand> a, b;
    PlanKey key{};
    key.ha = ha;
    key.hb = hb;
    key.nc = ncontract;
    for (int i = 0; i < ncontract; ++i) {
        key.ma[i] = modes_a[i];
        key.mb[i] = modes_b[i];
    }
    std::shared_ptr<PlanEntry> pe;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto ia = srv->operands.find(ha), ib = srv->operands.find(hb);
        if (ia == srv->operands.end() || ib == srv->operands.end()) return LCO_ERR_INVALID;
        a = ia->second;
        b = ib->second;
        auto pit = srv->plans.find(key);
        if (pit != srv->plans.end()) pe = pit->second;
    }
    if (!pe) {
        auto fresh = std::make_shared<PlanEntry>();
        int32_t rc = lco_contract_plan(&a->shape, &b->shape, ncontract, modes_a, modes_b, LCO_ALG_AUTO,
                                       &fresh->plan);
        if (rc != LCO_OK) return rc;
        lco_plan_get_info(fresh->plan, &fresh->info);
        std::lock_guard<std::mutex> g(srv->mu);
        auto ins = srv->plans.emplace(key, fresh);   // another thread may have made it meanwhile
        pe = ins.first->second;
    }
    auto r = std::make_unique<Request>();
    r->pe = pe;
    r->plan = pe->plan;
    r->info = pe->info;
    std::lock_guard<std::mutex> g(srv->mu);
    r->id = srv->next_req++;
    r->a = a;
    r->b = b;
    a->refs++;
    b->refs++;
    r->t_submit = srv->now_us();
    *req = r->id;
    srv->queue.push_back(r.get());
    srv->reqs[r->id] = std::move(r);
    srv->submitted++;
    srv->cv_work.notify_one();
    return LCO_OK;
}

int32_t lco_serve_poll(lco_server *srv, uint64_t req, lco_serve_result *out) {
    if (!srv || !out) return LCO_ERR_INVALID;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(req);
    if (it == srv->reqs.end()) return LCO_ERR_INVALID;
    return fill_result(srv, it->second.get(), out);
}

int32_t lco_serve_wait(lco_server *srv, uint64_t req, int64_t timeout_us, lco_serve_result *out) {
    if (!srv || !out) return LCO_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req);
    if (it == srv->reqs.end()) return LCO_ERR_INVALID;
    Request *r = it->second.get();
    auto done = [r] { return r->state == kDone; };
    if (timeout_us < 0) {
        srv->cv_done.wait(lk, done);
    } else {
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    }
    return fill_result(srv, r, out);
}

int32_t lco_serve_release(lco_server *srv, uint64_t req) {
    if (!srv) return LCO_ERR_INVALID;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(req);
    if (it == srv->reqs.end() || it->second->state != kDone) return LCO_ERR_INVALID;
    srv->pfree(it->second->cbuf);
    srv->reqs.erase(it);
    return LCO_OK;
}

int32_t lco_serve_get_stats(const lco_server *srv, lco_serve_stats *out) {
    if (!srv || !out) return LCO_ERR_INVALID;
    lco_server *s = const_cast<lco_server *>(srv);
    std::lock_guard<std::mutex> g(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = (int64_t)s->queue.size();
    out->in_flight = s->in_flight;
    size_t used = 0, peak = 0;
    lco_pool_stats(s->pool, &used, &peak, nullptr);
    out->pool_used = used;
    out->pool_peak = peak;
    out->pool_bytes = s->pool->bytes;
    return LCO_OK;
}

}  // extern "C"
