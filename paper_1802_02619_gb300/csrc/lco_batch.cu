// lco_batch.cu -- many independent contractions in one enqueue.
//
// Every problem keeps its own plan (the Table-4 choice of Sec. 5.2, or the
// tuner's forced choice) and its own region of one shared workspace, so the
// arithmetic is exactly that of lco_contract.  The problems are spread over
// a pool of streams forked from the caller's stream with events and joined
// back into it; the whole batch can therefore be captured into one CUDA
// graph and replayed as a single launch, with the small problems running
// concurrently on the device.
#include <cstring>
#include <new>
#include <vector>

#include "lco_host.h"

struct lco_batch {
    int32_t nprob;
    int32_t nstreams;
    std::vector<lco_plan *> plans;
    std::vector<size_t> p1_bytes;       // phase-1 workspace of each problem (cap 0)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> fork_ev, join_ev;
    int device;
};

namespace {

void destroy(lco_batch *b) {
    if (!b) return;
    for (lco_plan *p : b->plans) lco_plan_destroy(p);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->fork_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : b->join_ev) cudaEventDestroy(e);
    delete b;
}

// Offsets of every problem's workspace inside the batch workspace.
int32_t layout(const lco_batch *b, const int64_t *caps, std::vector<size_t> &offs, size_t *total) {
    offs.resize(b->nprob);
    size_t off = 0;
    for (int i = 0; i < b->nprob; ++i) {
        size_t nb = 0;
        const int64_t cap = caps ? caps[i] : 0;
        if (cap < 0) return LCO_ERR_INVALID;
        int32_t rc = lco_contract_workspace(b->plans[i], cap, &nb);
        if (rc != LCO_OK) return rc;
        offs[i] = off;
        off += lco::align_up(nb);
    }
    *total = off;
    return LCO_OK;
}

// Forks the pool from `origin`, runs fn(problem, stream) for every problem,
// joins the pool back into `origin`.
template <typename Fn>
int32_t fan_out(lco_batch *b, cudaStream_t origin, Fn fn) {
    if (cudaEventRecord(b->fork_ev[0], origin) != cudaSuccess) return LCO_ERR_CUDA;
    for (int s = 0; s < b->nstreams; ++s)
        if (cudaStreamWaitEvent(b->streams[s], b->fork_ev[0], 0) != cudaSuccess) return LCO_ERR_CUDA;
    int32_t rc = LCO_OK;
    for (int i = 0; i < b->nprob && rc == LCO_OK; ++i) rc = fn(i, b->streams[i % b->nstreams]);
    for (int s = 0; s < b->nstreams; ++s) {
        if (cudaEventRecord(b->join_ev[s], b->streams[s]) != cudaSuccess) return LCO_ERR_CUDA;
        if (cudaStreamWaitEvent(origin, b->join_ev[s], 0) != cudaSuccess) return LCO_ERR_CUDA;
    }
    return rc;
}

}  // namespace

extern "C" {

int32_t lco_batch_plan(int32_t nprob, const lco_problem *probs, int32_t nstreams, lco_batch **out) {
    if (!out || nprob < 1 || !probs) return LCO_ERR_INVALID;
    *out = nullptr;
    if (nstreams < 1) nstreams = 1;
    if (nstreams > 64) nstreams = 64;
    lco_batch *b = new (std::nothrow) lco_batch();
    if (!b) return LCO_ERR_OOM;
    b->nprob = nprob;
    b->nstreams = nstreams;
    cudaGetDevice(&b->device);
    for (int i = 0; i < nprob; ++i) {
        lco_plan *p = nullptr;
        lco_tune t;
        t.alg = probs[i].alg;
        t.max_digit_bits = probs[i].max_digit_bits;
        int32_t rc = lco_contract_plan_ex(&probs[i].a, &probs[i].b, probs[i].ncontract, probs[i].modes_a,
                                          probs[i].modes_b, &t, &p);
        if (rc != LCO_OK) {
            destroy(b);
            return rc;
        }
        b->plans.push_back(p);
    }
    b->streams.resize(nstreams);
    b->join_ev.resize(nstreams);
    b->fork_ev.resize(1);
    for (int s = 0; s < nstreams; ++s) {
        if (cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[s], cudaEventDisableTiming) != cudaSuccess) {
            destroy(b);
            return LCO_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&b->fork_ev[0], cudaEventDisableTiming) != cudaSuccess) {
        destroy(b);
        return LCO_ERR_CUDA;
    }
    *out = b;
    return LCO_OK;
}

int32_t lco_batch_destroy(lco_batch *b) {
    destroy(b);
    return LCO_OK;
}

int32_t lco_batch_info(const lco_batch *b, int32_t i, lco_plan_info *info) {
    if (!b || i < 0 || i >= b->nprob) return LCO_ERR_INVALID;
    return lco_plan_get_info(b->plans[i], info);
}

int32_t lco_batch_workspace(const lco_batch *b, const int64_t *caps, size_t *ws_bytes) {
    if (!b || !ws_bytes) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    return layout(b, caps, offs, ws_bytes);
}

int32_t lco_batch_symbolic(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws,
                           size_t ws_bytes, void *stream) {
    if (!b || !ops || !ws) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    char *base = reinterpret_cast<char *>(ws);
    return fan_out(b, (cudaStream_t)stream, [&](int i, cudaStream_t s) {
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps ? caps[i] : 0, &nb);
        return lco_contract_symbolic(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val,
                                     base + offs[i], nb, s);
    });
}

int32_t lco_batch_numeric(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws, size_t ws_bytes,
                          void *stream) {
    if (!b || !ops || !ws || !caps) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    char *base = reinterpret_cast<char *>(ws);
    return fan_out(b, (cudaStream_t)stream, [&](int i, cudaStream_t s) {
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps[i], &nb);
        return lco_contract_numeric(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val,
                                    ops[i].c_liv, ops[i].c_val, caps[i], base + offs[i], nb, s);
    });
}

int32_t lco_batch_contract(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws, size_t ws_bytes,
                           void *stream) {
    lco::NvtxRange nvtx("lco_batch_contract");
    if (!b || !ops || !ws || !caps) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    char *base = reinterpret_cast<char *>(ws);
    return fan_out(b, (cudaStream_t)stream, [&](int i, cudaStream_t s) {
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps[i], &nb);
        return lco_contract(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val, ops[i].c_liv,
                            ops[i].c_val, caps[i], base + offs[i], nb, s);
    });
}

int32_t lco_batch_results(const lco_batch *b, const int64_t *caps, const void *ws, lco_contract_result *out,
                          void *stream) {
    if (!b || !ws || !out) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCO_ERR_CUDA;
    const char *base = reinterpret_cast<const char *>(ws);
    for (int i = 0; i < b->nprob; ++i) {
        rc = lco_contract_result_get(base + offs[i], &out[i], stream);
        if (rc != LCO_OK) return rc;
    }
    return LCO_OK;
}

}  // extern "C"
