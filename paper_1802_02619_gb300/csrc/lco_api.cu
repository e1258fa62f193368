// lco_api.cu -- status strings, workspace helpers and kernel timing of the C ABI.
#include <atomic>
#include <cstring>
#include <mutex>

#include "lco_internal.cuh"

namespace lco {
namespace {

constexpr int kTimingSlots = 4096;

struct TimingSlot {
    char name[40];
    cudaEvent_t ev0, ev1;
    bool used;
};

std::mutex g_mu;
bool g_timing = false;
TimingSlot g_slots[kTimingSlots];
int g_nslots = 0;
int g_open = -1;
std::atomic<long long> g_launches{0};

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

}  // namespace

void timing_begin(const char *name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_mu);
    g_open = -1;
    if (!g_timing || g_nslots >= kTimingSlots || capturing(s)) return;
    TimingSlot &t = g_slots[g_nslots];
    if (!t.used) {
        if (cudaEventCreate(&t.ev0) != cudaSuccess || cudaEventCreate(&t.ev1) != cudaSuccess) return;
        t.used = true;
    }
    std::strncpy(t.name, name, sizeof(t.name) - 1);
    t.name[sizeof(t.name) - 1] = 0;
    if (cudaEventRecord(t.ev0, s) != cudaSuccess) return;
    g_open = g_nslots;
}

void timing_end(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_open < 0) return;
    if (cudaEventRecord(g_slots[g_open].ev1, s) == cudaSuccess) ++g_nslots;
    g_open = -1;
}

// Wait self-test: one warp looks back over predecessors that never publish,
// then one thread waits on an mbarrier phase that never completes.  Both
// waits give up after `budget` cycles (a kernel argument, so no other
// kernel's budget changes) and record LCO_ERR_TIMEOUT.
__global__ void k_selftest_wait(uint64_t *state, int32_t *status, long long budget) {
    __shared__ uint64_t s_bar;
    lookback_warp(state, 8, status, budget);     // tiles 0..7 never publish
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);                    // nothing arrives
        if (!mbar_wait_bounded(&s_bar, 0, budget)) set_error(status + 1, LCO_ERR_TIMEOUT);
    }
}

}  // namespace lco

extern "C" {

int32_t lco_selftest_wait(void *scratch, int64_t budget_cycles, int32_t *lookback_status, int32_t *mbarrier_status,
                          void *stream) {
    if (!scratch || budget_cycles <= 0 || !lookback_status || !mbarrier_status) return LCO_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = reinterpret_cast<char *>(scratch);
    uint64_t *state = reinterpret_cast<uint64_t *>(w);
    int32_t *status = reinterpret_cast<int32_t *>(w + 256);
    if (cudaMemsetAsync(w, 0, 512, s) != cudaSuccess) return LCO_ERR_CUDA;
    lco::k_selftest_wait<<<1, 32, 0, s>>>(state, status, (long long)budget_cycles);
    const cudaError_t le = cudaGetLastError();
    int32_t st[2] = {0, 0};
    if (le != cudaSuccess || cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LCO_ERR_CUDA;
    *lookback_status = st[0];
    *mbarrier_status = st[1];
    return LCO_OK;
}

const char *lco_status_str(int32_t status) {
    switch (status) {
    case LCO_OK: return "ok";
    case LCO_ERR_INVALID: return "invalid argument";
    case LCO_ERR_OVERFLOW: return "index space exceeds the LIV range (2^63-1; 2^127-1 for wide LIVs)";
    case LCO_ERR_UNSORTED: return "input LIVs not strictly ascending";
    case LCO_ERR_OOM: return "workspace too small or allocation failed";
    case LCO_ERR_TIMEOUT: return "device wait timed out";
    case LCO_ERR_CUDA: return "CUDA runtime error";
    case LCO_ERR_ADMISSION: return "request exceeds the memory budget";
    case LCO_ERR_CAPACITY: return "output capacity smaller than the product count";
    case LCO_ERR_TOO_LARGE: return "input larger than the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
    }
}

int32_t lco_build_arch(void) {
#ifdef LCO_BUILD_ARCH
    return LCO_BUILD_ARCH;
#else
    return 0;
#endif
}

int32_t lco_workspace_status(const void *ws, int32_t *status, void *stream) {
    if (!ws || !status) return LCO_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LCO_ERR_CUDA;
    if (cudaMemcpy(status, ws, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return LCO_ERR_CUDA;
    return LCO_OK;
}

int32_t lco_timing_enable(int32_t enable) {
    std::lock_guard<std::mutex> lk(lco::g_mu);
    lco::g_timing = enable != 0;
    lco::g_nslots = 0;
    lco::g_open = -1;
    return LCO_OK;
}

int32_t lco_timing_read(lco_timing_record *out, int32_t max, int32_t *count) {
    if (!count || (max > 0 && !out)) return LCO_ERR_INVALID;
    std::lock_guard<std::mutex> lk(lco::g_mu);
    int32_t n = 0;
    for (int i = 0; i < lco::g_nslots && n < max; ++i) {
        lco::TimingSlot &t = lco::g_slots[i];
        if (cudaEventSynchronize(t.ev1) != cudaSuccess) return LCO_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev0, t.ev1) != cudaSuccess) return LCO_ERR_CUDA;
        std::memcpy(out[n].name, t.name, sizeof(out[n].name));
        out[n].ms = ms;
        ++n;
    }
    *count = n;
    lco::g_nslots = 0;
    return LCO_OK;
}

int64_t lco_launch_count(void) { return lco::g_launches.load(); }

}  // extern "C"
