// lco_noalloc.cu -- radix permutation without a caller-supplied workspace.
//
// Some callers cannot allocate device memory at all: a plug-in running
// inside a host application that owns every device allocation (a framework
// with its own caching allocator that must not be bypassed, or a service
// that reserves all memory at start-up and forbids allocation in its steady
// state) can neither call cudaMalloc nor ask its host for a workspace of a
// size it does not know in advance.  lco_radix_permute_static serves them: it
// runs the same kernels as lco_radix_permute, with the scratch those kernels
// need taken from one fixed array in device memory that this library
// defines and that every GPU loading the library holds until the process
// exits.
#include <mutex>

#include "lco_host.h"

namespace lco {
namespace {

// Largest tensor (number of non-zeros) the fixed scratch serves.
constexpr int64_t kStaticMaxNnz = 65536;
// Header + digit counts and run starts + look-back words for the widest digit
// plan + two temporary (LIV, value) buffers, for kStaticMaxNnz elements.
constexpr size_t kStaticScratchBytes = 3u << 20;   // 3 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[64] = {nullptr};

// Device address of g_static_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
int32_t static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LCO_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return LCO_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return LCO_OK;
}

}  // namespace
}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_radix_permute_static(const lco_shape *t, const int32_t *new_sig, const int64_t *liv_in,
                                 const double *val_in, int64_t *liv_out, double *val_out, void *stream) {
    RpPlan p;
    int32_t rc = rp_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    if (t->nnz > kStaticMaxNnz) return LCO_ERR_TOO_LARGE;
    const size_t need = kWsHeaderBytes + rp_region_bytes(p, t->nnz);
    if (need > kStaticScratchBytes) return LCO_ERR_TOO_LARGE;
    if (t->nnz == 0) return LCO_OK;
    if (!liv_in || !val_in || !liv_out || !val_out) return LCO_ERR_INVALID;
    void *scratch = nullptr;
    if ((rc = static_scratch(&scratch)) != LCO_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = reinterpret_cast<char *>(scratch);
    // The array keeps the previous call's contents: the header (counters,
    // status) and the digit-histogram table must start at zero.
    if (cudaMemsetAsync(base, 0, kWsHeaderBytes + radix_hist_table_bytes(), s) != cudaSuccess) return LCO_ERR_CUDA;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(base);
    cudaError_t e = rp_enqueue(p, t->nnz, liv_in, val_in, liv_out, val_out, base + kWsHeaderBytes, hdr, s);
    return e == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

int32_t lco_radix_permute_static_status(int32_t *status, void *stream) {
    if (!status) return LCO_ERR_INVALID;
    void *scratch = nullptr;
    int32_t rc = static_scratch(&scratch);
    if (rc != LCO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCO_ERR_CUDA;
    // the status word is the first field of the header at the array's start
    if (cudaMemcpy(status, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return LCO_ERR_CUDA;
    return LCO_OK;
}

}  // extern "C"
