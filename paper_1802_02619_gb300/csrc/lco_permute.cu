// lco_permute.cu -- LIV shuffle (Sec. 3.1) and the radix permutation (Sec. 4.1).
#include <cstring>

#include "lco_host.h"

namespace lco {

// ---------------------------------------------------------------------------
// Host planning
// ---------------------------------------------------------------------------

int32_t check_sig(int32_t order, const int32_t *sig) {
    if (order < 1 || order > kMaxOrder || sig == nullptr) return LCO_ERR_INVALID;
    int seen[kMaxOrder] = {0};
    for (int t = 0; t < order; ++t) {
        if (sig[t] < 0 || sig[t] >= order || seen[sig[t]]) return LCO_ERR_INVALID;
        seen[sig[t]] = 1;
    }
    return LCO_OK;
}

int32_t check_shape(const lco_shape *t, int64_t *total) {
    if (t == nullptr) return LCO_ERR_INVALID;
    int32_t rc = check_sig(t->order, t->sig);
    if (rc != LCO_OK) return rc;
    if (t->nnz < 0) return LCO_ERR_INVALID;
    int64_t p = 1;
    for (int i = 0; i < t->order; ++i) {
        if (t->dims[i] < 1) return LCO_ERR_INVALID;
        if (p > INT64_MAX / t->dims[i]) return LCO_ERR_OVERFLOW;
        p *= t->dims[i];
    }
    if (total) *total = p;
    return LCO_OK;
}

RelinParams make_relin(int32_t order, const int64_t *dims, const int32_t *sig_old,
                       const int32_t *sig_new) {
    RelinParams r{};
    int pos_new[kMaxOrder];
    int64_t stride_new[kMaxOrder];
    int64_t s = 1;
    for (int t = 0; t < order; ++t) {
        pos_new[sig_new[t]] = t;
        stride_new[sig_new[t]] = s;
        s *= dims[sig_new[t]];
    }
    r.identity = 1;
    for (int t = 0; t < order; ++t)
        if (sig_old[t] != sig_new[t]) r.identity = 0;
    int nseg = 0;
    uint64_t range = 1;
    for (int t = 0; t < order; ++t) {
        const int x = sig_old[t];
        const bool extend = t > 0 && pos_new[x] == pos_new[sig_old[t - 1]] + 1;
        if (!extend) {
            if (nseg > 0) r.seg_div[nseg - 1] = make_div(range);
            r.seg_stride[nseg] = stride_new[x];
            ++nseg;
            range = 1;
        }
        range *= (uint64_t)dims[x];
    }
    r.seg_div[nseg - 1] = make_div(range);
    r.nseg = nseg;
    r.all_pow2 = 1;
    uint32_t bit = 0;
    for (int t = 0; t < nseg; ++t) {
        const uint64_t st = (uint64_t)r.seg_stride[t];
        if (!r.seg_div[t].pow2 || (st & (st - 1)) != 0) r.all_pow2 = 0;
        r.stride_shift[t] = st ? (uint32_t)__builtin_ctzll(st) : 0;
        const uint32_t w = r.seg_div[t].shift;   // log2 of the segment's range when it is a power of two
        r.in_shift[t] = bit;
        r.seg_mask[t] = w >= 64 ? ~0ull : (1ull << w) - 1;
        bit += w;
    }
    return r;
}

int32_t rp_plan(const lco_shape *t, const int32_t *new_sig, RpPlan *out, int max_digit_bits) {
    int64_t total = 0;
    int32_t rc = check_shape(t, &total);
    if (rc != LCO_OK) return rc;
    if ((rc = check_sig(t->order, new_sig)) != LCO_OK) return rc;
    const int N = t->order;
    int pos_old[kMaxOrder], pos_new[kMaxOrder];
    for (int i = 0; i < N; ++i) {
        pos_old[t->sig[i]] = i;
        pos_new[new_sig[i]] = i;
    }
    RpPlan p{};
    p.total = total;
    // Sec. 4.1: x is a rearrangement index when some index y that was more
    // significant than x becomes less significant than x.
    int nr = 0;
    for (int x = 0; x < N; ++x) {
        int r = 0;
        for (int y = 0; y < N; ++y)
            if (y != x && pos_old[y] > pos_old[x] && pos_new[y] < pos_new[x]) r = 1;
        p.info.is_rearr[x] = r;
        nr += r;
    }
    p.info.n_rearr = nr;
    p.relin = make_relin(N, t->dims, t->sig, new_sig);
    p.identity = p.relin.identity;
    if (nr == 0) {
        p.info.m_top = total;
        p.info.m_low = total;
        p.info.key_bits = 0;
        p.info.digit_bits = 0;
        p.info.passes = 0;
        p.info.segments = 1;
        p.key_div = make_div(1);
        *out = p;
        return LCO_OK;
    }
    int lowest = -1;
    for (int i = 0; i < N && lowest < 0; ++i)
        if (p.info.is_rearr[new_sig[i]]) lowest = i;
    int64_t m_low = 1;
    for (int i = 0; i < lowest; ++i) m_low *= t->dims[new_sig[i]];
    int64_t m_top = total;
    for (int i = N - 1; i >= 0; --i) {
        if (p.info.is_rearr[new_sig[i]]) break;
        m_top /= t->dims[new_sig[i]];
    }
    p.info.m_low = m_low;
    p.info.m_top = m_top;
    // flat LSD sort on newLIV div m_low (the region prefix stays in the key)
    const uint64_t range = (uint64_t)(total / m_low);
    int bits = 0;
    while (bits < 63 && (1ull << bits) < range) ++bits;
    int D, P;
    radix_digits(bits, &D, &P, max_digit_bits);
    p.info.key_bits = bits;
    p.info.digit_bits = D;
    p.info.passes = P;
    p.info.segments = 1;
    p.key_div = make_div((uint64_t)m_low);
    *out = p;
    return LCO_OK;
}

size_t rp_region_bytes(const RpPlan &plan, int64_t nnz) {
    if (plan.info.n_rearr == 0 || nnz == 0) return 0;
    return radix_state_bytes(nnz, plan.info.digit_bits, plan.info.passes) + 2 * align_up((size_t)nnz * 8);
}

cudaError_t rp_enqueue(const RpPlan &plan, int64_t nnz, const int64_t *in_liv, const double *in_val,
                       int64_t *out_liv, double *out_val, char *region, WsHeader *hdr,
                       cudaStream_t stream) {
    if (nnz == 0) return cudaSuccess;
    if (plan.info.n_rearr == 0) {
        cudaError_t e = cudaMemcpyAsync(out_liv, in_liv, (size_t)nnz * 8, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(out_val, in_val, (size_t)nnz * 8, cudaMemcpyDeviceToDevice, stream);
    }
    RadixJob j{};
    j.relin = plan.relin;
    j.key_div = plan.key_div;
    j.D = plan.info.digit_bits;
    j.P = plan.info.passes;
    j.n_host = nnz;
    j.n_dev = nullptr;
    j.n_cap = nnz;
    j.lsd_only = plan.lsd_only;
    j.src_liv = in_liv;
    j.src_val = in_val;
    j.dst_liv = out_liv;
    j.dst_val = out_val;
    const size_t sb = radix_state_bytes(nnz, j.D, j.P);
    j.tmp_liv = reinterpret_cast<int64_t *>(region + sb);
    j.tmp_val = reinterpret_cast<double *>(region + sb + align_up((size_t)nnz * 8));
    radix_carve(j, region);
    j.counters = hdr->counters;
    j.status = &hdr->status;
    return radix_enqueue(j, stream);
}

// ---------------------------------------------------------------------------
// Stand-alone LIV shuffle kernel: 16-byte vector loads and stores of LIV pairs.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_relin_pairs(const __grid_constant__ RelinParams p, int64_t npairs, const longlong2 *in,
                                                     longlong2 *out) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += gsz) {
        longlong2 v = in[i];
        v.x = relin(p, v.x);
        v.y = relin(p, v.y);
        out[i] = v;
    }
}

__global__ void __launch_bounds__(256) k_relin_scalar(const __grid_constant__ RelinParams p, int64_t n, const int64_t *in,
                                                      int64_t *out) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gsz)
        out[i] = relin(p, in[i]);
}

cudaError_t relin_enqueue(const RelinParams &p, int64_t n, const int64_t *in, int64_t *out,
                          cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int sms = radix_sm_count();
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (aligned) {
        const int64_t npairs = n / 2;
        if (npairs > 0) {
            int64_t grid = (npairs + 255) / 256;
            if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
            LCO_LAUNCH("k_relin_pairs", stream, k_relin_pairs<<<(unsigned)grid, 256, 0, stream>>>(p, npairs, reinterpret_cast<const longlong2 *>(in),
                                                             reinterpret_cast<longlong2 *>(out)));
        }
        if (n & 1) LCO_LAUNCH("k_relin_scalar", stream, k_relin_scalar<<<1, 32, 0, stream>>>(p, 1, in + n - 1, out + n - 1));
    } else {
        int64_t grid = (n + 255) / 256;
        if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
        LCO_LAUNCH("k_relin_scalar", stream, k_relin_scalar<<<(unsigned)grid, 256, 0, stream>>>(p, n, in, out));
    }
    return cudaGetLastError();
}

}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_relinearise(const lco_shape *t, const int32_t *new_sig, const int64_t *liv_in,
                        int64_t *liv_out, void *stream) {
    int64_t total = 0;
    int32_t rc = check_shape(t, &total);
    if (rc != LCO_OK) return rc;
    if ((rc = check_sig(t->order, new_sig)) != LCO_OK) return rc;
    if (t->nnz == 0) return LCO_OK;
    if (!liv_in || !liv_out) return LCO_ERR_INVALID;
    RelinParams p = make_relin(t->order, t->dims, t->sig, new_sig);
    return relin_enqueue(p, t->nnz, liv_in, liv_out, (cudaStream_t)stream) == cudaSuccess ? LCO_OK
                                                                                         : LCO_ERR_CUDA;
}

int32_t lco_radix_permute_info(const lco_shape *t, const int32_t *new_sig, lco_rp_info *info) {
    if (!info) return LCO_ERR_INVALID;
    RpPlan p;
    int32_t rc = rp_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    *info = p.info;
    return LCO_OK;
}

int32_t lco_radix_permute_workspace(const lco_shape *t, const int32_t *new_sig, size_t *ws_bytes) {
    if (!ws_bytes) return LCO_ERR_INVALID;
    RpPlan p;
    int32_t rc = rp_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    *ws_bytes = kWsHeaderBytes + rp_region_bytes(p, t->nnz);
    return LCO_OK;
}

int32_t lco_radix_permute(const lco_shape *t, const int32_t *new_sig, const int64_t *liv_in,
                          const double *val_in, int64_t *liv_out, double *val_out, void *ws,
                          size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_radix_permute");
    RpPlan p;
    int32_t rc = rp_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    if (t->nnz == 0) return LCO_OK;
    if (!liv_in || !val_in || !liv_out || !val_out || !ws) return LCO_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    if (ws_bytes < kWsHeaderBytes + rp_region_bytes(p, t->nnz)) return LCO_ERR_OOM;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    char *region = reinterpret_cast<char *>(ws) + kWsHeaderBytes;
    cudaError_t e = rp_enqueue(p, t->nnz, liv_in, val_in, liv_out, val_out, region, hdr,
                               (cudaStream_t)stream);
    return e == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

}  // extern "C"
