// lco_arith.cu -- sorting and addition of LCO tensors (Sec. 3.2; the sum of
// Eq. 4 after one term is re-sorted into the other's order).
//
// Sorting runs the radix engine of the permutation on the whole LIV with
// the identity re-linearisation: every digit is a sort digit (the engine
// still skips digits that are constant over the data).  Addition is a
// stable merge of the two sorted inputs (A first on equal LIVs) split by
// merge path, in which each run of equal LIVs -- at most one entry from
// each input -- becomes one entry of C; tiles of the merged sequence place
// their entries with decoupled look-back.
#include "lco_host.h"

namespace lco {
namespace {

constexpr int kAddThreads = 256;
constexpr int kAddItems = 8;
constexpr int kAddTile = kAddThreads * kAddItems;
constexpr int kAddWarps = kAddThreads / 32;

struct AddArgs {
    const int64_t *a_liv;
    const double *a_val;
    int64_t na;
    const int64_t *b_liv;
    const double *b_val;
    int64_t nb;
    double alpha, beta;
    int64_t *c_liv;
    double *c_val;
    uint64_t *state;     // look-back words, one per tile
    WsHeader *hdr;
};

// Number of A entries among the first d entries of the merged sequence.
__device__ __forceinline__ int64_t merge_split(const AddArgs &a, int64_t d) {
    int64_t lo = d > a.nb ? d - a.nb : 0, hi = d < a.na ? d : a.na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.a_liv[mid] <= a.b_liv[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kAddThreads) k_add(const __grid_constant__ AddArgs a) {
    __shared__ int64_t s_warp[kAddWarps + 1];
    __shared__ int64_t s_tile, s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = a.na + a.nb;
    if (tid == 0) s_tile = atomicAdd(&a.hdr->counters[0], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t ntiles = (n + kAddTile - 1) / kAddTile;
    if (tile >= ntiles) return;
    // this thread's positions p0..p0+7, with the one before and the one after
    const int64_t p0 = tile * kAddTile + (int64_t)tid * kAddItems;
    const int off = p0 > 0 ? 1 : 0;
    const int64_t d0 = p0 - off;
    int64_t ia = d0 < n ? merge_split(a, d0) : a.na;
    int64_t ib = d0 < n ? d0 - ia : a.nb;
    int64_t key[kAddItems + 2];
    double val[kAddItems + 2];
#pragma unroll
    for (int t = 0; t < kAddItems + 2; ++t) {
        key[t] = -1;
        val[t] = 0.0;
        if (ia < a.na && (ib >= a.nb || a.a_liv[ia] <= a.b_liv[ib])) {
            key[t] = a.a_liv[ia];
            val[t] = __dmul_rn(a.alpha, a.a_val[ia]);
            ++ia;
        } else if (ib < a.nb) {
            key[t] = a.b_liv[ib];
            val[t] = __dmul_rn(a.beta, a.b_val[ib]);
            ++ib;
        }
    }
    // an entry of C starts where the LIV differs from the one before
    // (static indices only: `off` selects between neighbours)
    unsigned heads = 0;
#pragma unroll
    for (int i = 0; i < kAddItems; ++i) {
        const int64_t cur = off ? key[i + 1] : key[i];
        const int64_t prev = off ? key[i] : (i > 0 ? key[i - 1] : -1);
        if (p0 + i < n && cur != prev) heads |= 1u << i;
    }
    // block exclusive scan of the head counts
    int64_t x = __popc(heads);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = lane < kAddWarps ? s_warp[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kAddWarps) s_warp[lane] = wi - w;
        if (lane == kAddWarps - 1) s_warp[kAddWarps] = wi;
    }
    __syncthreads();
    const int64_t tot = s_warp[kAddWarps];
    int64_t o = s_warp[warp] + x - __popc(heads);
    if (warp == 0) {
        if (lane == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
        int64_t pre = 0;
        if (tile > 0) pre = (int64_t)lookback_warp(a.state, tile, &a.hdr->status);
        if (lane == 0) {
            if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(pre + tot));
            s_excl = pre;
            if (tile == ntiles - 1) a.hdr->nnz_c = pre + tot;
        }
    }
    __syncthreads();
    o += s_excl;
#pragma unroll
    for (int i = 0; i < kAddItems; ++i) {
        if ((heads >> i) & 1u) {
            const int64_t cur = off ? key[i + 1] : key[i];
            const int64_t nxt = off ? key[i + 2] : key[i + 1];
            const double vc = off ? val[i + 1] : val[i];
            const double vn = off ? val[i + 2] : val[i + 1];
            const double v = nxt == cur ? __dadd_rn(vc, vn) : vc;
            a.c_liv[o] = cur;
            a.c_val[o] = v;
            ++o;
        }
    }
}

size_t add_state_bytes(int64_t n) { return align_up((size_t)((n + kAddTile - 1) / kAddTile + 2) * 8); }

int32_t sort_plan(const lco_shape *t, RpPlan *out) {
    int64_t total = 0;
    int32_t rc = check_shape(t, &total);
    if (rc != LCO_OK) return rc;
    RpPlan p{};
    p.total = total;
    p.relin = make_relin(t->order, t->dims, t->sig, t->sig);
    p.identity = 1;
    p.info.n_rearr = t->order;               // every digit is a sort digit
    for (int i = 0; i < t->order; ++i) p.info.is_rearr[i] = 1;
    p.info.m_low = 1;
    p.info.m_top = total;
    int bits = 0;
    while (bits < 63 && (1ull << bits) < (uint64_t)total) ++bits;
    int D, P;
    radix_digits(bits > 0 ? bits : 1, &D, &P);
    p.info.key_bits = bits;
    p.info.digit_bits = D;
    p.info.passes = P;
    p.info.segments = 1;
    p.key_div = make_div(1);
    *out = p;
    return LCO_OK;
}

}  // namespace
}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_sort_workspace(const lco_shape *t, size_t *ws_bytes) {
    if (!t || !ws_bytes) return LCO_ERR_INVALID;
    RpPlan p;
    const int32_t rc = sort_plan(t, &p);
    if (rc != LCO_OK) return rc;
    if (t->nnz < 0) return LCO_ERR_INVALID;
    *ws_bytes = kWsHeaderBytes + rp_region_bytes(p, t->nnz);
    return LCO_OK;
}

int32_t lco_sort(const lco_shape *t, const int64_t *in_liv, const double *in_val, int64_t *out_liv, double *out_val,
                 void *ws, size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_sort");
    if (!t || !ws) return LCO_ERR_INVALID;
    RpPlan p;
    int32_t rc = sort_plan(t, &p);
    if (rc != LCO_OK) return rc;
    if (t->nnz < 0 || (t->nnz > 0 && (!in_liv || !in_val || !out_liv || !out_val))) return LCO_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    const size_t region = rp_region_bytes(p, t->nnz);
    if (ws_bytes < kWsHeaderBytes + region) return LCO_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = reinterpret_cast<char *>(ws);
    // header, and the radix engine's histogram table, must start zeroed
    const size_t zero = kWsHeaderBytes + (region > 0 ? radix_hist_table_bytes() : 0);
    if (cudaMemsetAsync(w, 0, zero, s) != cudaSuccess) return LCO_ERR_CUDA;
    if (t->nnz == 0) return LCO_OK;
    return rp_enqueue(p, t->nnz, in_liv, in_val, out_liv, out_val, w + kWsHeaderBytes,
                      reinterpret_cast<WsHeader *>(w), s) == cudaSuccess
               ? LCO_OK
               : LCO_ERR_CUDA;
}

int32_t lco_add_workspace(int64_t nnz_a, int64_t nnz_b, size_t *ws_bytes) {
    if (!ws_bytes || nnz_a < 0 || nnz_b < 0) return LCO_ERR_INVALID;
    *ws_bytes = kWsHeaderBytes + add_state_bytes(nnz_a + nnz_b);
    return LCO_OK;
}

int32_t lco_add(const lco_shape *t, double alpha, const int64_t *a_liv, const double *a_val, int64_t nnz_a,
                double beta, const int64_t *b_liv, const double *b_val, int64_t nnz_b, int64_t *c_liv, double *c_val,
                void *ws, size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_add");
    if (!t || !ws || nnz_a < 0 || nnz_b < 0) return LCO_ERR_INVALID;
    int64_t total = 0;
    const int32_t rc = check_shape(t, &total);
    if (rc != LCO_OK) return rc;
    if ((nnz_a > 0 && (!a_liv || !a_val)) || (nnz_b > 0 && (!b_liv || !b_val))) return LCO_ERR_INVALID;
    if (nnz_a + nnz_b > 0 && (!c_liv || !c_val)) return LCO_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    const int64_t n = nnz_a + nnz_b;
    const size_t sb = add_state_bytes(n);
    if (ws_bytes < kWsHeaderBytes + sb) return LCO_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = reinterpret_cast<char *>(ws);
    if (cudaMemsetAsync(w, 0, kWsHeaderBytes + sb, s) != cudaSuccess) return LCO_ERR_CUDA;   // nnz_c = 0 when n = 0
    if (n == 0) return LCO_OK;
    AddArgs a{};
    a.a_liv = a_liv;
    a.a_val = a_val;
    a.na = nnz_a;
    a.b_liv = b_liv;
    a.b_val = b_val;
    a.nb = nnz_b;
    a.alpha = alpha;
    a.beta = beta;
    a.c_liv = c_liv;
    a.c_val = c_val;
    a.state = reinterpret_cast<uint64_t *>(w + kWsHeaderBytes);
    a.hdr = reinterpret_cast<WsHeader *>(w);
    const int64_t tiles = (n + kAddTile - 1) / kAddTile;
    LCO_LAUNCH("k_add", s, k_add<<<(unsigned)tiles, kAddThreads, 0, s>>>(a));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

int32_t lco_add_result(const void *ws, int64_t *nnz_c, int32_t *status, void *stream) {
    if (!ws || !nnz_c) return LCO_ERR_INVALID;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCO_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(WsHeader), cudaMemcpyDeviceToHost) != cudaSuccess) return LCO_ERR_CUDA;
    *nnz_c = h.nnz_c;
    if (status) *status = h.status;
    return LCO_OK;
}

}  // extern "C"
