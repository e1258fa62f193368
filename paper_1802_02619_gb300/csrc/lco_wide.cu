// lco_wide.cu -- wide LIVs: re-linearisation and radix permutation of tensors
// whose dims multiply past 2^63 - 1.  Sec. 3.1 limits LIVs to signed 64 bits
// and leaves larger ones to future work (so does Sec. 7); here a wide LIV is
// an unsigned 128-bit integer stored as two uint64 words, low word first,
// and the dims multiply to at most 2^127 - 1.
//
// The permutation follows Sec. 4.1 as the 64-bit path does: the sort key is
// the new LIV without its resting suffix (the suffix is supplied by
// stability), i.e. the Horner value of the new-order modes from the lowest
// rearrangement index upward.  That key can be up to 127 bits wide; it is
// sorted least-significant chunk first, kWideChunkBits at a time, with the
// stable 64-bit radix engine (which skips constant digits) carrying each
// element's input position as payload.  A last pass gathers the new LIVs and
// the values by position.
#include <cstring>

#include "lco_host.h"

namespace lco {
namespace {

typedef unsigned __int128 u128;

constexpr int kWideChunkBits = 54;   // six 9-bit digits per chunk

struct WideShape {
    int32_t order;
    int32_t t_low;                 // key = new-order modes t_low .. order-1
    int64_t dims[kMaxOrder];
    int32_t sig_old[kMaxOrder];
    int32_t sig_new[kMaxOrder];
    DivU128by64 div[kMaxOrder];    // division of a wide LIV by each mode's dim
};

struct WidePlan {
    WideShape s;
    int32_t n_rearr;
    int32_t key_bits;
    int32_t chunks;
    int32_t D[3], P[3];            // digit plan of each chunk
    int32_t passes;                // total radix passes before skipping
};

__device__ __forceinline__ u128 load_wide(const uint64_t *p, int64_t e) {
    return ((u128)p[2 * e + 1] << 64) | (u128)p[2 * e];
}

__device__ __forceinline__ void store_wide(uint64_t *p, int64_t e, u128 x) {
    p[2 * e] = (uint64_t)x;
    p[2 * e + 1] = (uint64_t)(x >> 64);
}

// New LIV and sort key of one wide LIV (coordinates from the old order, least
// significant first; Horner from the most significant new mode).
// Each coordinate comes off with one 128-by-64 division by an invariant dim
// (a reciprocal multiply, not a software long division).
__device__ __forceinline__ void wide_relin(const WideShape &s, u128 liv, u128 &newliv, u128 &key) {
    uint64_t c[kMaxOrder];
    u128 r = liv;
    for (int t = 0; t < s.order; ++t) {
        const int m = s.sig_old[t];
        uint64_t rem;
        r = divu128(s.div[m], r, rem);
        c[m] = rem;
    }
    u128 x = 0;
    for (int t = s.order - 1; t >= 0; --t) {
        const int m = s.sig_new[t];
        x = x * (uint64_t)s.dims[m] + c[m];
        if (t == s.t_low) key = x;
    }
    newliv = x;
}

__global__ void __launch_bounds__(256) k_wide_relin(const __grid_constant__ WideShape s, int64_t n,
                                                    const uint64_t *in, uint64_t *out) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        u128 nl, key = 0;
        wide_relin(s, load_wide(in, e), nl, key);
        store_wide(out, e, nl);
    }
}

// New LIVs and full keys; the first (least significant) key chunk and the
// input positions as the radix engine's (key, payload) source.
__global__ void __launch_bounds__(256) k_wide_prep(const __grid_constant__ WideShape s, int64_t n,
                                                   const uint64_t *in, uint64_t *newliv, uint64_t *keyw,
                                                   int64_t *chunk, double *pos) {
    const uint64_t mask = (1ull << kWideChunkBits) - 1;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256) {
        u128 nl, key = 0;
        wide_relin(s, load_wide(in, e), nl, key);
        store_wide(newliv, e, nl);
        store_wide(keyw, e, key);
        chunk[e] = (int64_t)((uint64_t)key & mask);
        pos[e] = __longlong_as_double((long long)e);
    }
}

// Chunk `c` of every key, in the order the previous chunks' sorts left the
// elements (pos holds each element's input position).
__global__ void __launch_bounds__(256) k_wide_chunk(int64_t n, const uint64_t *keyw, const double *pos_in,
                                                    int shift, int64_t *chunk, double *pos_out) {
    const uint64_t mask = (1ull << kWideChunkBits) - 1;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double p = pos_in[i];
        int64_t e = (int64_t)__double_as_longlong(p);
        if ((uint64_t)e >= (uint64_t)n) e = 0;   // positions are a permutation of [0, n); never read outside
        chunk[i] = (int64_t)((uint64_t)(load_wide(keyw, e) >> shift) & mask);
        pos_out[i] = p;
    }
}

__global__ void __launch_bounds__(256) k_wide_gather(int64_t n, const uint64_t *newliv, const double *val,
                                                     const double *pos, uint64_t *out_liv, double *out_val) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        int64_t e = (int64_t)__double_as_longlong(pos[i]);
        if ((uint64_t)e >= (uint64_t)n) e = 0;   // as in k_wide_chunk
        out_liv[2 * i] = newliv[2 * e];
        out_liv[2 * i + 1] = newliv[2 * e + 1];
        out_val[i] = val[e];
    }
}

unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)radix_sm_count() * 8;
    if (g > cap) g = cap;
    return (unsigned)(g > 0 ? g : 1);
}

int32_t check_wide_shape(const lco_shape *t, u128 *total) {
    if (t == nullptr) return LCO_ERR_INVALID;
    int32_t rc = check_sig(t->order, t->sig);
    if (rc != LCO_OK) return rc;
    if (t->nnz < 0) return LCO_ERR_INVALID;
    const u128 lim = ((u128)1 << 127) - 1;
    u128 p = 1;
    for (int i = 0; i < t->order; ++i) {
        if (t->dims[i] < 1) return LCO_ERR_INVALID;
        if (p > lim / (u128)(uint64_t)t->dims[i]) return LCO_ERR_OVERFLOW;
        p *= (u128)(uint64_t)t->dims[i];
    }
    if (total) *total = p;
    return LCO_OK;
}

int32_t wide_plan(const lco_shape *t, const int32_t *new_sig, WidePlan *out) {
    u128 total = 0;
    int32_t rc = check_wide_shape(t, &total);
    if (rc != LCO_OK) return rc;
    if ((rc = check_sig(t->order, new_sig)) != LCO_OK) return rc;
    const int N = t->order;
    WidePlan p{};
    p.s.order = N;
    int pos_old[kMaxOrder], pos_new[kMaxOrder];
    for (int i = 0; i < N; ++i) {
        p.s.dims[i] = t->dims[i];
        p.s.div[i] = make_div128((uint64_t)t->dims[i]);
        p.s.sig_old[i] = t->sig[i];
        p.s.sig_new[i] = new_sig[i];
        pos_old[t->sig[i]] = i;
        pos_new[new_sig[i]] = i;
    }
    // Sec. 4.1: x is a rearrangement index when some index that was more
    // significant than x becomes less significant than it
    int is_rearr[kMaxOrder] = {0};
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            if (y != x && pos_old[y] > pos_old[x] && pos_new[y] < pos_new[x]) is_rearr[x] = 1;
    for (int x = 0; x < N; ++x) p.n_rearr += is_rearr[x];
    p.s.t_low = 0;
    if (p.n_rearr > 0) {
        while (!is_rearr[new_sig[p.s.t_low]]) ++p.s.t_low;
        u128 range = 1;
        for (int i = p.s.t_low; i < N; ++i) range *= (u128)(uint64_t)t->dims[new_sig[i]];
        int bits = 0;
        while (bits < 127 && ((u128)1 << bits) < range) ++bits;
        // A key range of 1 (every new-order mode from t_low up has dim 1)
        // still takes one chunk: its single pass is constant and becomes the
        // engine's copy, which writes the positions the gather reads.
        if (bits < 1) bits = 1;
        p.key_bits = bits;
        p.chunks = (bits + kWideChunkBits - 1) / kWideChunkBits;
        for (int c = 0; c < p.chunks; ++c) {
            const int cb = bits - c * kWideChunkBits < kWideChunkBits ? bits - c * kWideChunkBits : kWideChunkBits;
            radix_digits(cb, &p.D[c], &p.P[c]);
            p.passes += p.P[c];
        }
    }
    *out = p;
    return LCO_OK;
}

struct WideLayout {
    size_t newliv, keyw, chunk_a, pos_a, chunk_b, pos_b, tmp_liv, tmp_val, radix, total;
};

WideLayout wide_layout(const WidePlan &p, int64_t n) {
    WideLayout L{};
    size_t off = kWsHeaderBytes;
    auto take = [&](size_t b) { const size_t o = off; off += align_up(b); return o; };
    L.newliv = take((size_t)n * 16);
    L.keyw = take((size_t)n * 16);
    L.chunk_a = take((size_t)n * 8);
    L.pos_a = take((size_t)n * 8);
    L.chunk_b = take((size_t)n * 8);
    L.pos_b = take((size_t)n * 8);
    L.tmp_liv = take((size_t)n * 8);
    L.tmp_val = take((size_t)n * 8);
    size_t rb = 0;
    for (int c = 0; c < p.chunks; ++c) {
        const size_t b = radix_state_bytes(n, p.D[c], p.P[c]);
        if (b > rb) rb = b;
    }
    L.radix = take(rb);
    L.total = off;
    return L;
}

}  // namespace
}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_relinearise_wide(const lco_shape *t, const int32_t *new_sig, const uint64_t *liv_in,
                             uint64_t *liv_out, void *stream) {
    NvtxRange nvtx("lco_relinearise_wide");
    WidePlan p;
    int32_t rc = wide_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    if (t->nnz == 0) return LCO_OK;
    if (!liv_in || !liv_out) return LCO_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    LCO_LAUNCH("k_wide_relin", s, k_wide_relin<<<grid_for(t->nnz), 256, 0, s>>>(p.s, t->nnz, liv_in, liv_out));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

int32_t lco_radix_permute_wide_info(const lco_shape *t, const int32_t *new_sig, lco_rp_wide_info *info) {
    if (!info) return LCO_ERR_INVALID;
    WidePlan p;
    int32_t rc = wide_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    info->n_rearr = p.n_rearr;
    info->key_bits = p.key_bits;
    info->chunks = p.chunks;
    info->passes = p.passes;
    return LCO_OK;
}

int32_t lco_radix_permute_wide_workspace(const lco_shape *t, const int32_t *new_sig, size_t *ws_bytes) {
    if (!ws_bytes) return LCO_ERR_INVALID;
    WidePlan p;
    int32_t rc = wide_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    *ws_bytes = wide_layout(p, t->nnz).total;
    return LCO_OK;
}

int32_t lco_radix_permute_wide(const lco_shape *t, const int32_t *new_sig, const uint64_t *liv_in,
                               const double *val_in, uint64_t *liv_out, double *val_out, void *ws,
                               size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_radix_permute_wide");
    WidePlan p;
    int32_t rc = wide_plan(t, new_sig, &p);
    if (rc != LCO_OK) return rc;
    const int64_t n = t->nnz;
    if (n == 0) return LCO_OK;
    if (!liv_in || !val_in || !liv_out || !val_out || !ws) return LCO_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    const WideLayout L = wide_layout(p, n);
    if (ws_bytes < L.total) return LCO_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    if (p.n_rearr == 0) {
        // same order: the LIVs and values are unchanged
        if (cudaMemcpyAsync(liv_out, liv_in, (size_t)n * 16, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(val_out, val_in, (size_t)n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return LCO_ERR_CUDA;
        return LCO_OK;
    }
    char *w = reinterpret_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    uint64_t *newliv = reinterpret_cast<uint64_t *>(w + L.newliv);
    uint64_t *keyw = reinterpret_cast<uint64_t *>(w + L.keyw);
    int64_t *chunk_a = reinterpret_cast<int64_t *>(w + L.chunk_a);
    double *pos_a = reinterpret_cast<double *>(w + L.pos_a);
    int64_t *chunk_b = reinterpret_cast<int64_t *>(w + L.chunk_b);
    double *pos_b = reinterpret_cast<double *>(w + L.pos_b);
    const unsigned g = grid_for(n);
    LCO_LAUNCH("k_wide_prep", s, k_wide_prep<<<g, 256, 0, s>>>(p.s, n, liv_in, newliv, keyw, chunk_a, pos_a));
    for (int c = 0; c < p.chunks; ++c) {
        if (c > 0)
            LCO_LAUNCH("k_wide_chunk", s, k_wide_chunk<<<g, 256, 0, s>>>(n, keyw, pos_b, c * kWideChunkBits,
                                                                          chunk_a, pos_a));
        // stable sort of (chunk c, position), the result in (chunk_b, pos_b)
        RadixJob j{};
        j.relin.nseg = 1;
        j.relin.identity = 1;
        j.key_div = make_div(1);
        j.D = p.D[c];
        j.P = p.P[c];
        j.n_host = n;
        j.n_dev = nullptr;
        j.n_cap = n;
        j.src_liv = chunk_a;
        j.src_val = pos_a;
        j.dst_liv = chunk_b;
        j.dst_val = pos_b;
        j.tmp_liv = reinterpret_cast<int64_t *>(w + L.tmp_liv);
        j.tmp_val = reinterpret_cast<double *>(w + L.tmp_val);
        radix_carve(j, w + L.radix);
        j.counters = hdr->counters;
        j.status = &hdr->status;
        if (radix_enqueue(j, s) != cudaSuccess) return LCO_ERR_CUDA;
    }
    LCO_LAUNCH("k_wide_gather", s, k_wide_gather<<<g, 256, 0, s>>>(n, newliv, val_in, pos_b, liv_out, val_out));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

}  // extern "C"
