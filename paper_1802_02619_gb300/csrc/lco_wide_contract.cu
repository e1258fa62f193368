// lco_wide_contract.cu -- contraction of tensors with wide (128-bit) LIVs.
//
// Sec. 3.1 keeps LIVs within 2^63 - 1 and leaves larger index spaces to
// future work (so does Sec. 7).  A product of wide tensors has the same
// definition as Sec. 5's: C[i, j] = sum_k A[i, k] B[k, j] over the
// matricised operands, with row, contracted and column indices that may
// each need up to 127 bits.  The GPU path keeps the 64-bit contraction and
// changes only the indices it sees:
//   1. A and B are permuted (wide radix permutation, Sec. 4.1) into their
//      matrix orders: A's free modes most significant, B's contracted modes
//      most significant;
//   2. every index is replaced by its rank among the distinct values that
//      occur -- A's row keys (sorted already), B's contracted keys (sorted
//      already; an A entry whose contracted key B lacks meets nothing and is
//      dropped) and B's column keys (sorted with the radix engine in 54-bit
//      chunks) -- so the matrices become at most nnz_A x (nnz_B + 1) and
//      (nnz_B + 1) x nnz_B;
//   3. the 64-bit contraction multiplies the rank matrices (any Table-4
//      branch: every branch sums in the same order);
//   4. each entry of the product maps back to row key * n + column key.
// Ranks keep the order of the keys, so the rank matrices and the product
// are sorted LCO tensors and C comes out sorted in row-major order of (A's
// free modes, B's free modes).  The rank matrices have a fixed shape known
// on the host: dropped entries of A are replaced at the end by entries in
// rows past the real ones meeting B's empty last row, so no count crosses
// back to the host before the inner plan runs.
#include <cstring>
#include <new>

#include "lco_host.h"

namespace lco {
namespace {

typedef unsigned __int128 u128;

constexpr int kWT = 256;                        // threads of the element kernels
constexpr int kScanItems = 8;
constexpr int kScanTile = kWT * kScanItems;     // scan tile (elements)
constexpr int kChunkBits = 54;                  // radix chunk of a wide key

__device__ __forceinline__ u128 ld128(const uint64_t *p, int64_t e) {
    return ((u128)p[2 * e + 1] << 64) | (u128)p[2 * e];
}
__device__ __forceinline__ void st128(uint64_t *p, int64_t e, u128 x) {
    p[2 * e] = (uint64_t)x;
    p[2 * e + 1] = (uint64_t)(x >> 64);
}

struct Div128 {   // a 128-bit divisor, kept as two words so the struct is a plain kernel argument
    uint64_t lo, hi;
};
__host__ __device__ __forceinline__ u128 val128(const Div128 &d) { return ((u128)d.hi << 64) | (u128)d.lo; }
inline Div128 mk128(u128 x) { return Div128{(uint64_t)x, (uint64_t)(x >> 64)}; }

// Row and column keys of a matrix-ordered wide LIV: x = key_hi * div + key_lo.
__global__ void __launch_bounds__(kWT) k_wide_split(int64_t n, const uint64_t *liv, Div128 div, uint64_t *hi_out,
                                                    uint64_t *lo_out) {
    const u128 d = val128(div);
    for (int64_t e = (int64_t)blockIdx.x * kWT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kWT) {
        const u128 x = ld128(liv, e);
        const u128 q = x / d;
        st128(hi_out, e, q);
        st128(lo_out, e, x - q * d);
    }
}

// Head flag of element i of a key sequence read through an optional
// permutation (pos: position of the i-th element, stored as double bits).
__device__ __forceinline__ int64_t pos_at(const double *pos, int64_t i, int64_t n) {
    if (!pos) return i;
    int64_t e = (int64_t)__double_as_longlong(pos[i]);
    return (uint64_t)e < (uint64_t)n ? e : 0;   // positions are a permutation of [0, n)
}

// Ranks of a non-decreasing key sequence (keys[pos[i]], i ascending): rank[i]
// = number of distinct keys before it.  Single-pass scan over the head
// flags with decoupled look-back; the heads also record their key in
// of_rank[rank], and the last tile writes the distinct count.  With pos,
// rank is scattered to rank[pos[i]].
struct RankArgs {
    int64_t n;
    const uint64_t *keys;     // wide keys
    const double *pos;        // optional order of the keys
    int64_t *rank;            // out, per element (by position)
    uint64_t *of_rank;        // out, wide key of each rank
    int64_t *count;           // out, number of distinct keys
    uint64_t *state;          // look-back words, zeroed
    uint32_t *tile_ctr;       // zeroed
    int32_t *status;
};

__global__ void __launch_bounds__(kWT) k_wide_rank(const __grid_constant__ RankArgs a) {
    __shared__ int64_t s_warp[kWT / 32 + 1];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t heads = 0;
    int64_t cnt = 0;
    u128 prev = 0;
    if (base > 0 && base - 1 < a.n) prev = ld128(a.keys, pos_at(a.pos, base - 1, a.n));
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < a.n) {
            const u128 k = ld128(a.keys, pos_at(a.pos, e, a.n));
            if (e == 0 || k != prev) {
                heads |= 1u << i;
                ++cnt;
            }
            prev = k;
        }
    }
    int64_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int64_t wex = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kWT / 32; ++w) {
        wex += w < warp ? s_warp[w] : 0;
        tot += s_warp[w];
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
        int64_t ex = 0;
        if (tile > 0) ex = (int64_t)lookback_warp(a.state, tile, a.status);
        if (lane == 0) {
            if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(ex + tot));
            s_warp[kWT / 32] = ex;
            const int64_t ntiles = (a.n + kScanTile - 1) / kScanTile;
            if (tile == ntiles - 1) *a.count = ex + tot;
        }
    }
    __syncthreads();
    int64_t r = s_warp[kWT / 32] + wex + x - cnt;   // distinct keys before this thread's first element
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < a.n) {
            const int64_t p = pos_at(a.pos, e, a.n);
            if (heads & (1u << i)) {
                st128(a.of_rank, r, ld128(a.keys, p));
                ++r;
            }
            a.rank[p] = r - 1;
        }
    }
}

// First chunk of every key and the identity positions (radix source).
__global__ void __launch_bounds__(kWT) k_wide_key_prep(int64_t n, const uint64_t *keys, int64_t *chunk, double *pos) {
    const uint64_t mask = (1ull << kChunkBits) - 1;
    for (int64_t e = (int64_t)blockIdx.x * kWT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kWT) {
        chunk[e] = (int64_t)(keys[2 * e] & mask);
        pos[e] = __longlong_as_double((long long)e);
    }
}

// Chunk `shift` of every key, in the order the earlier chunks' sorts left.
__global__ void __launch_bounds__(kWT) k_wide_key_chunk(int64_t n, const uint64_t *keys, const double *pos_in,
                                                        int shift, int64_t *chunk, double *pos_out) {
    const uint64_t mask = (1ull << kChunkBits) - 1;
    for (int64_t i = (int64_t)blockIdx.x * kWT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kWT) {
        const double p = pos_in[i];
        const int64_t e = pos_at(pos_in, i, n);
        chunk[i] = (int64_t)((uint64_t)(ld128(keys, e) >> shift) & mask);
        pos_out[i] = p;
    }
}

// A' (ranks): A entries whose contracted key B has, at (row rank, key rank);
// the others (they meet no B row) are dropped, and as many entries are
// appended past the real rows in B's empty last row, so that A' always has
// nnz_A entries.  keep[e] = 1 for kept entries (scanned into positions).
__device__ __forceinline__ int64_t find_key(const uint64_t *sorted, int64_t m, u128 k) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ld128(sorted, mid) < k) lo = mid + 1; else hi = mid;
    }
    return (lo < m && ld128(sorted, lo) == k) ? lo : -1;
}

__global__ void __launch_bounds__(kWT) k_wide_a_keep(int64_t n, const uint64_t *colkey, const uint64_t *bkeys,
                                                     const int64_t *nbkeys, int64_t *krank) {
    const int64_t m = *nbkeys;
    for (int64_t e = (int64_t)blockIdx.x * kWT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kWT)
        krank[e] = find_key(bkeys, m, ld128(colkey, e));
}

// Exclusive positions of the kept entries, from a scan of keep flags
// (krank >= 0), and the A' entries: kept ones at their positions, fillers
// after them.
struct BuildA {
    int64_t n;
    const int64_t *row_rank;
    const int64_t *krank;
    const double *val;
    int64_t Kp;              // A' columns (= B' rows)
    int64_t Mhalf;           // first filler row
    int64_t *out_liv;
    double *out_val;
    uint64_t *state;
    uint32_t *tile_ctr;
    int64_t *nkeep;
    int32_t *status;
};

__global__ void __launch_bounds__(kWT) k_wide_a_build(const __grid_constant__ BuildA a) {
    __shared__ int64_t s_warp[kWT / 32 + 1];
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) cnt += (base + i < a.n && a.krank[base + i] >= 0);
    int64_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    int64_t wex = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kWT / 32; ++w) {
        wex += w < warp ? s_warp[w] : 0;
        tot += s_warp[w];
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
        int64_t ex = 0;
        if (tile > 0) ex = (int64_t)lookback_warp(a.state, tile, a.status);
        if (lane == 0) {
            if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(ex + tot));
            s_warp[kWT / 32] = ex;
            const int64_t ntiles = (a.n + kScanTile - 1) / kScanTile;
            if (tile == ntiles - 1) *a.nkeep = ex + tot;
        }
    }
    __syncthreads();
    int64_t o = s_warp[kWT / 32] + wex + x - cnt;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < a.n && a.krank[e] >= 0) {
            a.out_liv[o] = a.row_rank[e] * a.Kp + a.krank[e];
            a.out_val[o] = a.val[e];
            ++o;
        }
    }
}

__global__ void __launch_bounds__(kWT) k_wide_a_fill(int64_t n, const int64_t *nkeep, int64_t Kp, int64_t Mhalf,
                                                     int64_t *out_liv, double *out_val) {
    const int64_t k = *nkeep;
    for (int64_t e = k + (int64_t)blockIdx.x * kWT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kWT) {
        out_liv[e] = (Mhalf + (e - k)) * Kp + (Kp - 1);
        out_val[e] = 0.0;
    }
}

// B' (ranks): (contracted-key rank, column-key rank).
__global__ void __launch_bounds__(kWT) k_wide_b_build(int64_t n, const int64_t *krank, const int64_t *crank,
                                                      const double *val, int64_t Np, int64_t *out_liv,
                                                      double *out_val) {
    for (int64_t e = (int64_t)blockIdx.x * kWT + threadIdx.x; e < n; e += (int64_t)gridDim.x * kWT) {
        out_liv[e] = krank[e] * Np + crank[e];
        out_val[e] = val[e];
    }
}

// C from the rank product: row key * n + column key.
__global__ void __launch_bounds__(kWT) k_wide_c_map(const WsHeader *inner, DivU64 div_np, const uint64_t *row_of,
                                                    const uint64_t *col_of, Div128 nB, const int64_t *c_liv,
                                                    const double *c_val, int64_t cap, uint64_t *out_liv,
                                                    double *out_val) {
    if (inner->status != 0 || inner->f > cap) return;
    const int64_t nc = inner->nnz_c;
    const u128 n = val128(nB);
    for (int64_t i = (int64_t)blockIdx.x * kWT + threadIdx.x; i < nc; i += (int64_t)gridDim.x * kWT) {
        const uint64_t l = (uint64_t)c_liv[i];
        const uint64_t ra = divu(div_np, l);
        const uint64_t rb = l - ra * div_np.d;
        st128(out_liv, i, ld128(row_of, (int64_t)ra) * n + ld128(col_of, (int64_t)rb));
        out_val[i] = c_val[i];
    }
}

unsigned grid_of(int64_t n) {
    int64_t g = (n + kWT - 1) / kWT;
    const int64_t cap = (int64_t)radix_sm_count() * 8;
    if (g > cap) g = cap;
    return (unsigned)(g > 0 ? g : 1);
}

int bits128(u128 range) {
    int b = 0;
    while (b < 127 && ((u128)1 << b) < range) ++b;
    return b;
}

}  // namespace
}  // namespace lco

struct lco_wide_plan {
    lco_shape a, b;               // operand shapes (wide: dims multiply past 2^63 - 1 allowed)
    int32_t ncontract;
    int32_t modes_a[LCO_MAX_ORDER], modes_b[LCO_MAX_ORDER];
    int32_t sig_am[LCO_MAX_ORDER], sig_bm[LCO_MAX_ORDER];   // matrix orders
    int32_t perm_a, perm_b;       // 1: the operand needs the wide permutation
    lco::u128 kc, mA, nB;         // contracted, A-free and B-free index ranges
    int32_t col_bits;             // bits of B's column keys
    int64_t Mp, Kp, Np;           // rank-matrix shapes
    lco_plan *inner;              // the 64-bit contraction of the rank matrices
    lco_shape c_shape;            // C's modes (A free, B free), row-major; nnz 0
    size_t perm_ws;               // wide permutation workspace (largest of the two)
    // workspace layout (offsets from the base)
    size_t o_am_liv, o_am_val, o_bm_liv, o_bm_val, o_perm;
    size_t o_a_row, o_a_col, o_a_rrank, o_a_krank, o_row_of;
    size_t o_b_key, o_b_col, o_b_krank, o_b_crank, o_key_of, o_col_of;
    size_t o_chunk_a, o_pos_a, o_chunk_b, o_pos_b, o_tmp_l, o_tmp_v, o_radix;
    size_t o_state, state_bytes, o_counts;
    size_t o_ap_liv, o_ap_val, o_bp_liv, o_bp_val;
    size_t o_inner, o_cp_liv, o_cp_val;   // cap-dependent from o_inner on
    size_t radix_bytes;
};

namespace lco {
namespace {

constexpr int kNumScans = 4;   // look-back regions: A rows, B keys, B columns, A' positions

size_t wide_layout(lco_wide_plan *p, int64_t cap) {
    const int64_t na = p->a.nnz > 0 ? p->a.nnz : 1, nb = p->b.nnz > 0 ? p->b.nnz : 1;
    size_t off = kWsHeaderBytes;
    auto take = [&](size_t b) { const size_t o = off; off += align_up(b ? b : 1); return o; };
    p->o_am_liv = p->perm_a ? take((size_t)na * 16) : 0;
    p->o_am_val = p->perm_a ? take((size_t)na * 8) : 0;
    p->o_bm_liv = p->perm_b ? take((size_t)nb * 16) : 0;
    p->o_bm_val = p->perm_b ? take((size_t)nb * 8) : 0;
    p->o_perm = take(p->perm_ws);
    p->o_a_row = take((size_t)na * 16);
    p->o_a_col = take((size_t)na * 16);
    p->o_a_rrank = take((size_t)na * 8);
    p->o_a_krank = take((size_t)na * 8);
    p->o_row_of = take((size_t)na * 16);
    p->o_b_key = take((size_t)nb * 16);
    p->o_b_col = take((size_t)nb * 16);
    p->o_b_krank = take((size_t)nb * 8);
    p->o_b_crank = take((size_t)nb * 8);
    p->o_key_of = take((size_t)nb * 16);
    p->o_col_of = take((size_t)nb * 16);
    p->o_chunk_a = take((size_t)nb * 8);
    p->o_pos_a = take((size_t)nb * 8);
    p->o_chunk_b = take((size_t)nb * 8);
    p->o_pos_b = take((size_t)nb * 8);
    p->o_tmp_l = take((size_t)nb * 8);
    p->o_tmp_v = take((size_t)nb * 8);
    p->o_radix = take(p->radix_bytes);
    const int64_t nmax = na > nb ? na : nb;
    // look-back words of the scans, then their tile counters (64 bytes)
    p->state_bytes = align_up((size_t)kNumScans * (size_t)((nmax + kScanTile - 1) / kScanTile + 1) * 8 + 64);
    p->o_state = take(p->state_bytes);
    p->o_counts = take(64);
    p->o_ap_liv = take((size_t)na * 8);
    p->o_ap_val = take((size_t)na * 8);
    p->o_bp_liv = take((size_t)nb * 8);
    p->o_bp_val = take((size_t)nb * 8);
    p->o_inner = off;
    size_t inner_bytes = 0;
    lco_contract_workspace(p->inner, cap < 0 ? 0 : cap, &inner_bytes);
    take(inner_bytes);
    const int64_t c = cap > 0 ? cap : 1;
    p->o_cp_liv = take((size_t)c * 8);
    p->o_cp_val = take((size_t)c * 8);
    return off;
}

int32_t wide_shape_check(const lco_shape *t, u128 *total) {
    if (!t) return LCO_ERR_INVALID;
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
    *total = p;
    return LCO_OK;
}

bool same_order(int order, const int32_t *x, const int32_t *y) {
    for (int i = 0; i < order; ++i)
        if (x[i] != y[i]) return false;
    return true;
}

// Zeroed look-back region r of a call.
uint64_t *scan_region(const lco_wide_plan *p, char *w, int r) {
    const int64_t na = p->a.nnz > 0 ? p->a.nnz : 1, nb = p->b.nnz > 0 ? p->b.nnz : 1;
    const int64_t nmax = na > nb ? na : nb;
    return reinterpret_cast<uint64_t *>(w + p->o_state) + (size_t)r * (size_t)((nmax + kScanTile - 1) / kScanTile + 1);
}

}  // namespace
}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_contract_wide_plan(const lco_shape *a, const lco_shape *b, int32_t ncontract, const int32_t *modes_a,
                               const int32_t *modes_b, lco_wide_plan **out) {
    if (!out) return LCO_ERR_INVALID;
    *out = nullptr;
    u128 ta, tb;
    int32_t rc;
    if ((rc = wide_shape_check(a, &ta)) != LCO_OK) return rc;
    if ((rc = wide_shape_check(b, &tb)) != LCO_OK) return rc;
    if (ncontract < 0 || ncontract > a->order || ncontract > b->order) return LCO_ERR_INVALID;
    if (ncontract > 0 && (!modes_a || !modes_b)) return LCO_ERR_INVALID;
    int con_a[kMaxOrder] = {0}, con_b[kMaxOrder] = {0};
    for (int i = 0; i < ncontract; ++i) {
        const int ma = modes_a[i], mb = modes_b[i];
        if (ma < 0 || ma >= a->order || mb < 0 || mb >= b->order || con_a[ma] || con_b[mb]) return LCO_ERR_INVALID;
        if (a->dims[ma] != b->dims[mb]) return LCO_ERR_INVALID;
        con_a[ma] = con_b[mb] = 1;
    }
    int free_a[kMaxOrder], free_b[kMaxOrder], nfa = 0, nfb = 0;
    for (int t = 0; t < a->order; ++t) if (!con_a[t]) free_a[nfa++] = t;
    for (int t = 0; t < b->order; ++t) if (!con_b[t]) free_b[nfb++] = t;
    if (nfa + nfb > kMaxOrder) return LCO_ERR_INVALID;
    u128 kc = 1, mA = 1, nB = 1;
    for (int i = 0; i < ncontract; ++i) kc *= (u128)(uint64_t)a->dims[modes_a[i]];
    for (int i = 0; i < nfa; ++i) mA *= (u128)(uint64_t)a->dims[free_a[i]];
    for (int i = 0; i < nfb; ++i) nB *= (u128)(uint64_t)b->dims[free_b[i]];
    const u128 lim = ((u128)1 << 127) - 1;
    if (mA > lim / nB) return LCO_ERR_OVERFLOW;
    // rank-matrix shapes (A' gets up to nnz_A filler rows past its real ones)
    const int64_t na = a->nnz > 0 ? a->nnz : 1, nb = b->nnz > 0 ? b->nnz : 1;
    const int64_t Mp = 2 * na, Kp = nb + 1, Np = nb;
    if (Mp > INT64_MAX / Kp || Mp > INT64_MAX / Np || Kp > INT64_MAX / Np) return LCO_ERR_OVERFLOW;

    lco_wide_plan *p = new (std::nothrow) lco_wide_plan();
    if (!p) return LCO_ERR_OOM;
    std::memset(p, 0, sizeof(*p));
    p->a = *a;
    p->b = *b;
    p->ncontract = ncontract;
    for (int i = 0; i < ncontract; ++i) {
        p->modes_a[i] = modes_a[i];
        p->modes_b[i] = modes_b[i];
    }
    // matrix orders, most significant first, turned into sig (least significant first)
    {
        int32_t msf[kMaxOrder];
        int q = 0;
        for (int i = 0; i < nfa; ++i) msf[q++] = free_a[i];
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_a[i];
        for (int i = 0; i < q; ++i) p->sig_am[i] = msf[q - 1 - i];
        q = 0;
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_b[i];
        for (int i = 0; i < nfb; ++i) msf[q++] = free_b[i];
        for (int i = 0; i < q; ++i) p->sig_bm[i] = msf[q - 1 - i];
    }
    p->perm_a = !same_order(a->order, a->sig, p->sig_am);
    p->perm_b = !same_order(b->order, b->sig, p->sig_bm);
    p->kc = kc;
    p->mA = mA;
    p->nB = nB;
    p->col_bits = bits128(nB);
    if (p->col_bits < 1) p->col_bits = 1;
    p->Mp = Mp;
    p->Kp = Kp;
    p->Np = Np;
    {
        size_t wa = 0, wb = 0;
        if (p->perm_a && (rc = lco_radix_permute_wide_workspace(a, p->sig_am, &wa)) != LCO_OK) { delete p; return rc; }
        if (p->perm_b && (rc = lco_radix_permute_wide_workspace(b, p->sig_bm, &wb)) != LCO_OK) { delete p; return rc; }
        p->perm_ws = wa > wb ? wa : wb;
    }
    // the column-key sort: radix state for the largest chunk plan
    {
        size_t rb = 0;
        for (int c0 = 0; c0 < p->col_bits; c0 += kChunkBits) {
            const int cb = p->col_bits - c0 < kChunkBits ? p->col_bits - c0 : kChunkBits;
            int D, P;
            radix_digits(cb, &D, &P);
            const size_t x = radix_state_bytes(nb, D, P);
            rb = x > rb ? x : rb;
        }
        p->radix_bytes = rb;
    }
    // the 64-bit product of the rank matrices (Table 4 on their shapes)
    lco_shape ap{}, bp{};
    ap.order = 2;
    ap.dims[0] = Mp;
    ap.dims[1] = Kp;
    ap.sig[0] = 1;
    ap.sig[1] = 0;
    ap.nnz = a->nnz;
    bp.order = 2;
    bp.dims[0] = Kp;
    bp.dims[1] = Np;
    bp.sig[0] = 1;
    bp.sig[1] = 0;
    bp.nnz = b->nnz;
    const int32_t ma1 = 1, mb0 = 0;
    if ((rc = lco_contract_plan(&ap, &bp, 1, &ma1, &mb0, LCO_ALG_AUTO, &p->inner)) != LCO_OK) { delete p; return rc; }
    // C: A's free modes, then B's, row-major
    lco_shape &cs = p->c_shape;
    cs.order = nfa + nfb;
    for (int i = 0; i < nfa; ++i) cs.dims[i] = a->dims[free_a[i]];
    for (int i = 0; i < nfb; ++i) cs.dims[nfa + i] = b->dims[free_b[i]];
    if (cs.order == 0) {
        cs.order = 1;
        cs.dims[0] = 1;
    }
    for (int i = 0; i < cs.order; ++i) cs.sig[i] = cs.order - 1 - i;
    cs.nnz = 0;
    *out = p;
    return LCO_OK;
}

int32_t lco_contract_wide_plan_destroy(lco_wide_plan *plan) {
    if (plan) {
        lco_plan_destroy(plan->inner);
        delete plan;
    }
    return LCO_OK;
}

int32_t lco_contract_wide_info(const lco_wide_plan *plan, lco_shape *c_shape, int32_t *inner_alg) {
    if (!plan || !c_shape) return LCO_ERR_INVALID;
    *c_shape = plan->c_shape;
    if (inner_alg) {
        lco_plan_info pi;
        lco_plan_get_info(plan->inner, &pi);
        *inner_alg = pi.alg;
    }
    return LCO_OK;
}

int32_t lco_contract_wide_workspace(const lco_wide_plan *plan, int64_t cap, size_t *ws_bytes) {
    if (!plan || !ws_bytes || cap < 0) return LCO_ERR_INVALID;
    lco_wide_plan tmp = *plan;
    *ws_bytes = wide_layout(&tmp, cap);
    return LCO_OK;
}

int32_t lco_contract_wide_symbolic(const lco_wide_plan *plan, const uint64_t *a_liv, const double *a_val,
                                   const uint64_t *b_liv, const double *b_val, void *ws, size_t ws_bytes,
                                   void *stream) {
    NvtxRange nvtx("lco_contract_wide_symbolic");
    if (!plan || !ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    lco_wide_plan p = *plan;
    const size_t need = wide_layout(&p, 0);
    if (ws_bytes < need) return LCO_ERR_OOM;
    const int64_t na = p.a.nnz, nb = p.b.nnz;
    if ((na > 0 && (!a_liv || !a_val)) || (nb > 0 && (!b_liv || !b_val))) return LCO_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = reinterpret_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(w);
    if (cudaMemsetAsync(w, 0, kWsHeaderBytes, s) != cudaSuccess) return LCO_ERR_CUDA;
    if (cudaMemsetAsync(w + p.o_state, 0, p.state_bytes, s) != cudaSuccess) return LCO_ERR_CUDA;
    char *inner_ws = w + p.o_inner;
    size_t inner_bytes = 0;
    lco_contract_workspace(p.inner, 0, &inner_bytes);
    if (na == 0 || nb == 0) {
        // empty product: the inner plan records it (the rank buffers are
        // valid pointers; nothing is read from an empty operand)
        return lco_contract_symbolic(p.inner, reinterpret_cast<int64_t *>(w + p.o_ap_liv),
                                     reinterpret_cast<double *>(w + p.o_ap_val),
                                     reinterpret_cast<int64_t *>(w + p.o_bp_liv),
                                     reinterpret_cast<double *>(w + p.o_bp_val), inner_ws, inner_bytes, s);
    }
    int32_t rc;
    // 1. matrix orders
    const uint64_t *am_liv = a_liv, *bm_liv = b_liv;
    const double *am_val = a_val, *bm_val = b_val;
    // the wide permutations share one workspace region, whose header must be
    // zero before each of them
    const size_t perm_hdr = p.perm_ws < (size_t)kWsHeaderBytes ? p.perm_ws : (size_t)kWsHeaderBytes;
    if (p.perm_a) {
        if (cudaMemsetAsync(w + p.o_perm, 0, perm_hdr, s) != cudaSuccess) return LCO_ERR_CUDA;
        if ((rc = lco_radix_permute_wide(&p.a, p.sig_am, a_liv, a_val, reinterpret_cast<uint64_t *>(w + p.o_am_liv),
                                         reinterpret_cast<double *>(w + p.o_am_val), w + p.o_perm, p.perm_ws, s)) !=
            LCO_OK)
            return rc;
        am_liv = reinterpret_cast<uint64_t *>(w + p.o_am_liv);
        am_val = reinterpret_cast<double *>(w + p.o_am_val);
    }
    if (p.perm_b) {
        if (cudaMemsetAsync(w + p.o_perm, 0, perm_hdr, s) != cudaSuccess) return LCO_ERR_CUDA;
        if ((rc = lco_radix_permute_wide(&p.b, p.sig_bm, b_liv, b_val, reinterpret_cast<uint64_t *>(w + p.o_bm_liv),
                                         reinterpret_cast<double *>(w + p.o_bm_val), w + p.o_perm, p.perm_ws, s)) !=
            LCO_OK)
            return rc;
        bm_liv = reinterpret_cast<uint64_t *>(w + p.o_bm_liv);
        bm_val = reinterpret_cast<double *>(w + p.o_bm_val);
    }
    uint64_t *a_row = reinterpret_cast<uint64_t *>(w + p.o_a_row);
    uint64_t *a_col = reinterpret_cast<uint64_t *>(w + p.o_a_col);
    uint64_t *b_key = reinterpret_cast<uint64_t *>(w + p.o_b_key);
    uint64_t *b_col = reinterpret_cast<uint64_t *>(w + p.o_b_col);
    int64_t *counts = reinterpret_cast<int64_t *>(w + p.o_counts);   // [0] A rows, [1] B keys, [2] B columns, [3] kept
    uint32_t *tctr = reinterpret_cast<uint32_t *>(w + p.o_state + p.state_bytes - 64);
    // 2. keys: A = (row, contracted), B = (contracted, column)
    LCO_LAUNCH("k_wide_split", s, k_wide_split<<<grid_of(na), kWT, 0, s>>>(na, am_liv, mk128(p.kc), a_row, a_col));
    LCO_LAUNCH("k_wide_split", s, k_wide_split<<<grid_of(nb), kWT, 0, s>>>(nb, bm_liv, mk128(p.nB), b_key, b_col));
    // 3. ranks of A's rows and B's contracted keys (both sequences are sorted)
    RankArgs ra{};
    ra.n = na;
    ra.keys = a_row;
    ra.rank = reinterpret_cast<int64_t *>(w + p.o_a_rrank);
    ra.of_rank = reinterpret_cast<uint64_t *>(w + p.o_row_of);
    ra.count = counts + 0;
    ra.state = scan_region(&p, w, 0);
    ra.tile_ctr = tctr + 0;
    ra.status = &hdr->status;
    LCO_LAUNCH("k_wide_rank", s, k_wide_rank<<<(unsigned)((na + kScanTile - 1) / kScanTile), kWT, 0, s>>>(ra));
    RankArgs rb{};
    rb.n = nb;
    rb.keys = b_key;
    rb.rank = reinterpret_cast<int64_t *>(w + p.o_b_krank);
    rb.of_rank = reinterpret_cast<uint64_t *>(w + p.o_key_of);
    rb.count = counts + 1;
    rb.state = scan_region(&p, w, 1);
    rb.tile_ctr = tctr + 1;
    rb.status = &hdr->status;
    LCO_LAUNCH("k_wide_rank", s, k_wide_rank<<<(unsigned)((nb + kScanTile - 1) / kScanTile), kWT, 0, s>>>(rb));
    // 4. ranks of B's column keys: stable radix sort of (54-bit chunk,
    //    position), least significant chunk first, then ranks in sorted order
    int64_t *chunk_a = reinterpret_cast<int64_t *>(w + p.o_chunk_a);
    double *pos_a = reinterpret_cast<double *>(w + p.o_pos_a);
    int64_t *chunk_b = reinterpret_cast<int64_t *>(w + p.o_chunk_b);
    double *pos_b = reinterpret_cast<double *>(w + p.o_pos_b);
    LCO_LAUNCH("k_wide_key_prep", s, k_wide_key_prep<<<grid_of(nb), kWT, 0, s>>>(nb, b_col, chunk_a, pos_a));
    for (int c0 = 0; c0 < p.col_bits; c0 += kChunkBits) {
        if (c0 > 0)
            LCO_LAUNCH("k_wide_key_chunk", s, k_wide_key_chunk<<<grid_of(nb), kWT, 0, s>>>(nb, b_col, pos_b, c0,
                                                                                             chunk_a, pos_a));
        const int cb = p.col_bits - c0 < kChunkBits ? p.col_bits - c0 : kChunkBits;
        RadixJob j{};
        j.relin.nseg = 1;
        j.relin.identity = 1;
        j.key_div = make_div(1);
        radix_digits(cb, &j.D, &j.P);
        j.n_host = nb;
        j.n_dev = nullptr;
        j.n_cap = nb;
        j.src_liv = chunk_a;
        j.src_val = pos_a;
        j.dst_liv = chunk_b;
        j.dst_val = pos_b;
        j.tmp_liv = reinterpret_cast<int64_t *>(w + p.o_tmp_l);
        j.tmp_val = reinterpret_cast<double *>(w + p.o_tmp_v);
        radix_carve(j, w + p.o_radix);
        j.counters = hdr->counters;
        j.status = &hdr->status;
        if (radix_enqueue(j, s) != cudaSuccess) return LCO_ERR_CUDA;
    }
    RankArgs rc2{};
    rc2.n = nb;
    rc2.keys = b_col;
    rc2.pos = pos_b;
    rc2.rank = reinterpret_cast<int64_t *>(w + p.o_b_crank);
    rc2.of_rank = reinterpret_cast<uint64_t *>(w + p.o_col_of);
    rc2.count = counts + 2;
    rc2.state = scan_region(&p, w, 2);
    rc2.tile_ctr = tctr + 2;
    rc2.status = &hdr->status;
    LCO_LAUNCH("k_wide_rank", s, k_wide_rank<<<(unsigned)((nb + kScanTile - 1) / kScanTile), kWT, 0, s>>>(rc2));
    // 5. the rank matrices
    int64_t *a_krank = reinterpret_cast<int64_t *>(w + p.o_a_krank);
    LCO_LAUNCH("k_wide_a_keep", s, k_wide_a_keep<<<grid_of(na), kWT, 0, s>>>(na, a_col,
                                                   reinterpret_cast<uint64_t *>(w + p.o_key_of), counts + 1, a_krank));
    int64_t *ap_liv = reinterpret_cast<int64_t *>(w + p.o_ap_liv);
    double *ap_val = reinterpret_cast<double *>(w + p.o_ap_val);
    int64_t *bp_liv = reinterpret_cast<int64_t *>(w + p.o_bp_liv);
    double *bp_val = reinterpret_cast<double *>(w + p.o_bp_val);
    BuildA ba{};
    ba.n = na;
    ba.row_rank = reinterpret_cast<int64_t *>(w + p.o_a_rrank);
    ba.krank = a_krank;
    ba.val = am_val;
    ba.Kp = p.Kp;
    ba.Mhalf = p.Mp / 2;
    ba.out_liv = ap_liv;
    ba.out_val = ap_val;
    ba.state = scan_region(&p, w, 3);
    ba.tile_ctr = tctr + 3;
    ba.nkeep = counts + 3;
    ba.status = &hdr->status;
    LCO_LAUNCH("k_wide_a_build", s, k_wide_a_build<<<(unsigned)((na + kScanTile - 1) / kScanTile), kWT, 0, s>>>(ba));
    LCO_LAUNCH("k_wide_a_fill", s, k_wide_a_fill<<<grid_of(na), kWT, 0, s>>>(na, counts + 3, p.Kp, p.Mp / 2,
                                                                              ap_liv, ap_val));
    LCO_LAUNCH("k_wide_b_build", s, k_wide_b_build<<<grid_of(nb), kWT, 0, s>>>(
                                        nb, reinterpret_cast<int64_t *>(w + p.o_b_krank),
                                        reinterpret_cast<int64_t *>(w + p.o_b_crank), bm_val, p.Np, bp_liv, bp_val));
    if (cudaGetLastError() != cudaSuccess) return LCO_ERR_CUDA;
    // 6. phase 1 of the 64-bit product
    return lco_contract_symbolic(p.inner, ap_liv, ap_val, bp_liv, bp_val, inner_ws, inner_bytes, s);
}

int32_t lco_contract_wide_numeric(const lco_wide_plan *plan, uint64_t *c_liv, double *c_val, int64_t cap, void *ws,
                                  size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_contract_wide_numeric");
    if (!plan || !ws || cap < 0 || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    if (cap > 0 && (!c_liv || !c_val)) return LCO_ERR_INVALID;
    lco_wide_plan p = *plan;
    const size_t need = wide_layout(&p, cap);
    if (ws_bytes < need) return LCO_ERR_OOM;
    cudaStream_t s = (cudaStream_t)stream;
    char *w = reinterpret_cast<char *>(ws);
    char *inner_ws = w + p.o_inner;
    size_t inner_bytes = 0;
    lco_contract_workspace(p.inner, cap, &inner_bytes);
    int64_t *cp_liv = reinterpret_cast<int64_t *>(w + p.o_cp_liv);
    double *cp_val = reinterpret_cast<double *>(w + p.o_cp_val);
    const bool empty = p.a.nnz == 0 || p.b.nnz == 0;
    int32_t rc = lco_contract_numeric(p.inner, reinterpret_cast<int64_t *>(w + p.o_ap_liv),
                                      reinterpret_cast<double *>(w + p.o_ap_val),
                                      reinterpret_cast<int64_t *>(w + p.o_bp_liv),
                                      reinterpret_cast<double *>(w + p.o_bp_val), cp_liv, cp_val, cap, inner_ws,
                                      inner_bytes, s);
    if (rc != LCO_OK || empty || cap == 0) return rc;
    LCO_LAUNCH("k_wide_c_map", s, k_wide_c_map<<<grid_of(cap), kWT, 0, s>>>(
                                      reinterpret_cast<const WsHeader *>(inner_ws), make_div((uint64_t)p.Np),
                                      reinterpret_cast<uint64_t *>(w + p.o_row_of),
                                      reinterpret_cast<uint64_t *>(w + p.o_col_of), mk128(p.nB), cp_liv, cp_val, cap,
                                      c_liv, c_val));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

int32_t lco_contract_wide_result_get(const lco_wide_plan *plan, const void *ws, lco_contract_result *out,
                                     void *stream) {
    if (!plan || !ws || !out) return LCO_ERR_INVALID;
    lco_wide_plan p = *plan;
    wide_layout(&p, 0);
    const char *w = reinterpret_cast<const char *>(ws);
    int32_t rc = lco_contract_result_get(w + p.o_inner, out, stream);
    if (rc != LCO_OK) return rc;
    // a device error of the rank stages (a look-back that ran out) comes first
    int32_t st = 0;
    if (cudaMemcpy(&st, w, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return LCO_ERR_CUDA;
    if (st != 0) out->status = st;
    return LCO_OK;
}

}  // extern "C"
