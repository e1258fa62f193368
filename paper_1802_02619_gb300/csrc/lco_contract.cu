// lco_contract.cu -- sparse tensor contraction over LCO (Sec. 5 of the paper).
//
// The product is computed on the matricised operands (Sec. 5.2, "map to a
// matrix, convert to a multiplication datatype and multiply, map back"):
//   L : mL x k, LIV = row * k + c        (the left operand, sorted row-major)
//   R : k x nR, LIV = c * nR + col       (the right operand, sorted row-major)
//   C : mL x nR, LIV = row * nR + col    (sorted, row-major)
// Row variants (CSR, DCSR, CSRNA, SOP) take L = A, R = B.  Column variants
// (CSC, DCSC, CSCNA) run the same row kernels on the transposed product
// C^T = B^T A^T, i.e. L = B, R = A, which yields C in column-major order.
//
// Phase 1 (symbolic): rearrange operands into their matrix orders (radix
// permutation), build R's multiplication datatype -- CSR row pointers
// (Sec. 5.2.2) or DCSR rows with an auxiliary coarse index (Sec. 5.2.3) --
// and scan the work 1 + |R row| of every L entry, which gives f and L's row
// table.
// Phase 2 (numeric): rows whose work exceeds kHeavyWork are multiplied first,
// one CTA per row, by a stable sort of the row's f(i) products by column and
// a sum of each run (the no-accumulator scheme of Sec. 5.2.4; on the GPU it
// also serves the accumulator branches, because an atomic accumulator would
// make the summation order, and so the rounding, vary from run to run).
// Every product is therefore summed in generation order on every path, and
// results are bit-identical across runs.  The remaining (light) rows go one
// lane per row, 32 rows per warp: a lane merges a row's sorted B rows, which
// accumulates and sorts in one go.  Tiles of rows find their place in C by
// decoupled look-back (small L) or write through scratch at their product
// offsets and are then moved into C by k_compact (large L).  SOP (Sec.
// 5.2.5) expands all f products, sorts them by output LIV with the radix
// engine and sums runs.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lco_host.h"

namespace lco {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCT = 256;                    // threads of the chunk / scan kernels
constexpr int kCW = kCT / 32;
constexpr int kEntCap = 2048;               // heavy rows, shared-memory path: L entries
constexpr int kProdCap = 2048;              // heavy rows, shared-memory path: products
constexpr int kSortItems = 8;               // CTA sort: items per thread
constexpr int kSortTile = kCT * kSortItems; // == kProdCap
constexpr int kScanItems = 8;
constexpr int kScanTile = kCT * kScanItems;

// light-row kernel
constexpr int kHeavyWork = 256;             // rows above this work go to the heavy-row kernel
constexpr int kMergeRuns = 8;               // runs a lane merges at once

// header counter slots
constexpr int kCtrDcsr = 10;
constexpr int kCtrScan = 11;

enum Lookup { kLookupCsr = 0, kLookupDcsr = 1 };

struct Mdt {                 // multiplication datatype of R
    int32_t kind;            // Lookup
    int64_t k;
    int64_t nnz;
    const int64_t *row_ptr;  // CSR: [k+1]; DCSR: [nzr+1]
    const int64_t *row_id;   // DCSR: [nzr]
    const int64_t *aux;      // DCSR: [naux+1]
    int32_t aux_shift;
    int64_t naux;
    const uint64_t *ec;      // DCSR, numeric phase: the symbolic phase's lookup of every L entry
};

// Entry cache word: R-row start in the low 40 bits, length above; kEcMiss
// when either does not fit (the consumer then looks the row up itself).
constexpr int kEcB0Bits = 40;
constexpr uint64_t kEcB0Mask = (1ull << kEcB0Bits) - 1;
constexpr uint64_t kEcMiss = ~0ull;

__device__ __forceinline__ uint64_t ec_pack(int64_t b0, int64_t len) {
    if (len == 0) return 0;
    if ((uint64_t)b0 >= kEcB0Mask || (uint64_t)len >= (1ull << (64 - kEcB0Bits)) - 1) return kEcMiss;
    return (uint64_t)b0 | ((uint64_t)len << kEcB0Bits);
}

// (start, length) of R's row c, length 0 when the row is empty.
__device__ __forceinline__ void mdt_lookup(const Mdt &m, int64_t c, int64_t &b0, int64_t &len) {
    if (m.kind == kLookupCsr) {
        b0 = m.row_ptr[c];
        len = m.row_ptr[c + 1] - b0;
        return;
    }
    const int64_t bkt = c >> m.aux_shift;
    int64_t lo = m.aux[bkt], hi = m.aux[bkt + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (m.row_id[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < m.aux[bkt + 1] && m.row_id[lo] == c) {
        b0 = m.row_ptr[lo];
        len = m.row_ptr[lo + 1] - b0;
    } else {
        b0 = 0;
        len = 0;
    }
}

// (start, length) of the R row that L entry e (column c) meets: from the
// entry cache when there is one, else by lookup.
__device__ __forceinline__ void mdt_lookup_entry(const Mdt &m, int64_t e, int64_t c, int64_t &b0, int64_t &len) {
    if (m.ec) {
        const uint64_t x = m.ec[e];
        if (x != kEcMiss) {
            b0 = (int64_t)(x & kEcB0Mask);
            len = (int64_t)(x >> kEcB0Bits);
            return;
        }
    }
    mdt_lookup(m, c, b0, len);
}

// Same, with the column taken from L's LIV only when the cache misses.
__device__ __forceinline__ void mdt_lookup_entry(const Mdt &m, int64_t e, const int64_t *l_liv, int64_t rbase,
                                                 int64_t &b0, int64_t &len) {
    if (m.ec) {
        const uint64_t x = m.ec[e];
        if (x != kEcMiss) {
            b0 = (int64_t)(x & kEcB0Mask);
            len = (int64_t)(x >> kEcB0Bits);
            return;
        }
    }
    mdt_lookup(m, l_liv[e] - rbase, b0, len);
}

// R's row met by an L entry in column c of L's row `row`.  With entrywise
// mode pairs (Sec. 5) L's rows are (h, i) and R's rows (h, k): the entry
// meets R row h * K + c, h = row div I (I = L rows per value of h); without
// them I is all of L's rows and this is c.
__device__ __forceinline__ int64_t r_row(const DivU64 &div_h, int64_t k, uint64_t row, int64_t c) {
    return c + (int64_t)divu(div_h, row) * k;
}

// ------------------------------------------------------------------------
// Block-wide scans (kCT threads)
// ------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread; returns the exclusive prefix and
// the block total in *total.  Uses `s_tmp` (kCW entries).
template <typename T>
__device__ __forceinline__ T block_excl(T v, T *s_tmp, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    __syncthreads();
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kCW ? s_tmp[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < kCW) s_tmp[lane] = wi - w;
        if (lane == kCW - 1) s_tmp[kCW] = wi;
    }
    __syncthreads();
    T r = s_tmp[warp] + incl - v;
    *total = s_tmp[kCW];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------
// CTA-level stable LSD radix sort of (uint64 key, double value) pairs held
// in shared or global memory (generic pointers), 8-bit digits over the low
// `kbits` bits.  Ping-pongs between (k0,v0) and (k1,v1); returns 0 if the
// result ends in (k0,v0), 1 otherwise.  s_whist: kCW*256 u32, s_run: 256 i64.
// ------------------------------------------------------------------------
__device__ int cta_sort(uint64_t *k0, double *v0, uint64_t *k1, double *v1, int64_t n, int kbits,
                        uint32_t *s_whist, int64_t *s_run, int64_t *s_tmp64) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = lanemask_lt();
    int cur = 0;
    for (int shift = 0; shift < kbits; shift += 8) {
        uint64_t *sk = cur ? k1 : k0;
        double *sv = cur ? v1 : v0;
        uint64_t *dk = cur ? k0 : k1;
        double *dv = cur ? v0 : v1;
        // digit histogram over the whole range -> running digit offsets
        for (int d = tid; d < kCW * 256; d += kCT) s_whist[d] = 0;
        __syncthreads();
        for (int64_t i = tid; i < n; i += kCT) atomicAdd(&s_whist[(uint32_t)(sk[i] >> shift) & 255u], 1u);
        __syncthreads();
        {
            int64_t c = s_whist[tid], tot;
            int64_t ex = block_excl<int64_t>(c, s_tmp64, &tot);
            s_run[tid] = ex;
        }
        __syncthreads();
        for (int64_t base = 0; base < n; base += kSortTile) {
            for (int d = tid; d < kCW * 256; d += kCT) s_whist[d] = 0;
            __syncthreads();
            uint32_t pk[kSortItems];
            uint64_t key[kSortItems];
            double val[kSortItems];
            uint32_t *wh = s_whist + warp * 256;
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                const int64_t e = base + warp * (32 * kSortItems) + i * 32 + lane;
                const bool valid = e < n;
                key[i] = valid ? sk[e] : 0;
                val[i] = valid ? sv[e] : 0.0;
                const uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
                unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const unsigned bit = (d >> b) & 1u;
                    const unsigned bal = __ballot_sync(kFull, bit);
                    peers &= bit ? bal : ~bal;
                }
                const int leader = valid ? __ffs(peers) - 1 : lane;
                uint32_t bv = 0;
                if (valid && lane == leader) {
                    bv = wh[d];
                    wh[d] = bv + (uint32_t)__popc(peers);
                }
                bv = __shfl_sync(kFull, bv, leader);
                pk[i] = d | ((bv + (uint32_t)__popc(peers & lt)) << 8);
                __syncwarp();
            }
            __syncthreads();
            // per digit: offsets of each warp, tile total
            {
                const int d = tid;   // kCT == 256 digits
                uint32_t run = 0;
                for (int w = 0; w < kCW; ++w) {
                    uint32_t c = s_whist[w * 256 + d];
                    s_whist[w * 256 + d] = run;
                    run += c;
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < kSortItems; ++i) {
                    const int64_t e = base + warp * (32 * kSortItems) + i * 32 + lane;
                    if (e < n) {
                        const uint32_t dd = pk[i] & 255u;
                        const int64_t pos = s_run[dd] + wh[dd] + (pk[i] >> 8);
                        dk[pos] = key[i];
                        dv[pos] = val[i];
                    }
                }
                __syncthreads();
                s_run[d] += run;
            }
            __syncthreads();
        }
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------------------------
// MDT kernels (Sec. 5.2.2 CSR, Sec. 5.2.3 DCSR)
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_csr_rowptr(const int64_t *liv, int64_t nnz, DivU64 div_n, int64_t k,
                                                    int64_t *row_ptr) {
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // rows are clamped to [0, k - 1] so that LIVs outside the index space
    // can never address past row_ptr
    for (int64_t e = gt; e < nnz; e += gsz) {
        const uint64_t r0 = divu(div_n, (uint64_t)liv[e]);
        const int64_t row = r0 < (uint64_t)k ? (int64_t)r0 : k - 1;
        int64_t prev = -1;
        if (e > 0) {
            const uint64_t p0 = divu(div_n, (uint64_t)liv[e - 1]);
            prev = p0 < (uint64_t)k ? (int64_t)p0 : k - 1;
        }
        for (int64_t r = prev + 1; r <= row; ++r) row_ptr[r] = e;
    }
    int64_t last = -1;
    if (nnz > 0) {
        const uint64_t l0 = divu(div_n, (uint64_t)liv[nnz - 1]);
        last = l0 < (uint64_t)k ? (int64_t)l0 : k - 1;
    }
    for (int64_t r = last + 1 + gt; r <= k; r += gsz) row_ptr[r] = nnz;
}

struct DcsrArgs {
    const int64_t *liv;
    int64_t nnz;
    DivU64 div_n;
    int64_t *row_id;
    int64_t *row_ptr;
    uint64_t *state;
    WsHeader *hdr;
};

// Head flags -> single-pass scan -> compacted (row_id, row_ptr).  Rows are
// computed warp-striped and scanned blocked, through shared memory as in
// the work scan below.
constexpr int kScanPitch = kCT + 4;

__global__ void __launch_bounds__(kCT) k_dcsr_build(const __grid_constant__ DcsrArgs a) {
    __shared__ int64_t s_tmp[kCW + 1];
    __shared__ int64_t s_tile, s_excl;
    __shared__ int64_t s_rows[kScanItems * kScanPitch];
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.hdr->counters[kCtrDcsr], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t tbase = tile * kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t prev0 = -1;
    if (threadIdx.x == 0 && tbase > 0 && tbase - 1 < a.nnz)
        prev0 = (int64_t)divu(a.div_n, (uint64_t)a.liv[tbase - 1]);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int j = warp * (32 * kScanItems) + 32 * i + lane;
        const int64_t e = tbase + j;
        s_rows[(j % kScanItems) * kScanPitch + j / kScanItems] =
            e < a.nnz ? (int64_t)divu(a.div_n, (uint64_t)a.liv[e]) : -2;
    }
    __syncthreads();
    const int64_t base = tbase + (int64_t)threadIdx.x * kScanItems;
    if (threadIdx.x > 0) prev0 = s_rows[(kScanItems - 1) * kScanPitch + threadIdx.x - 1];
    int64_t rows[kScanItems];
    int heads = 0;
    int64_t prev = prev0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        rows[i] = s_rows[i * kScanPitch + threadIdx.x];
        if (base + i < a.nnz) {
            heads += rows[i] != prev;
            prev = rows[i];
        }
    }
    int64_t tot;
    int64_t ex = block_excl<int64_t>((int64_t)heads, s_tmp, &tot);
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
        int64_t e = 0;
        if (tile > 0) e = (int64_t)lookback_warp(a.state, tile, &a.hdr->status);
        if (threadIdx.x == 0) {
            if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(e + tot));
            s_excl = e;
            const int64_t ntiles = (a.nnz + kScanTile - 1) / kScanTile;
            if (tile == ntiles - 1) {
                a.row_ptr[e + tot] = a.nnz;
                a.hdr->nzr_b = e + tot;
            }
        }
    }
    __syncthreads();
    int64_t pos = s_excl + ex;
    prev = prev0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < a.nnz && rows[i] != prev) {
            a.row_id[pos] = rows[i];
            a.row_ptr[pos] = e;
            ++pos;
        }
        if (e < a.nnz) prev = rows[i];
    }
}

// Auxiliary coarse index over the sorted row ids: aux[b] = first i with
// (row_id[i] >> shift) >= b (Buluc & Gilbert's AUX array idea).
__global__ void __launch_bounds__(256) k_dcsr_aux(const int64_t *row_id, const WsHeader *hdr, int32_t shift,
                                                  int64_t naux, int64_t *aux, int64_t cap) {
    const int64_t nzr = hdr->nzr_b;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= nzr && i <= cap; i += gsz) {
        int64_t bi = i < nzr ? (int64_t)((uint64_t)row_id[i] >> shift) : naux;
        int64_t bp = i > 0 ? (int64_t)((uint64_t)row_id[i - 1] >> shift) : -1;
        if (bi > naux) bi = naux;      // row ids outside [0, k) cannot address past aux
        if (bp > naux) bp = naux;
        for (int64_t b = bp + 1; b <= bi; ++b) aux[b] = i;
    }
}

// ------------------------------------------------------------------------
// Phase 1 (DCSR R): every L entry's R row, found by searching R's row ids,
// into the entry cache -- one entry per thread, so that the searches (chains
// of dependent loads) of many entries overlap; the ordered scan below then
// reads the cache.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_entry_lookup(const int64_t *l_liv, int64_t nnz_l, DivU64 div_k, int64_t k,
                                                      DivU64 div_h, const __grid_constant__ Mdt mdt, uint64_t *ec) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < nnz_l; e += (int64_t)gridDim.x * 256) {
        const uint64_t liv = (uint64_t)l_liv[e];
        const uint64_t row = divu(div_k, liv);
        const int64_t c = r_row(div_h, k, row, (int64_t)(liv - row * (uint64_t)k));
        int64_t b0, len;
        mdt_lookup(mdt, c, b0, len);
        ec[e] = ec_pack(b0, len);
    }
}

// ------------------------------------------------------------------------
// Phase 1: work scan over L entries.  An entry costs 1 + |R row of its
// column| work units.  The scan produces the row table of L (first entry,
// row id, work offset of every non-empty row) and, for SOP, the per-entry
// work prefix P.
// ------------------------------------------------------------------------
struct ScanArgs {
    int32_t alg;
    const int64_t *l_liv;
    int64_t nnz_l;
    DivU64 div_k;
    int64_t k;
    DivU64 div_h;          // L rows per value of the entrywise indices
    Mdt mdt;               // with the entry cache (DCSR) already filled
    int64_t *P;            // [nnz_l + 1] or null
    int64_t *row_start;    // [nrows + 1]
    int64_t *row_id;       // [nrows]
    int64_t *row_work;     // [nrows + 1]
    uint64_t *state_w;     // look-back words (work)
    uint64_t *state_h;     // look-back words (row heads)
    WsHeader *hdr;
};

// The entries are loaded and looked up warp-striped (entry w * 256 + 32 i +
// lane in item i of warp w: every load instruction reads consecutive
// entries, and consecutive entries of a row meet nearby R rows), then
// scanned blocked (thread t owns the tile's entries 8 t .. 8 t + 7).  Entry
// j's work and row id pass between the two through shared memory at
// (j mod 8) * kScanPitch + j / 8: the warp-striped stores hit every bank
// pair twice and the blocked loads are conflict-free.  Six CTAs fit on an
// SM, so that more tiles are in flight at once and fewer wait on their
// look-backs.  The lookups are two loads (CSR R) or read from the entry
// cache (DCSR R).
__global__ void __launch_bounds__(kCT, 6) k_work_scan(const __grid_constant__ ScanArgs a) {
    __shared__ int64_t s_tmp[kCW + 1];
    __shared__ int64_t s_tile, s_ew, s_eh;
    __shared__ int64_t s_w[kScanItems * kScanPitch], s_rows[kScanItems * kScanPitch];
    grid_dep_wait();
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.hdr->counters[kCtrScan], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t tbase = tile * kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // row of the entry before the tile (thread 0 only)
    int64_t prev = -1;
    if (threadIdx.x == 0 && tbase > 0 && tbase - 1 < a.nnz_l)
        prev = (int64_t)divu(a.div_k, (uint64_t)a.l_liv[tbase - 1]);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int j = warp * (32 * kScanItems) + 32 * i + lane;
        const int64_t e = tbase + j;
        int64_t wi = 0, ri = -1;
        if (e < a.nnz_l) {
            const uint64_t liv = (uint64_t)a.l_liv[e];
            const uint64_t row = divu(a.div_k, liv);
            const int64_t c = r_row(a.div_h, a.k, row, (int64_t)(liv - row * (uint64_t)a.k));
            int64_t b0, len;
            mdt_lookup_entry(a.mdt, e, c, b0, len);
            wi = 1 + len;
            ri = (int64_t)row;
        }
        const int slot = (j % kScanItems) * kScanPitch + j / kScanItems;
        s_w[slot] = wi;
        s_rows[slot] = ri;
    }
    __syncthreads();
    const int64_t base = tbase + (int64_t)threadIdx.x * kScanItems;
    if (threadIdx.x > 0) prev = s_rows[(kScanItems - 1) * kScanPitch + threadIdx.x - 1];
    int64_t wsum = 0, hsum = 0;
    uint32_t heads = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t ri = s_rows[i * kScanPitch + threadIdx.x];
        if (base + i < a.nnz_l) {
            if (ri != prev) heads |= 1u << i;
            prev = ri;
        }
        wsum += s_w[i * kScanPitch + threadIdx.x];
    }
    hsum = __popc(heads);
    int64_t wtot, htot;
    const int64_t wex = block_excl<int64_t>(wsum, s_tmp, &wtot);
    const int64_t hex = block_excl<int64_t>(hsum, s_tmp, &htot);
    // the two look-backs (work, row heads) run in warps 0 and 1
    if (threadIdx.x < 64) {
        const bool hw = threadIdx.x >= 32;
        uint64_t *st = hw ? a.state_h : a.state_w;
        const int64_t tv = hw ? htot : wtot;
        if ((threadIdx.x & 31) == 0) lb_store(st + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tv);
        int64_t ex = 0;
        if (tile > 0) ex = (int64_t)lookback_warp(st, tile, &a.hdr->status);
        if ((threadIdx.x & 31) == 0) {
            if (tile > 0) lb_store(st + tile, kFlagIncl | (uint64_t)(ex + tv));
            if (hw) s_eh = ex; else s_ew = ex;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t ew = s_ew, eh = s_eh;
        const int64_t ntiles = (a.nnz_l + kScanTile - 1) / kScanTile;
        if (tile == ntiles - 1) {
            const int64_t W = ew + wtot, R = eh + htot;
            if (a.P) a.P[a.nnz_l] = W;
            a.row_start[R] = a.nnz_l;
            a.row_work[R] = W;
            a.hdr->work_total = W;
            a.hdr->f = W - a.nnz_l;
            a.hdr->nrows_l = R;
            a.hdr->nchunks = 0;
            a.hdr->alg = a.alg;
        }
    }
    __syncthreads();
    int64_t run = s_ew + wex;
    int64_t h = s_eh + hex;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < a.nnz_l) {
            if (a.P) a.P[e] = run;
            if (heads & (1u << i)) {
                a.row_start[h] = e;
                a.row_id[h] = s_rows[i * kScanPitch + threadIdx.x];
                a.row_work[h] = run;
                ++h;
            }
        }
        run += s_w[i * kScanPitch + threadIdx.x];
    }
}

// Heavy rows: rows whose work exceeds kHeavyWork are listed for the
// CTA-level heavy-row kernel.
struct TableArgs {
    const int64_t *row_start;
    const int64_t *row_work;
    int64_t *heavy_list;   // [nrows]
    unsigned long long *nheavy;
    int64_t *act_rows;     // [nrows] rows with at least one product, in order
    unsigned long long *nact;
    uint64_t *state;       // look-back words, one per tile of rows
    uint32_t *tile_ctr;
    int64_t cap;           // output capacity (f must not exceed it)
    WsHeader *hdr;
};

constexpr int kTabItems = 8;
constexpr int kTabTile = kCT * kTabItems;

// Row classification: the ordered list of rows with at least one product
// (rows whose entries all miss R produce nothing and are dropped), and the
// heavy rows.  A heavy row with one entry is a scaled copy of one R row and
// stays with the light-row kernel, which copies it without sorting.
// Without compaction (every row kept, as when R is not row-sparse and
// nearly every entry meets an R row): only the heavy-row list is built, so
// that k_heavy spreads the heavy rows over all its CTAs.
__global__ void __launch_bounds__(256) k_row_heavy(const __grid_constant__ TableArgs a) {
    if (a.hdr->f > a.cap) return;
    const int64_t nrows = a.hdr->nrows_l;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gsz) {
        const int64_t work = a.row_work[r + 1] - a.row_work[r];
        if (work > kHeavyWork) {
            const int64_t nent = a.row_start[r + 1] - a.row_start[r];
            if (work > nent && nent > 1) {
                const unsigned long long h = atomicAdd(a.nheavy, 1ull);
                a.heavy_list[h] = r;
            }
        }
    }
}

__global__ void __launch_bounds__(kCT) k_row_table(const __grid_constant__ TableArgs a) {
    __shared__ int64_t s_tmp[kCW + 1];
    __shared__ int64_t s_tile, s_ex;
    __shared__ int64_t s_work[kTabTile + 1], s_start[kTabTile + 1];
    if (a.hdr->f > a.cap) return;
    const int64_t nrows = a.hdr->nrows_l;
    const int64_t ntiles = (nrows + kTabTile - 1) / kTabTile;
    if (ntiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {   // no rows at all
            *a.nact = 0;
            a.hdr->nnz_c = 0;
        }
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t t0 = tile * kTabTile;
        const int64_t nt = (nrows - t0 < kTabTile ? nrows - t0 : kTabTile) + 1;   // row boundaries
        {
            // coalesced staging, every load in flight before the first store
            constexpr int kStg = (kTabTile + 1 + kCT - 1) / kCT;
            int64_t wv[kStg], sv[kStg];
#pragma unroll
            for (int q = 0; q < kStg; ++q) {
                const int i = q * kCT + threadIdx.x;
                if (i < nt) {
                    wv[q] = a.row_work[t0 + i];
                    sv[q] = a.row_start[t0 + i];
                }
            }
#pragma unroll
            for (int q = 0; q < kStg; ++q) {
                const int i = q * kCT + threadIdx.x;
                if (i < nt) {
                    s_work[i] = wv[q];
                    s_start[i] = sv[q];
                }
            }
        }
        __syncthreads();
        const int lb = threadIdx.x * kTabItems;
        uint32_t act = 0;
#pragma unroll
        for (int i = 0; i < kTabItems; ++i) {
            const int j = lb + i;
            if (j + 1 < nt) {
                const int64_t work = s_work[j + 1] - s_work[j];
                const int64_t nent = s_start[j + 1] - s_start[j];
                if (work > nent) {
                    act |= 1u << i;
                    if (work > kHeavyWork && nent > 1) {
                        const unsigned long long h = atomicAdd(a.nheavy, 1ull);
                        a.heavy_list[h] = t0 + j;
                    }
                }
            }
        }
        int64_t tot;
        const int64_t ex = block_excl<int64_t>((int64_t)__popc(act), s_tmp, &tot);
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
            int64_t pre = 0;
            if (tile > 0) pre = (int64_t)lookback_warp(a.state, tile, &a.hdr->status);
            if (threadIdx.x == 0) {
                if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(pre + tot));
                s_ex = pre;
                if (tile == ntiles - 1) {
                    *a.nact = (unsigned long long)(pre + tot);
                    if (pre + tot == 0) a.hdr->nnz_c = 0;
                }
            }
        }
        __syncthreads();
        int64_t o = s_ex + ex;
#pragma unroll
        for (int i = 0; i < kTabItems; ++i)
            if (act & (1u << i)) a.act_rows[o++] = t0 + lb + i;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// Heavy rows (work > kHeavyWork): one CTA per row.  The row's products are
// sorted stably by column and each run summed in generation order, in shared
// memory when they fit, else in global scratch.  The reduced row is left at the row's product offset in scratch
// and its length in row_hout[r] (bit 62 set when it lies in the second
// scratch buffer).
// ------------------------------------------------------------------------
struct HeavyArgs {
    const int64_t *l_liv;
    const double *l_val;
    const int64_t *r_liv;
    const double *r_val;
    DivU64 div_k;
    int64_t k;
    DivU64 div_h;
    DivU64 div_n;
    int64_t nR;
    int32_t colbits;
    Mdt mdt;
    const int64_t *row_start;
    const int64_t *row_work;
    const int64_t *heavy_list;
    const unsigned long long *nheavy;
    int64_t *row_hout;
    int64_t cap;
    uint64_t *sk0;
    double *sv0;
    uint64_t *sk1;
    double *sv1;
    uint32_t *ctr;
    WsHeader *hdr;
    int32_t acc;          // 1: accumulator plans (window or hash), 0: no accumulator (sort)
};

struct HeavySmem {
    int32_t poff[kEntCap + 1];
    int64_t b0[kEntCap];
    double aval[kEntCap];
    uint64_t pk0[kProdCap];
    uint64_t pk1[kProdCap];
    double pv0[kProdCap];
    double pv1[kProdCap];
    uint64_t ok[kProdCap];
    double ov[kProdCap];
    uint32_t whist[kCW * 256];
    int64_t run[256];
    int64_t tmp64[kCW + 2];
    int32_t tmp32[kCW + 2];
};

// One heavy row r, by the whole CTA.
__device__ __forceinline__ void heavy_row(const HeavyArgs &a, HeavySmem &S, int64_t r) {
    const int tid = threadIdx.x;
    const int64_t h0 = a.row_start[r], eend = a.row_start[r + 1];
    const int64_t pbase = a.row_work[r] - h0;
    const int64_t nprod = (a.row_work[r + 1] - eend) - pbase;
    const int64_t nent = eend - h0;
    if (nent <= kEntCap && nprod <= kProdCap) {
        // ---- shared-memory path ----
        int64_t len_i[kEntCap / kCT];
        int64_t lsum = 0;
#pragma unroll
        for (int q = 0; q < kEntCap / kCT; ++q) {
            const int j = tid * (kEntCap / kCT) + q;
            len_i[q] = 0;
            if (j < nent) {
                const int64_t e = h0 + j;
                const uint64_t liv = (uint64_t)a.l_liv[e];
                const uint64_t row = divu(a.div_k, liv);
                const int64_t c = r_row(a.div_h, a.k, row, (int64_t)(liv - row * (uint64_t)a.k));
                int64_t b0, len;
                mdt_lookup_entry(a.mdt, e, c, b0, len);
                S.b0[j] = b0;
                S.aval[j] = a.l_val[e];
                len_i[q] = len;
            }
            lsum += len_i[q];
        }
        int32_t ltot;
        int32_t lex = block_excl<int32_t>((int32_t)lsum, S.tmp32, &ltot);
#pragma unroll
        for (int q = 0; q < kEntCap / kCT; ++q) {
            const int j = tid * (kEntCap / kCT) + q;
            if (j < nent) S.poff[j] = lex;
            lex += (int32_t)len_i[q];
        }
        if (tid == 0) S.poff[nent] = ltot;
        __syncthreads();
        const int np = ltot;
        for (int p = tid; p < np; p += kCT) {
            int lo = 0, hi = (int)nent;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (S.poff[mid] <= p) lo = mid; else hi = mid;
            }
            const int64_t b = S.b0[lo] + (p - S.poff[lo]);
            const uint64_t rl = (uint64_t)a.r_liv[b];
            const uint64_t col = rl - divu(a.div_n, rl) * (uint64_t)a.nR;
            const double v = S.aval[lo] * a.r_val[b];
            S.pk0[p] = col;
            S.pv0[p] = v;
        }
        __syncthreads();
        // stable sort by column, then sum each run in generation order
        const int rs = cta_sort(S.pk0, S.pv0, S.pk1, S.pv1, np, a.colbits, S.whist, S.run, S.tmp64);
        const uint64_t *k = rs ? S.pk1 : S.pk0;
        const double *v = rs ? S.pv1 : S.pv0;
        int32_t hc = 0;
        for (int q = 0; q < kProdCap / kCT; ++q) {
            const int i = tid * (kProdCap / kCT) + q;
            if (i < np && (i == 0 || k[i] != k[i - 1])) ++hc;
        }
        int32_t htot;
        int32_t o = block_excl<int32_t>(hc, S.tmp32, &htot);
        for (int q = 0; q < kProdCap / kCT; ++q) {
            const int i = tid * (kProdCap / kCT) + q;
            if (i < np && (i == 0 || k[i] != k[i - 1])) {
                double s = v[i];
                for (int t = i + 1; t < np && k[t] == k[i]; ++t) s += v[t];
                S.ok[o] = k[i];
                S.ov[o] = s;
                ++o;
            }
        }
        const int64_t nout = htot;
        __syncthreads();
        for (int64_t i = tid; i < nout; i += kCT) {
            a.sk0[pbase + i] = S.ok[i];
            a.sv0[pbase + i] = S.ov[i];
        }
        if (tid == 0) a.row_hout[r] = nout;
        __syncthreads();
    } else {
        // ---- global path: expand, sort and reduce in scratch ----
        uint64_t *gk0 = a.sk0 + pbase;
        double *gv0 = a.sv0 + pbase;
        uint64_t *gk1 = a.sk1 + pbase;
        double *gv1 = a.sv1 + pbase;
        int64_t prod_before = 0;
        for (int64_t t0 = h0; t0 < eend; t0 += kCT) {
            const int64_t e = t0 + tid;
            int64_t b0 = 0, len = 0;
            double av = 0.0;
            int64_t c = 0;
            if (e < eend) {
                const uint64_t liv = (uint64_t)a.l_liv[e];
                const uint64_t row = divu(a.div_k, liv);
                c = r_row(a.div_h, a.k, row, (int64_t)(liv - row * (uint64_t)a.k));
                mdt_lookup_entry(a.mdt, e, c, b0, len);
                av = a.l_val[e];
            }
            int64_t ltot;
            const int64_t lex = block_excl<int64_t>(len, S.tmp64, &ltot);
            for (int64_t t = 0; t < len; ++t) {
                const int64_t rl = a.r_liv[b0 + t];
                gk0[prod_before + lex + t] = (uint64_t)(rl - c * a.nR);
                gv0[prod_before + lex + t] = av * a.r_val[b0 + t];
            }
            prod_before += ltot;
        }
        __syncthreads();
        const int rs = cta_sort(gk0, gv0, gk1, gv1, nprod, a.colbits, S.whist, S.run, S.tmp64);
        const uint64_t *k = rs ? gk1 : gk0;
        const double *v = rs ? gv1 : gv0;
        uint64_t *ok = rs ? gk0 : gk1;
        double *ov = rs ? gv0 : gv1;
        int64_t outc = 0;
        for (int64_t t0 = 0; t0 < nprod; t0 += kCT) {
            const int64_t i = t0 + tid;
            const int hd = (i < nprod) && (i == 0 || k[i] != k[i - 1]);
            int32_t tot;
            const int32_t o = block_excl<int32_t>(hd, S.tmp32, &tot);
            if (hd) {
                double s = v[i];
                for (int64_t t = i + 1; t < nprod && k[t] == k[i]; ++t) s += v[t];
                ok[outc + o] = k[i];
                ov[outc + o] = s;
            }
            outc += tot;
        }
        __syncthreads();
        if (tid == 0) a.row_hout[r] = outc | (rs ? 0ll : (1ll << 62));
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// Heavy rows with an accumulator (Sec. 5.2.2: the row-by-row product keeps
// an accumulator over the columns of C; Sec. 5.2.3's doubly compressed
// variant keeps it).  On the GPU the accumulator is a per-row structure in
// shared memory that maps each product's column to the index of its output
// entry:
//   - a dense bitmap over the row's column window [min, max] of the R rows
//     it meets, when the window has at most kAccWin columns -- the prefix
//     count of the set bits is the output index, already in column order;
//   - otherwise an open-addressing hash of the row's distinct columns,
//     whose distinct columns are then sorted so that each slot takes its
//     rank.
// The products are then bucketed by output index, each bucket is put in
// generation order (L entry order; an entry contributes at most one product
// per column) and summed from its first product: the same rounding as every
// other path.  The no-accumulator plans (Sec. 5.2.4: CSRNA, CSCNA) expand,
// sort and sum instead (heavy_row), as do rows whose entry or product count
// exceeds the shared-memory capacities.
// ------------------------------------------------------------------------
constexpr int kAccEnt = 1024;          // L entries of a row
constexpr int kAccProd = 2048;         // products of a row
constexpr int kAccWin = 16384;         // columns of the dense window
constexpr int kAccHash = 2 * kAccProd; // hash slots (load at most 1/2)
constexpr uint64_t kHashEmpty = ~0ull;

struct AccSmem {
    int32_t poff[kAccEnt + 1];
    int64_t b0[kAccEnt];
    double aval[kAccEnt];
    uint64_t pcol[kAccProd];           // product columns; hash plans: the sorted distinct columns later
    double pv[kAccProd];               // product values (rounded products)
    uint32_t pidx[kAccProd];           // hash slot, then output index of each product
    uint16_t pe[kAccProd];             // L entry (row-local) of each product
    union {
        struct {
            uint32_t bits[kAccWin / 32];
            uint32_t wpre[kAccWin / 32 + 1];
            uint64_t outcol[kAccProd];
        } win;
        struct {
            uint64_t key[kAccHash];
            uint32_t idx[kAccHash];
            uint32_t dslot[kAccProd];
        } hash;
    };
    union {
        struct {                       // sort of the distinct columns (hash plans)
            uint64_t k0[kAccProd], k1[kAccProd];
            double v0[kAccProd], v1[kAccProd];
        } sort;
        struct {                       // buckets by output index
            uint32_t start[kAccProd + 1];
            uint32_t cur[kAccProd];
            uint16_t be[kAccProd];
            double bv[kAccProd];
        } bkt;
    };
    uint32_t whist[kCW * 256];
    int64_t run[256];
    int64_t tmp64[kCW + 2];
    int32_t tmp32[kCW + 2];
    uint32_t ndist;
    int32_t fits;
    uint64_t cmin, cmax;
};

// One heavy row r through the accumulator; false (nothing written) when
// the row does not fit the shared-memory structures.
__device__ __noinline__ bool accumulate_row(const HeavyArgs &a, AccSmem &S, int64_t r) {
    const int tid = threadIdx.x;
    const int64_t h0 = a.row_start[r], eend = a.row_start[r + 1];
    const int64_t pbase = a.row_work[r] - h0;
    const int64_t nprod = (a.row_work[r + 1] - eend) - pbase;
    const int64_t nent = eend - h0;
    if (a.acc != 1 || nent > kAccEnt || nprod > kAccProd) return false;
    // ---- entries: R row of each, products offsets, column range ----
    if (tid == 0) {
        S.cmin = ~0ull;
        S.cmax = 0;
        S.ndist = 0;
        S.fits = 1;
    }
    int64_t len_i[kAccEnt / kCT];
    int64_t lsum = 0;
    uint64_t cmin = ~0ull, cmax = 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kAccEnt / kCT; ++q) {
        const int j = tid * (kAccEnt / kCT) + q;
        len_i[q] = 0;
        if (j < nent) {
            const int64_t e = h0 + j;
            const uint64_t liv = (uint64_t)a.l_liv[e];
            const uint64_t row = divu(a.div_k, liv);
            const int64_t c = r_row(a.div_h, a.k, row, (int64_t)(liv - row * (uint64_t)a.k));
            int64_t b0, len;
            mdt_lookup_entry(a.mdt, e, c, b0, len);
            S.b0[j] = b0;
            S.aval[j] = a.l_val[e];
            len_i[q] = len;
            if (len > 0) {
                const uint64_t f0 = (uint64_t)a.r_liv[b0], f1 = (uint64_t)a.r_liv[b0 + len - 1];
                const uint64_t c0 = f0 - divu(a.div_n, f0) * (uint64_t)a.nR;
                const uint64_t c1 = f1 - divu(a.div_n, f1) * (uint64_t)a.nR;
                cmin = c0 < cmin ? c0 : cmin;
                cmax = c1 > cmax ? c1 : cmax;
            }
        }
        lsum += len_i[q];
    }
    if (cmax >= cmin) {
        atomicMin(reinterpret_cast<unsigned long long *>(&S.cmin), (unsigned long long)cmin);
        atomicMax(reinterpret_cast<unsigned long long *>(&S.cmax), (unsigned long long)cmax);
    }
    int32_t ltot;
    int32_t lex = block_excl<int32_t>((int32_t)lsum, S.tmp32, &ltot);
#pragma unroll
    for (int q = 0; q < kAccEnt / kCT; ++q) {
        const int j = tid * (kAccEnt / kCT) + q;
        if (j < nent) S.poff[j] = lex;
        lex += (int32_t)len_i[q];
    }
    if (tid == 0) S.poff[nent] = ltot;
    __syncthreads();
    const int np = ltot;
    const uint64_t wmin = S.cmin;
    // dense window when the columns span at most kAccWin (uniform over the CTA)
    const bool window = S.cmax >= wmin && S.cmax - wmin < (uint64_t)kAccWin;
    const int nwin = window ? (int)((S.cmax - wmin) / 32 + 1) : 0;
    if (window) {
        for (int w = tid; w < nwin; w += kCT) S.win.bits[w] = 0;
    } else {
        for (int i = tid; i < kAccHash; i += kCT) S.hash.key[i] = kHashEmpty;
    }
    __syncthreads();
    // ---- products (rounded, in generation order), columns into the map ----
    for (int p = tid; p < np; p += kCT) {
        int lo = 0, hi = (int)nent;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S.poff[mid] <= p) lo = mid; else hi = mid;
        }
        const int64_t b = S.b0[lo] + (p - S.poff[lo]);
        const uint64_t rl = (uint64_t)a.r_liv[b];
        const uint64_t col = rl - divu(a.div_n, rl) * (uint64_t)a.nR;
        S.pcol[p] = col;
        S.pv[p] = __dmul_rn(S.aval[lo], a.r_val[b]);
        S.pe[p] = (uint16_t)lo;
        if (window) {
            const uint32_t x = (uint32_t)(col - wmin);
            atomicOr(&S.win.bits[x >> 5], 1u << (x & 31));
        } else {
            // linear probing from a multiplicative hash; at most half full
            uint32_t slot = (uint32_t)((col * 0x9E3779B97F4A7C15ull) >> 40) & (kAccHash - 1);
            for (int t = 0; t < kAccHash; ++t) {
                const unsigned long long old = atomicCAS(
                    reinterpret_cast<unsigned long long *>(&S.hash.key[slot]), (unsigned long long)kHashEmpty,
                    (unsigned long long)col);
                if (old == kHashEmpty) {
                    S.hash.dslot[atomicAdd(&S.ndist, 1u)] = slot;
                    break;
                }
                if (old == col) break;
                slot = (slot + 1) & (kAccHash - 1);
            }
            S.pidx[p] = slot;
        }
    }
    __syncthreads();
    // ---- output index of every distinct column, in column order ----
    int nd;
    if (window) {
        // exclusive prefix of the set bits per window word
        constexpr int kPer = kAccWin / 32 / kCT;
        int c[kPer];
        int csum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int w = tid * kPer + q;
            c[q] = w < nwin ? __popc(S.win.bits[w]) : 0;
            csum += c[q];
        }
        int32_t tot;
        int32_t ex = block_excl<int32_t>(csum, S.tmp32, &tot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int w = tid * kPer + q;
            if (w < nwin) S.win.wpre[w] = (uint32_t)ex;
            ex += c[q];
        }
        nd = tot;
        __syncthreads();
        for (int p = tid; p < np; p += kCT) {
            const uint32_t x = (uint32_t)(S.pcol[p] - wmin);
            const uint32_t o = S.win.wpre[x >> 5] + (uint32_t)__popc(S.win.bits[x >> 5] & ((1u << (x & 31)) - 1u));
            S.pidx[p] = o;
            S.win.outcol[o] = S.pcol[p];   // every product of the column writes the same value
        }
    } else {
        nd = (int)S.ndist;
        for (int i = tid; i < nd; i += kCT) {
            const uint32_t sl = S.hash.dslot[i];
            S.sort.k0[i] = S.hash.key[sl];
            S.sort.v0[i] = __longlong_as_double((long long)sl);
        }
        __syncthreads();
        const int rs = cta_sort(S.sort.k0, S.sort.v0, S.sort.k1, S.sort.v1, nd, a.colbits, S.whist, S.run, S.tmp64);
        const uint64_t *sk = rs ? S.sort.k1 : S.sort.k0;
        const double *sv = rs ? S.sort.v1 : S.sort.v0;
        for (int i = tid; i < nd; i += kCT) {
            S.hash.idx[(uint32_t)__double_as_longlong(sv[i])] = (uint32_t)i;
            S.pcol[i] = sk[i];            // the product columns are no longer needed
        }
        __syncthreads();
        for (int p = tid; p < np; p += kCT) S.pidx[p] = S.hash.idx[S.pidx[p]];
    }
    __syncthreads();
    const uint64_t *outcol = window ? S.win.outcol : S.pcol;
    // ---- buckets by output index ----
    for (int o = tid; o <= nd; o += kCT) S.bkt.start[o] = 0;
    __syncthreads();
    for (int p = tid; p < np; p += kCT) atomicAdd(&S.bkt.start[S.pidx[p]], 1u);
    __syncthreads();
    {
        constexpr int kPer = kAccProd / kCT;
        uint32_t c[kPer];
        uint32_t csum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int o = tid * kPer + q;
            c[q] = o < nd ? S.bkt.start[o] : 0u;
            csum += c[q];
        }
        int32_t tot;
        int32_t ex = block_excl<int32_t>((int32_t)csum, S.tmp32, &tot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int o = tid * kPer + q;
            if (o < nd) {
                S.bkt.start[o] = (uint32_t)ex;
                S.bkt.cur[o] = 0;
            }
            ex += (int32_t)c[q];
        }
        if (tid == 0) S.bkt.start[nd] = (uint32_t)tot;
    }
    __syncthreads();
    for (int p = tid; p < np; p += kCT) {
        const uint32_t o = S.pidx[p];
        const uint32_t pos = S.bkt.start[o] + atomicAdd(&S.bkt.cur[o], 1u);
        S.bkt.be[pos] = S.pe[p];
        S.bkt.bv[pos] = S.pv[p];
    }
    __syncthreads();
    // ---- each output: its products in entry order, summed from the first ----
    for (int o = tid; o < nd; o += kCT) {
        const int s0 = (int)S.bkt.start[o], s1 = (int)S.bkt.start[o + 1];
        for (int i = s0 + 1; i < s1; ++i) {      // insertion sort by entry (buckets are short)
            const uint16_t e = S.bkt.be[i];
            const double v = S.bkt.bv[i];
            int t = i - 1;
            while (t >= s0 && S.bkt.be[t] > e) {
                S.bkt.be[t + 1] = S.bkt.be[t];
                S.bkt.bv[t + 1] = S.bkt.bv[t];
                --t;
            }
            S.bkt.be[t + 1] = e;
            S.bkt.bv[t + 1] = v;
        }
        double sum = S.bkt.bv[s0];
        for (int i = s0 + 1; i < s1; ++i) sum = __dadd_rn(sum, S.bkt.bv[i]);
        a.sk0[pbase + o] = outcol[o];
        a.sv0[pbase + o] = sum;
    }
    if (tid == 0) a.row_hout[r] = nd;
    __syncthreads();
    return true;
}

// Heavy-row kernel: persistent CTAs over the heavy-row list; rows of
// accumulator plans go through the accumulator when they fit, every other
// row through the sort-based path.
__global__ void __launch_bounds__(kCT, 1) k_heavy(const __grid_constant__ HeavyArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HeavySmem &S = *reinterpret_cast<HeavySmem *>(smem_raw);
    AccSmem &SA = *reinterpret_cast<AccSmem *>(smem_raw);
    __shared__ int64_t s_h;
    grid_dep_wait();
    const int tid = threadIdx.x;
    if (a.hdr->f > a.cap) return;
    const int64_t nheavy = (int64_t)*a.nheavy;
    for (;;) {
        if (tid == 0) s_h = atomicAdd(a.ctr, 1u);
        __syncthreads();
        const int64_t h = s_h;
        if (h >= nheavy) break;
        const int64_t r = a.heavy_list[h];
        if (!accumulate_row(a, SA, r)) heavy_row(a, S, r);
    }
}

constexpr size_t kHeavySmemBytes = sizeof(HeavySmem) > sizeof(AccSmem) ? sizeof(HeavySmem) : sizeof(AccSmem);
static_assert(kHeavySmemBytes <= 227 * 1024, "heavy-row shared memory exceeds a CTA's limit");

// ------------------------------------------------------------------------
// Light rows (work <= kHeavyWork): one warp per tile of 32 consecutive rows
// of L, one lane per row, no block barriers.  A lane collects its row's
// non-empty runs -- the B rows selected by the row's L entries, each sorted
// by column -- and merges them (k-way, up to kMergeRuns at once), summing
// equal columns in run order: the merge is at the same time the
// accumulation and the per-row sort of Table 6.  The B rows are read from
// L1/L2 directly.  Rows a lane does not merge are taken by the whole warp:
// a row with a single run is copied (coalesced, scaled) and a row with more
// runs or more products is gathered into shared memory, sorted (bitonic) and
// reduced into scratch.  Heavy rows were reduced by k_heavy.  Network rows
// are sorted in registers and staged in shared memory; a tile's outputs are
// placed once its offset is known (see k_rows for the two placements).
// ------------------------------------------------------------------------
constexpr int kLaneProd = 64;          // products a lane merges by itself
constexpr int kRowsThreads = 128;      // 4 warps per CTA
constexpr int kRowsCtas = 4;           // resident CTAs per SM (registers and shared memory)
constexpr int kWarpSortCap = kHeavyWork;   // products of a warp-sorted row

struct RowsArgs {
    const int64_t *l_liv;
    const double *l_val;
    const int64_t *r_liv;
    const double *r_val;
    int64_t k;
    DivU64 div_h;
    DivU64 div_n;
    int64_t nR;
    Mdt mdt;
    const int64_t *row_start;
    const int64_t *row_id;
    const int64_t *row_work;
    int64_t *row_hout;            // heavy rows: reduced length in; long copies: output offset out
    const int64_t *act_rows;      // rows with at least one product, in order
    const unsigned long long *nact;
    int64_t *copy_list;           // long single-run rows, filled from the end (shares the heavy list)
    unsigned long long *ncopy;
    int64_t nlist;                // length of the shared list
    int64_t *c_liv;
    double *c_val;
    int64_t cap;
    uint64_t *sk0;
    double *sv0;
    const uint64_t *sk1;
    const double *sv1;
    uint64_t *tile_state;
    uint32_t *tile_ctr;
    WsHeader *hdr;
    // placement by scratch (large problems): c_liv / c_val are the scratch
    // arrays, tile t's outputs start at tile_base[t] and number tile_cnt[t]
    int64_t *tile_cnt;
    int64_t *tile_base;
    unsigned long long *blk_tot;  // per kBlkTiles tiles: sum of their counts
    unsigned long long *sup_tot;  // per kSupTiles tiles: sum of their counts
};

// Placement by scratch: the row kernel adds every tile's count into the
// totals of its block and super-block, so that the compaction finds a
// block's place by summing at most kSupTiles / kBlkTiles block totals and
// the super-block totals before it, with no look-back.
constexpr int kBlkTiles = 8;
constexpr int kSupTiles = 2048;

constexpr int kStage = 32 * 16;           // staged outputs of a tile's register-sorted rows
constexpr int kLaneEnt = 16;              // rows with more entries look their R rows up warp-wide
constexpr int kLaneCopy = 8;              // merged lane rows: entries copied per round of loads

// Per warp: the warp-sort buffer, later reused to stage the outputs of the
// register-sorted rows so that they reach C as coalesced stores.
struct RowsSmem {
    union {
        struct {
            uint64_t pcol[kWarpSortCap];
            double pval[kWarpSortCap];
            uint16_t pslot[kWarpSortCap];
        } sort;
        struct {
            int64_t liv[kStage];
            double val[kStage];
            int32_t soff[33];   // staged start of each lane's row
            int32_t doff[32];   // tile-local output offset of each lane's row
        } stage;
    };
    // register-network rows: product values by slot ([slot][lane]: no bank
    // conflicts); the keys (column, slot) are sorted in registers
    double nval[16][32];
};

__device__ __forceinline__ uint64_t col_of(const DivU64 &div_n, uint64_t nR, int64_t liv) {
    const uint64_t x = (uint64_t)liv;
    return x - divu(div_n, x) * nR;
}

// k-way merge of up to kMergeRuns runs of B entries (columns ascending
// within a run): run i is [st[i], st[i] + ln[i]).  With kWrite, writes
// (base + col, sum of av[i] * b) to out; returns the number of distinct
// columns.  KeyT holds a column (uint32_t when every column fits).
template <bool kWrite, typename KeyT>
__device__ __forceinline__ int lane_merge_g(const RowsArgs &a, const int64_t (&st)[kMergeRuns],
                                            const int32_t (&ln)[kMergeRuns], const double (&av)[kMergeRuns],
                                            int64_t base, int64_t *out_liv,
                                            double *out_val) {
    constexpr KeyT kNone = (KeyT)~(KeyT)0;
    // run i's next entry and the entries it has left; a column is the R
    // entry's LIV less its row's first LIV cb[i] (one division per run),
    // taken in KeyT arithmetic (exact: every column fits KeyT)
    int64_t p[kMergeRuns];
    int32_t left[kMergeRuns];
    KeyT cb[kMergeRuns];
    KeyT hk[kMergeRuns];
#pragma unroll
    for (int i = 0; i < kMergeRuns; ++i) {
        p[i] = st[i];
        left[i] = ln[i];
        cb[i] = 0;
        hk[i] = kNone;
        if (left[i] > 0) {
            const int64_t l0 = a.r_liv[p[i]];
            const uint64_t c0 = col_of(a.div_n, (uint64_t)a.nR, l0);
            cb[i] = (KeyT)((uint64_t)l0 - c0);
            hk[i] = (KeyT)c0;
        }
    }
    int o = 0;
    for (;;) {
        KeyT m = hk[0];
#pragma unroll
        for (int i = 1; i < kMergeRuns; ++i) m = hk[i] < m ? hk[i] : m;
        if (m == kNone) break;
        // products rounded before they are added, and added in run order,
        // starting from the first: the same arithmetic as every other path
        double s = 0.0;
        bool first = true;
#pragma unroll
        for (int i = 0; i < kMergeRuns; ++i) {
            if (hk[i] == m) {
                if (kWrite) {
                    const double pr = __dmul_rn(av[i], a.r_val[p[i]]);
                    s = first ? pr : __dadd_rn(s, pr);
                    first = false;
                }
                ++p[i];
                --left[i];
                hk[i] = left[i] > 0 ? (KeyT)a.r_liv[p[i]] - cb[i] : kNone;
            }
        }
        if (kWrite) {
            out_liv[o] = base + (int64_t)m;
            out_val[o] = s;
        }
        ++o;
    }
    return o;
}

// Sort n (col, val) pairs in place with a bitonic network (elements at
// n..pow2 are treated as +infinity), then sum runs of equal columns and
// compact them to the front.  Whole warp; returns the distinct count.
__device__ int warp_sort_reduce(uint64_t *col, double *val, uint16_t *slot, int n) {
    const int lane = threadIdx.x & 31;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (n2 >> 1); t += 32) {
                const int i = 2 * j * (t / j) + (t % j);
                const int l = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i + j);
                const int lo = i < l ? i : l, hi = i < l ? l : i;
                // (column, slot) order: slots are generation indices, so
                // equal columns keep generation order
                if (hi < n && (col[lo] > col[hi] || (col[lo] == col[hi] && slot[lo] > slot[hi]))) {
                    const uint64_t tc = col[lo];
                    col[lo] = col[hi];
                    col[hi] = tc;
                    const double tv = val[lo];
                    val[lo] = val[hi];
                    val[hi] = tv;
                    const uint16_t ts = slot[lo];
                    slot[lo] = slot[hi];
                    slot[hi] = ts;
                }
            }
            __syncwarp();
        }
    }
    int outc = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int i = c0 + lane;
        const bool head = i < n && (i == 0 || col[i] != col[i - 1]);
        double s = 0.0;
        uint64_t key = 0;
        if (head) {
            key = col[i];
            s = val[i];
            for (int t = i + 1; t < n && col[t] == key; ++t) s += val[t];
        }
        const unsigned hb = __ballot_sync(kFull, head);
        __syncwarp();
        if (head) {
            const int o = outc + __popc(hb & lanemask_lt());
            col[o] = key;
            val[o] = s;
        }
        outc += __popc(hb);
        __syncwarp();
    }
    return outc;
}

enum RowKind { kRowNone = -1, kRowLane = 0, kRowCopy = 1, kRowSort = 2, kRowHeavy = 3, kRowNet = 4 };

// Small rows (at most kNetEnt L entries and kNetProd products) are sorted in
// registers: the products are gathered into kNetProd slots (independent
// loads), sorted by an unrolled bitonic network and kept in registers until
// the row's place in C is known.  KeyT is uint32_t when every column fits.
constexpr int kNetEnt = 8;
constexpr int kNetProd = 16;

// Bitonic network over kNetProd keys (column << 4 | slot): every key is
// distinct, so the order is total and equal columns stay in slot order.
template <typename KeyT>
__device__ __forceinline__ void net_sort(KeyT (&k)[kNetProd]) {
#pragma unroll
    for (int kk = 2; kk <= kNetProd; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < kNetProd; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const KeyT lo = k[i] < k[l] ? k[i] : k[l];
                    const KeyT hi = k[i] < k[l] ? k[l] : k[i];
                    if ((i & kk) == 0) {
                        k[i] = lo;
                        k[l] = hi;
                    } else {
                        k[i] = hi;
                        k[l] = lo;
                    }
                }
            }
        }
    }
}

// Collects the non-empty runs (the B rows selected by the L entries
// [es, ee) of row rid); returns the number of non-empty runs (the first
// kMergeRuns are stored).
__device__ __forceinline__ int collect_runs(const RowsArgs &a, int64_t es, int64_t ee, int64_t rid,
                                            int64_t (&st)[kMergeRuns], int32_t (&ln)[kMergeRuns],
                                            double (&av)[kMergeRuns]) {
    int nr = 0;
    const int64_t rbase = (rid - (int64_t)divu(a.div_h, (uint64_t)rid)) * a.k;
#pragma unroll
    for (int i = 0; i < kMergeRuns; ++i) {
        st[i] = 0;
        ln[i] = 0;
        av[i] = 0.0;
    }
    for (int64_t e = es; e < ee; ++e) {
        int64_t b0, len;
        mdt_lookup_entry(a.mdt, e, a.l_liv, rbase, b0, len);
        if (len > 0) {
            if (nr < kMergeRuns) {
                const double v = a.l_val[e];
#pragma unroll
                for (int i = 0; i < kMergeRuns; ++i)
                    if (i == nr) {
                        st[i] = b0;
                        ln[i] = (int32_t)len;
                        av[i] = v;
                    }
            }
            ++nr;
        }
    }
    return nr;
}

// Direct register-slot gather of a network row (see k_rows): E entries at
// most, each meeting an R row of at most kNetProd / E entries; slot
// s2 + E t holds entry s2's t-th product.
template <int E, typename KeyT>
__device__ __forceinline__ void net_gather_direct(const RowsArgs &a, int64_t es, int64_t nent, int64_t rbase,
                                                  const int64_t (&lv)[kNetEnt], const int64_t (&b0)[kNetEnt],
                                                  const int (&pre)[kNetEnt + 1], KeyT (&nk)[kNetProd],
                                                  double (&nval)[16][32], int lane) {
    constexpr KeyT kNone = (KeyT)~(KeyT)0;
#pragma unroll
    for (int s2 = 0; s2 < E; ++s2) {
        const bool live = s2 < nent;
        const double av = live ? a.l_val[es + s2] : 0.0;
        const int64_t cb = (lv[s2] - rbase) * a.nR;
#pragma unroll
        for (int t = 0; t < kNetProd / E; ++t) {
            const int p = s2 + E * t;
            nk[p] = kNone;
            if (live && t < pre[s2 + 1] - pre[s2]) {
                const int64_t b = b0[s2] + t;
                nk[p] = ((KeyT)(a.r_liv[b] - cb) << 4) | (KeyT)(pre[s2] + t);
                nval[pre[s2] + t][lane] = av * a.r_val[b];
            }
        }
    }
}

// kScratch: each 32-row tile writes its outputs to scratch from the product
// offset of its first row (a row has at most as many outputs as products),
// with no ordering between tiles; k_compact then places the tiles in C.
// Otherwise a CTA takes kWarps consecutive 32-row tiles at a time (one per
// warp) and finds their place in C with one decoupled look-back.
template <typename KeyT, bool kScratch>
__global__ void __launch_bounds__(kRowsThreads, kRowsCtas) k_rows(const __grid_constant__ RowsArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RowsSmem &S = reinterpret_cast<RowsSmem *>(smem_raw)[warp];
    grid_dep_wait();
    if (a.hdr->f > a.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_error(&a.hdr->status, LCO_ERR_CAPACITY);
            a.hdr->nnz_c = 0;
        }
        return;
    }
    constexpr KeyT kNone = (KeyT)~(KeyT)0;
    constexpr int kWarps = kRowsThreads / 32;
    __shared__ int64_t s_ctile, s_goff;
    __shared__ int64_t s_wtot[kWarps];
    const int64_t nact = a.act_rows ? (int64_t)*a.nact : a.hdr->nrows_l;
    const int64_t ntiles = (nact + 31) / 32;
    const int64_t nctiles = (nact + 32 * kWarps - 1) / (32 * kWarps);
    const uint64_t nR = (uint64_t)a.nR;
    for (;;) {
        int64_t t = 0, ct = 0;
        if constexpr (kScratch) {
            int64_t tt = 0;
            if (lane == 0) tt = atomicAdd(a.tile_ctr, 1u);
            t = __shfl_sync(kFull, tt, 0);
            if (t >= ntiles) break;
        } else {
            if (threadIdx.x == 0) s_ctile = atomicAdd(a.tile_ctr, 1u);
            __syncthreads();
            ct = s_ctile;
            if (ct >= nctiles) break;
            t = ct * kWarps + warp;
        }
        const int64_t idx = t * 32 + lane;
        const int64_t r = idx < nact ? (a.act_rows ? a.act_rows[idx] : idx) : -1;
        int kind = kRowNone;
        int64_t es = 0, ee = 0, rid = 0, pb = 0, work = 0;
        int64_t copy_b0 = 0;
        double copy_a = 0.0;
        KeyT nk[kNetProd];
        int64_t cnt = 0;
        if (r >= 0) {
            es = a.row_start[r];
            ee = a.row_start[r + 1];
            const int64_t w0 = a.row_work[r];
            work = a.row_work[r + 1] - w0;
            rid = a.row_id[r];
            pb = w0 - es;
            const int64_t nent = ee - es;
            const int64_t frow = work - nent;
            if (frow == 0) {
                // no entry of the row meets a non-empty R row
                kind = kRowNone;
            } else if (work > kHeavyWork && nent > 1) {
                kind = kRowHeavy;
                cnt = a.row_hout[r] & ((1ll << 62) - 1);
            } else if (nent > kLaneEnt) {
                // many entries, few products (work <= kHeavyWork): the warp
                // looks the entries up in parallel and sorts in shared memory
                kind = kRowSort;
            } else if (nent <= kNetEnt && frow <= kNetProd && (sizeof(KeyT) == 4 || nR < (1ull << 59))) {
                // ---- register network path ----
                kind = kRowNet;
                const int64_t rbase = (rid - (int64_t)divu(a.div_h, (uint64_t)rid)) * a.k;
                int64_t b0[kNetEnt];
                int pre[kNetEnt + 1];
#pragma unroll
                for (int s2 = 0; s2 < kNetEnt; ++s2) {
                    b0[s2] = 0;
                    pre[s2] = 0;
                }
                pre[kNetEnt] = 0;
                int64_t lv[kNetEnt];
#pragma unroll
                for (int s2 = 0; s2 < kNetEnt; ++s2) lv[s2] = s2 < nent ? a.l_liv[es + s2] : 0;
                int run = 0, mx = 0;
#pragma unroll
                for (int s2 = 0; s2 < kNetEnt; ++s2) {
                    int64_t len = 0;
                    if (s2 < nent) mdt_lookup_entry(a.mdt, es + s2, lv[s2] - rbase, b0[s2], len);
                    pre[s2] = run;
                    run += (int)len;
                    mx = (int)len > mx ? (int)len : mx;
                }
                pre[kNetEnt] = run;
                // rows whose R rows are short gather straight into register
                // slots: with at most E entries of at most kNetProd / E
                // products each, entry s2's t-th product takes slot s2 + E t
                // (the sort ignores positions; the key carries the generation
                // index) and its column is its LIV minus the R row's base
                if (mx <= kNetProd / 8) {
                    net_gather_direct<8, KeyT>(a, es, nent, rbase, lv, b0, pre, nk, S.nval, lane);
                } else if (nent <= 4 && mx <= kNetProd / 4) {
                    net_gather_direct<4, KeyT>(a, es, nent, rbase, lv, b0, pre, nk, S.nval, lane);
                } else if (nent <= 2 && mx <= kNetProd / 2) {
                    net_gather_direct<2, KeyT>(a, es, nent, rbase, lv, b0, pre, nk, S.nval, lane);
                } else {
#pragma unroll
                for (int q = 0; q < kNetProd; ++q) {
                    nk[q] = kNone;
                    if (q < run) {
                        int sel = 0;
#pragma unroll
                        for (int s2 = 1; s2 < kNetEnt; ++s2) sel = (pre[s2] <= q) ? s2 : sel;
                        int64_t bsel = b0[0];
                        int psel = pre[0];
#pragma unroll
                        for (int s2 = 1; s2 < kNetEnt; ++s2)
                            if (s2 == sel) {
                                bsel = b0[s2];
                                psel = pre[s2];
                            }
                        const int64_t b = bsel + (q - psel);
                        nk[q] = ((KeyT)col_of(a.div_n, nR, a.r_liv[b]) << 4) | (KeyT)q;
                        S.nval[q][lane] = a.l_val[es + sel] * a.r_val[b];
                    }
                }
                }
                net_sort<KeyT>(nk);
                int u = 0;
#pragma unroll
                for (int q = 0; q < kNetProd; ++q)
                    u += (nk[q] != kNone) && (q == 0 || (nk[q] >> 4) != (nk[q - 1] >> 4));
                cnt = u;
            } else {
                int64_t st[kMergeRuns];
                int32_t ln[kMergeRuns];
                double av[kMergeRuns];
                const int nr = collect_runs(a, es, ee, rid, st, ln, av);
                if (nr <= kMergeRuns && frow <= kLaneProd) {
                    kind = kRowLane;
                    if constexpr (kScratch) {
                        cnt = lane_merge_g<false, KeyT>(a, st, ln, av, 0, nullptr, nullptr);
                    } else {
                        // look-back placement (small L, the latency regime):
                        // merge once, into the product-offset scratch that
                        // warp-sorted rows use, and copy out once placed,
                        // instead of merging a second time after the look-back
                        cnt = lane_merge_g<true, KeyT>(a, st, ln, av, 0, reinterpret_cast<int64_t *>(a.sk0 + pb),
                                                       a.sv0 + pb);
                    }
                } else if (nr == 1) {
                    kind = kRowCopy;
                    cnt = ln[0];
                    copy_b0 = st[0];
                    copy_a = av[0];
                } else {
                    kind = kRowSort;
                }
            }
        }
        // rows sorted by the whole warp (more runs or products than a lane merges)
        unsigned sm = __ballot_sync(kFull, kind == kRowSort);
        while (sm) {
            const int src = __ffs(sm) - 1;
            sm &= sm - 1;
            const int64_t ses = __shfl_sync(kFull, es, src);
            const int64_t see = __shfl_sync(kFull, ee, src);
            const int64_t srid = __shfl_sync(kFull, rid, src);
            const int64_t srb = (srid - (int64_t)divu(a.div_h, (uint64_t)srid)) * a.k;
            const int64_t spb = __shfl_sync(kFull, pb, src);
            int carry = 0;
            for (int64_t e0 = ses; e0 < see; e0 += 32) {
                const int64_t e = e0 + lane;
                int64_t b0 = 0, len = 0;
                double v = 0.0;
                if (e < see) {
                    mdt_lookup_entry(a.mdt, e, a.l_liv, srb, b0, len);
                    v = a.l_val[e];
                }
                int x = (int)len, tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u2 = __shfl_up_sync(kFull, x, o);
                    if (lane >= o) x += u2;
                }
                tot = __shfl_sync(kFull, x, 31);
                const int off = carry + x - (int)len;
                for (int64_t q = 0; q < len; ++q) {
                    S.sort.pcol[off + q] = col_of(a.div_n, nR, a.r_liv[b0 + q]);
                    S.sort.pval[off + q] = v * a.r_val[b0 + q];
                    S.sort.pslot[off + q] = (uint16_t)(off + q);
                }
                carry += tot;
            }
            __syncwarp();
            const int n = warp_sort_reduce(S.sort.pcol, S.sort.pval, S.sort.pslot, carry);
            for (int i = lane; i < n; i += 32) {
                a.sk0[spb + i] = S.sort.pcol[i];
                a.sv0[spb + i] = S.sort.pval[i];
            }
            if (lane == src) cnt = n;
            __syncwarp();
        }
        // exclusive scan of the row counts, then the tile's place in C
        int64_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u2 = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += u2;
        }
        const int64_t tot = __shfl_sync(kFull, x, 31);
        const int64_t off = x - cnt;
        // register-sorted rows: stage their outputs (row-local LIV, value)
        __syncwarp();
        {
            const int ncnt = kind == kRowNet ? (int)cnt : 0;
            int y = ncnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u2 = __shfl_up_sync(kFull, y, o);
                if (lane >= o) y += u2;
            }
            const int soff = y - ncnt;
            S.stage.soff[lane] = soff;
            S.stage.doff[lane] = (int32_t)off;
            if (lane == 31) S.stage.soff[32] = y;
            if (kind == kRowNet) {
                const int64_t cb = rid * a.nR;
                int o = -1;
                KeyT ck = kNone;
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < kNetProd; ++q) {
                    if (nk[q] != kNone) {
                        const KeyT col = nk[q] >> 4;
                        const double v = S.nval[(int)(nk[q] & 15)][lane];
                        if (q == 0 || col != ck) {
                            if (o >= 0) {
                                S.stage.liv[soff + o] = cb + (int64_t)ck;
                                S.stage.val[soff + o] = acc;
                            }
                            ++o;
                            ck = col;
                            acc = v;
                        } else {
                            acc += v;
                        }
                    }
                }
                if (o >= 0) {
                    S.stage.liv[soff + o] = cb + (int64_t)ck;
                    S.stage.val[soff + o] = acc;
                }
            }
        }
        __syncwarp();
        int64_t goff = 0;
        if constexpr (kScratch) {
            // lane 0's row exists (t < ntiles): products before it
            goff = __shfl_sync(kFull, pb, 0);
            if (lane == 0) {
                a.tile_cnt[t] = tot;
                a.tile_base[t] = goff;
                if (tot) {
                    atomicAdd(a.blk_tot + t / kBlkTiles, (unsigned long long)tot);
                    atomicAdd(a.sup_tot + t / kSupTiles, (unsigned long long)tot);
                }
            }
        } else {
            if (lane == 0) s_wtot[warp] = tot;
            __syncthreads();
            if (warp == 0) {
                int64_t ctot = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) ctot += s_wtot[w];
                if (lane == 0) lb_store(a.tile_state + ct, (ct == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)ctot);
                int64_t cg = 0;
                if (ct > 0) cg = (int64_t)lookback_warp(a.tile_state, ct, &a.hdr->status);
                if (lane == 0) {
                    if (ct > 0) lb_store(a.tile_state + ct, kFlagIncl | (uint64_t)(cg + ctot));
                    if (ct == nctiles - 1) a.hdr->nnz_c = cg + ctot;
                    s_goff = cg;
                }
            }
            __syncthreads();
            goff = s_goff;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) goff += w < warp ? s_wtot[w] : 0;
        }
        const int64_t obase = goff + off;
        const int64_t cbase = rid * a.nR;
        {
            // coalesced copy of the staged outputs: entry i belongs to the
            // lane whose staged range holds it (binary search over 32 starts)
            const int ns = S.stage.soff[32];
            if (__all_sync(kFull, kind == kRowNet || kind == kRowNone)) {
                // every row of the tile was staged: staged order is C order
                for (int i = lane; i < ns; i += 32) {
                    a.c_liv[goff + i] = S.stage.liv[i];
                    a.c_val[goff + i] = S.stage.val[i];
                }
            } else {
                for (int i = lane; i < ns; i += 32) {
                    int lo = 0, hi = 32;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.stage.soff[mid] <= i) lo = mid; else hi = mid;
                    }
                    const int64_t g = goff + S.stage.doff[lo] + (i - S.stage.soff[lo]);
                    a.c_liv[g] = S.stage.liv[i];
                    a.c_val[g] = S.stage.val[i];
                }
            }
        }
        if (kind == kRowLane) {
            if constexpr (kScratch) {
                int64_t st[kMergeRuns];
                int32_t ln[kMergeRuns];
                double av[kMergeRuns];
                collect_runs(a, es, ee, rid, st, ln, av);
                lane_merge_g<true, KeyT>(a, st, ln, av, cbase, a.c_liv + obase, a.c_val + obase);
            } else {
                // the merged row, from the product-offset scratch: eight
                // entries' loads in flight at a time
                const uint64_t *hk = a.sk0 + pb;
                const double *hv = a.sv0 + pb;
                for (int64_t i0 = 0; i0 < cnt; i0 += kLaneCopy) {
                    uint64_t kk[kLaneCopy];
                    double vv[kLaneCopy];
#pragma unroll
                    for (int u = 0; u < kLaneCopy; ++u) {
                        kk[u] = i0 + u < cnt ? hk[i0 + u] : 0;
                        vv[u] = i0 + u < cnt ? hv[i0 + u] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < kLaneCopy; ++u) {
                        if (i0 + u < cnt) {
                            a.c_liv[obase + i0 + u] = cbase + (int64_t)kk[u];
                            a.c_val[obase + i0 + u] = vv[u];
                        }
                    }
                }
            }
        }
        // copies done by the whole warp
        unsigned wm = __ballot_sync(kFull, kind == kRowCopy || kind == kRowSort || kind == kRowHeavy);
        while (wm) {
            const int src = __ffs(wm) - 1;
            wm &= wm - 1;
            const int skind = __shfl_sync(kFull, kind, src);
            const int64_t sob = __shfl_sync(kFull, obase, src);
            const int64_t scnt = __shfl_sync(kFull, cnt, src);
            const int64_t scb = __shfl_sync(kFull, cbase, src);
            if (skind == kRowCopy) {
                if (scnt > kHeavyWork) {
                    // long copy: left to k_copy_rows, one CTA per row
                    if (lane == src) {
                        a.row_hout[r] = sob;
                        const unsigned long long q = atomicAdd(a.ncopy, 1ull);
                        a.copy_list[a.nlist - 1 - (int64_t)q] = r;
                    }
                    continue;
                }
                const int64_t b0 = __shfl_sync(kFull, copy_b0, src);
                const double v = __shfl_sync(kFull, copy_a, src);
                for (int64_t i = lane; i < scnt; i += 32) {
                    const int64_t rl = a.r_liv[b0 + i];
                    a.c_liv[sob + i] = scb + (int64_t)col_of(a.div_n, nR, rl);
                    a.c_val[sob + i] = v * a.r_val[b0 + i];
                }
            } else {
                const int64_t spb = __shfl_sync(kFull, pb, src);
                bool second = false;
                if (skind == kRowHeavy) {
                    const int64_t rr = __shfl_sync(kFull, r, src);
                    second = (a.row_hout[rr] >> 62) & 1;
                }
                const uint64_t *hk = (second ? a.sk1 : a.sk0) + spb;
                const double *hv = (second ? a.sv1 : a.sv0) + spb;
                for (int64_t i = lane; i < scnt; i += 32) {
                    a.c_liv[sob + i] = scb + (int64_t)hk[i];
                    a.c_val[sob + i] = hv[i];
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Long single-run rows (one entry of L meets an R row of more than
// kHeavyWork entries): the row of C is that R row scaled by the entry.
// k_rows has placed them (row_hout[r] = output offset); one CTA copies each.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_copy_rows(const __grid_constant__ RowsArgs a) {
    grid_dep_wait();
    if (a.hdr->f > a.cap) return;
    const int64_t ncopy = (int64_t)*a.ncopy;
    for (int64_t q = blockIdx.x; q < ncopy; q += gridDim.x) {
        const int64_t r = a.copy_list[a.nlist - 1 - q];
        const int64_t es = a.row_start[r], ee = a.row_start[r + 1];
        const int64_t rid = a.row_id[r];
        int64_t b0 = 0, len = 0;
        double v = 0.0;
        for (int64_t e = es; e < ee && len == 0; ++e) {   // the row's one matching entry
            mdt_lookup_entry(a.mdt, e, a.l_liv, (rid - (int64_t)divu(a.div_h, (uint64_t)rid)) * a.k, b0, len);
            v = a.l_val[e];
        }
        const int64_t obase = a.row_hout[r];
        const int64_t cbase = rid * a.nR;
        for (int64_t i0 = 0; i0 < len; i0 += 4 * 256) {
            int64_t rl[4];
            double rv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + u * 256 + threadIdx.x;
                if (i < len) {
                    rl[u] = a.r_liv[b0 + i];
                    rv[u] = a.r_val[b0 + i];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = i0 + u * 256 + threadIdx.x;
                if (i < len) {
                    a.c_liv[obase + i] = cbase + (int64_t)col_of(a.div_n, (uint64_t)a.nR, rl[u]);
                    a.c_val[obase + i] = v * rv[u];
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Placement of scratch-mode tiles: C receives tile t's outputs (scratch
// [tile_base[t], + tile_cnt[t])) at the exclusive prefix of the counts.  A
// CTA takes a block of tiles (8, or 32 when there are many tiles), finds the
// block's prefix from the super-block and block totals the row kernel
// accumulated (all known: nothing waits), and spreads the block's entries
// over its threads.
// ------------------------------------------------------------------------
constexpr int kCompactTiles = 32;   // largest block (tiles)
constexpr int kCompactThreads = 256;
constexpr int kCompactCtas = 6;      // resident per SM
constexpr int kCompactUnroll = 4;
constexpr int64_t kCompactWideTiles = 32768;   // from this many tiles, 32-tile blocks
static_assert(kCompactTiles % kBlkTiles == 0 && kSupTiles % kCompactTiles == 0, "compaction block shape");

struct CompactArgs {
    const int64_t *s_liv;
    const double *s_val;
    const int64_t *tile_cnt;
    const int64_t *tile_base;
    const unsigned long long *blk_tot;
    const unsigned long long *sup_tot;
    const int64_t *act_rows;
    const unsigned long long *nact;
    int64_t *c_liv;
    double *c_val;
    int64_t cap;
    WsHeader *hdr;
};

__global__ void __launch_bounds__(kCompactThreads, kCompactCtas) k_compact(const __grid_constant__ CompactArgs a) {
    __shared__ int64_t s_goff;
    __shared__ int64_t s_pre[kCompactTiles + 1];
    __shared__ int64_t s_src[kCompactTiles];
    grid_dep_wait();
    if (a.hdr->f > a.cap) return;
    const int64_t nact = a.act_rows ? (int64_t)*a.nact : a.hdr->nrows_l;
    const int64_t ntiles = (nact + 31) / 32;
    const bool wide = ntiles >= kCompactWideTiles;
    const int tpb = wide ? 32 : 8, steps = wide ? 5 : 3;
    const int64_t nblk = (ntiles + tpb - 1) / tpb;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
        if (tid < 32) {
            const int64_t t0 = b * tpb;
            // the block's prefix: super-blocks before it, then the blocks
            // before it in its super-block
            unsigned long long pre = 0;
            const int64_t ns = t0 / kSupTiles;
            for (int64_t q = lane; q < ns; q += 32) pre += a.sup_tot[q];
            const int64_t b8_end = t0 / kBlkTiles;
            for (int64_t q = ns * (kSupTiles / kBlkTiles) + lane; q < b8_end; q += 32) pre += a.blk_tot[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
            const int64_t t = t0 + lane;
            const bool mine = lane < tpb && t < ntiles;
            const int64_t c = mine ? a.tile_cnt[t] : 0;
            s_src[lane] = mine ? a.tile_base[t] : 0;
            int64_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += u;
            }
            const int64_t tot = __shfl_sync(kFull, x, 31);
            s_pre[lane] = x - c;
            if (lane == 31) s_pre[kCompactTiles] = tot;
            if (lane == 0) {
                s_goff = (int64_t)pre;
                if (b == nblk - 1) a.hdr->nnz_c = (int64_t)pre + tot;
            }
        }
        __syncthreads();
        const int64_t n = s_pre[tpb], g = s_goff;
        // kCompactUnroll entries per thread per step, all loads issued first
        for (int64_t i0 = tid; i0 < n; i0 += kCompactThreads * kCompactUnroll) {
            int64_t src[kCompactUnroll];
#pragma unroll
            for (int u = 0; u < kCompactUnroll; ++u) {
                const int64_t i = i0 + kCompactThreads * u;
                // the tile holding entry i: the last one whose prefix is <= i
                int lo = 0, hi = tpb;
                for (int step = 0; step < steps; ++step) {
                    const int mid = (lo + hi) >> 1;
                    if (s_pre[mid] <= i) lo = mid; else hi = mid;
                }
                src[u] = i < n ? s_src[lo] + (i - s_pre[lo]) : -1;
            }
            int64_t lv[kCompactUnroll];
            double vv[kCompactUnroll];
#pragma unroll
            for (int u = 0; u < kCompactUnroll; ++u) {
                lv[u] = src[u] >= 0 ? a.s_liv[src[u]] : 0;
                vv[u] = src[u] >= 0 ? a.s_val[src[u]] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kCompactUnroll; ++u) {
                if (src[u] >= 0) {
                    a.c_liv[g + i0 + kCompactThreads * u] = lv[u];
                    a.c_val[g + i0 + kCompactThreads * u] = vv[u];
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// SOP (Sec. 5.2.5): expand every product with its output LIV, sort, sum runs
// ------------------------------------------------------------------------
struct SopArgs {
    const int64_t *l_liv;
    const double *l_val;
    const int64_t *r_liv;
    const double *r_val;
    int64_t nnz_l;
    DivU64 div_k;
    int64_t k;
    DivU64 div_h;
    int64_t nR;
    Mdt mdt;
    const int64_t *P;
    int64_t cap;
    int64_t *out_liv;
    double *out_val;
    WsHeader *hdr;
};

__global__ void __launch_bounds__(256) k_sop_expand(const __grid_constant__ SopArgs a) {
    if (a.hdr->f > a.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(&a.hdr->status, LCO_ERR_CAPACITY);
        return;
    }
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.nnz_l; e += gsz) {
        const uint64_t liv = (uint64_t)a.l_liv[e];
        const uint64_t row = divu(a.div_k, liv);
        const int64_t c = r_row(a.div_h, a.k, row, (int64_t)(liv - row * (uint64_t)a.k));
        int64_t b0, len;
        mdt_lookup_entry(a.mdt, e, c, b0, len);
        const int64_t po = a.P[e] - e;
        const double av = a.l_val[e];
        const int64_t rowbase = (int64_t)row * a.nR;
        for (int64_t t = 0; t < len; ++t) {
            const int64_t rl = a.r_liv[b0 + t];
            a.out_liv[po + t] = rowbase + (rl - c * a.nR);
            a.out_val[po + t] = av * a.r_val[b0 + t];
        }
    }
}

struct ReduceArgs {
    const int64_t *key;
    const double *val;
    int64_t cap;
    int64_t *c_liv;
    double *c_val;
    uint64_t *state;
    uint32_t *ctr;
    WsHeader *hdr;
};

__global__ void __launch_bounds__(kCT) k_reduce_by_key(const __grid_constant__ ReduceArgs a) {
    __shared__ int64_t s_tmp[kCW + 1];
    __shared__ int64_t s_tile, s_excl;
    const int64_t n = a.hdr->f;
    if (n > a.cap) return;
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (tile >= ntiles) {
        if (n == 0 && tile == 0 && threadIdx.x == 0) a.hdr->nnz_c = 0;
        return;
    }
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int heads = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < n && (e == 0 || a.key[e] != a.key[e - 1])) ++heads;
    }
    int64_t tot;
    int64_t ex = block_excl<int64_t>((int64_t)heads, s_tmp, &tot);
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) lb_store(a.state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
        int64_t e = 0;
        if (tile > 0) e = (int64_t)lookback_warp(a.state, tile, &a.hdr->status);
        if (threadIdx.x == 0) {
            if (tile > 0) lb_store(a.state + tile, kFlagIncl | (uint64_t)(e + tot));
            s_excl = e;
            if (tile == ntiles - 1) a.hdr->nnz_c = e + tot;
        }
    }
    __syncthreads();
    int64_t o = s_excl + ex;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t e = base + i;
        if (e < n && (e == 0 || a.key[e] != a.key[e - 1])) {
            double s = a.val[e];
            for (int64_t t = e + 1; t < n && a.key[t] == a.key[e]; ++t) s += a.val[t];
            a.c_liv[o] = a.key[e];
            a.c_val[o] = s;
            ++o;
        }
    }
}

__global__ void k_set_empty(WsHeader *hdr, int32_t alg) {
    hdr->alg = alg;
    hdr->f = 0;
    hdr->work_total = 0;
    hdr->nchunks = 0;
    hdr->nnz_c = 0;
    hdr->nzr_b = 0;
}

int sm_count() { return radix_sm_count(); }

int bits_host(uint64_t range) {
    int b = 0;
    while (b < 63 && (1ull << b) < range) ++b;
    return b;
}

}  // namespace

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
}  // namespace lco

struct lco_plan {
    lco::RpPlan rp_l, rp_r;      // L and R rearrangements (source shapes -> matrix orders)
    lco_shape src_l, src_r;      // shapes of the operands feeding L and R
    int32_t l_is_a;              // 1: L = A (row variants), 0: L = B (column variants)
    int32_t need_l, need_r;
    int32_t lookup;              // lco::Lookup
    int32_t acc;                 // 1 accumulator, 0 no accumulator, 2 SOP
    int64_t mL, k, nR;
    int64_t rows_h;              // L rows per value of the entrywise indices (mL without them)
    int64_t kr;                  // R's rows: k per value of the entrywise indices
    int64_t nnz_l, nnz_r;
    int32_t colbits;
    int32_t aux_shift;
    int64_t naux;
    int32_t sop_bits;
    lco_plan_info info;
    // workspace layout (offsets from ws)
    size_t off_l_liv, off_l_val, off_r_liv, off_r_val, off_rp;
    size_t off_p1state, p1state_bytes;
    size_t off_mdt_rowptr, off_mdt_rowid, off_mdt_aux;
    size_t off_P;                    // per-entry work prefix (SOP only)
    size_t off_row_start, off_row_id, off_row_work, off_row_hout, off_heavy, off_ec;
    size_t phase1_end;
};

namespace lco {
namespace {

int sparsity_class(int64_t rows, int64_t cols, int64_t nnz) {
    if (nnz <= 0) return 3;
    const bool rs = (double)rows / (double)nnz > 3.0;
    const bool cs = (double)cols / (double)nnz > 3.0;
    return rs && cs ? 3 : (rs ? 1 : (cs ? 2 : 0));
}

// Table 4 (rows: A class, columns: B class; order sparse, row-, column-, index-sparse).
// Values >= 10 mark cells naming a column/row pair.
const int kTable4[4][4] = {
    {10, LCO_ALG_CSC, LCO_ALG_CSC, LCO_ALG_CSC},
    {LCO_ALG_CSR, LCO_ALG_DCSR, 12, LCO_ALG_CSCNA},
    {LCO_ALG_CSR, 11, LCO_ALG_DCSC, LCO_ALG_DCSC},
    {LCO_ALG_CSR, LCO_ALG_DCSR, LCO_ALG_CSRNA, LCO_ALG_SOP},
};

bool same_sig(int order, const int32_t *a, const int32_t *b) {
    for (int i = 0; i < order; ++i)
        if (a[i] != b[i]) return false;
    return true;
}

// Phase-2 workspace layout (offsets from the end of the phase-1 region).
struct P2Layout {
    int64_t capc, nchunks_max;
    size_t chunk_state, chunk_ctr, reduce_state, table_state, zero_bytes;
    size_t act_rows;
    size_t arr[6];          // cap-sized scratch arrays (8 bytes per entry; 4 used off SOP, 6 with placement by scratch)
    size_t tile_cnt, tile_base;   // placement by scratch: per 32-row tile
    size_t blk_tot, sup_tot;      // placement by scratch: block and super-block totals (zeroed)
    size_t sop_radix;
    int sop_D, sop_P;
    size_t total;
};

P2Layout p2_layout(const lco_plan *p, int64_t cap);

size_t contract_phase2_bytes(const lco_plan *p, int64_t cap) { return p2_layout(p, cap).total; }

// Row kernels place their outputs through scratch (k_rows<., true> +
// k_compact) when L has this many entries: with thousands of 32-row tiles in
// flight, ordering them by look-back makes every tile wait for the slowest
// of its predecessors.
constexpr int64_t kScratchMinEntries = 1 << 16;
bool rows_scratch(const lco_plan *p) { return p->acc != 2 && p->nnz_l >= kScratchMinEntries; }

}  // namespace
}  // namespace lco

using namespace lco;

extern "C" {

int32_t lco_contract_plan(const lco_shape *a, const lco_shape *b, int32_t ncontract, const int32_t *modes_a,
                          const int32_t *modes_b, int32_t force_alg, lco_plan **plan_out) {
    lco_tune t;
    t.alg = force_alg;
    t.max_digit_bits = 0;
    t.radix_order = 0;
    return lco_contract_plan_ex(a, b, ncontract, modes_a, modes_b, &t, plan_out);
}

int32_t lco_contract_plan_ex(const lco_shape *a, const lco_shape *b, int32_t ncontract, const int32_t *modes_a,
                             const int32_t *modes_b, const lco_tune *tune, lco_plan **plan_out) {
    return lco_contract_plan_entrywise(a, b, ncontract, modes_a, modes_b, 0, nullptr, nullptr, tune, plan_out);
}

int32_t lco_contract_plan_entrywise(const lco_shape *a, const lco_shape *b, int32_t ncontract,
                                    const int32_t *modes_a, const int32_t *modes_b, int32_t nentry,
                                    const int32_t *emodes_a, const int32_t *emodes_b, const lco_tune *tune,
                                    lco_plan **plan_out) {
    const int32_t force_alg = tune ? tune->alg : LCO_ALG_AUTO;
    const int max_bits = tune && tune->max_digit_bits > 0 ? tune->max_digit_bits : kDefaultDigitBits;
    if (tune && (tune->max_digit_bits < 0 || tune->max_digit_bits > kMaxDigitBits)) return LCO_ERR_INVALID;
    if (tune && (tune->radix_order < 0 || tune->radix_order > 1)) return LCO_ERR_INVALID;
    if (!plan_out) return LCO_ERR_INVALID;
    *plan_out = nullptr;
    int64_t ta, tb;
    int32_t rc;
    if ((rc = check_shape(a, &ta)) != LCO_OK) return rc;
    if ((rc = check_shape(b, &tb)) != LCO_OK) return rc;
    if (ncontract < 0 || ncontract > a->order || ncontract > b->order) return LCO_ERR_INVALID;
    if (ncontract > 0 && (!modes_a || !modes_b)) return LCO_ERR_INVALID;
    if (force_alg < -1 || force_alg > LCO_ALG_SOP) return LCO_ERR_INVALID;
    int con_a[kMaxOrder] = {0}, con_b[kMaxOrder] = {0};
    for (int i = 0; i < ncontract; ++i) {
        const int ma = modes_a[i], mb = modes_b[i];
        if (ma < 0 || ma >= a->order || mb < 0 || mb >= b->order) return LCO_ERR_INVALID;
        if (con_a[ma] || con_b[mb]) return LCO_ERR_INVALID;
        if (a->dims[ma] != b->dims[mb]) return LCO_ERR_INVALID;
        con_a[ma] = con_b[mb] = 1;
    }
    // entrywise pairs (Sec. 5): shared, kept in C, not summed
    if (nentry < 0 || ncontract + nentry > a->order || ncontract + nentry > b->order) return LCO_ERR_INVALID;
    if (nentry > 0 && (!emodes_a || !emodes_b)) return LCO_ERR_INVALID;
    int64_t H = 1;
    for (int i = 0; i < nentry; ++i) {
        const int ma = emodes_a[i], mb = emodes_b[i];
        if (ma < 0 || ma >= a->order || mb < 0 || mb >= b->order) return LCO_ERR_INVALID;
        if (con_a[ma] || con_b[mb]) return LCO_ERR_INVALID;
        if (a->dims[ma] != b->dims[mb]) return LCO_ERR_INVALID;
        con_a[ma] = con_b[mb] = 2;
        H *= a->dims[ma];
    }
    int free_a[kMaxOrder], free_b[kMaxOrder], nfa = 0, nfb = 0;
    for (int t = 0; t < a->order; ++t) if (!con_a[t]) free_a[nfa++] = t;
    for (int t = 0; t < b->order; ++t) if (!con_b[t]) free_b[nfb++] = t;
    if (nentry + nfa + nfb > kMaxOrder) return LCO_ERR_INVALID;
    int64_t m = 1, k = 1, n = 1;
    for (int i = 0; i < nfa; ++i) m *= a->dims[free_a[i]];
    for (int i = 0; i < ncontract; ++i) k *= a->dims[modes_a[i]];
    for (int i = 0; i < nfb; ++i) n *= b->dims[free_b[i]];
    if (m > INT64_MAX / n || H > INT64_MAX / (m * n)) return LCO_ERR_OVERFLOW;

    // matrix orders (most significant first), converted to sig (least significant first)
    int32_t a_row[kMaxOrder], a_col[kMaxOrder], b_row[kMaxOrder], b_col[kMaxOrder];
    {
        // the entrywise modes lead every matrix order: one matrix product
        // per value of them (Sec. 5)
        int32_t msf[kMaxOrder];
        int q = 0;
        for (int i = 0; i < nentry; ++i) msf[q++] = emodes_a[i];
        for (int i = 0; i < nfa; ++i) msf[q++] = free_a[i];
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_a[i];
        for (int i = 0; i < q; ++i) a_row[i] = msf[q - 1 - i];
        q = 0;
        for (int i = 0; i < nentry; ++i) msf[q++] = emodes_a[i];
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_a[i];
        for (int i = 0; i < nfa; ++i) msf[q++] = free_a[i];
        for (int i = 0; i < q; ++i) a_col[i] = msf[q - 1 - i];
        q = 0;
        for (int i = 0; i < nentry; ++i) msf[q++] = emodes_b[i];
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_b[i];
        for (int i = 0; i < nfb; ++i) msf[q++] = free_b[i];
        for (int i = 0; i < q; ++i) b_row[i] = msf[q - 1 - i];
        q = 0;
        for (int i = 0; i < nentry; ++i) msf[q++] = emodes_b[i];
        for (int i = 0; i < nfb; ++i) msf[q++] = free_b[i];
        for (int i = 0; i < ncontract; ++i) msf[q++] = modes_b[i];
        for (int i = 0; i < q; ++i) b_col[i] = msf[q - 1 - i];
    }
    const int perm_row = !same_sig(a->order, a->sig, a_row) + !same_sig(b->order, b->sig, b_row);
    const int perm_col = !same_sig(a->order, a->sig, a_col) + !same_sig(b->order, b->sig, b_col);
    // the flattened operands ((h, i) x (h, k) and (h, k) x (h, j)) have the
    // per-batch ratios dim / (nnz / H)
    const int ca = sparsity_class(H * m, H * k, a->nnz), cb = sparsity_class(H * k, H * n, b->nnz);
    int alg = force_alg;
    if (alg < 0) {
        const int cell = kTable4[ca][cb];
        if (cell < 10) {
            alg = cell;
        } else {
            const bool colv = perm_col < perm_row ? true : (perm_row < perm_col ? false : n > m);
            alg = cell == 10 ? (colv ? LCO_ALG_CSC : LCO_ALG_CSR)
                : cell == 11 ? (colv ? LCO_ALG_DCSC : LCO_ALG_DCSR)
                             : (colv ? LCO_ALG_CSCNA : LCO_ALG_CSRNA);
        }
    }
    const bool transposed = alg == LCO_ALG_CSC || alg == LCO_ALG_DCSC || alg == LCO_ALG_CSCNA;

    lco_plan *p = new (std::nothrow) lco_plan();
    if (!p) return LCO_ERR_OOM;
    std::memset(p, 0, sizeof(*p));
    p->l_is_a = !transposed;
    p->src_l = transposed ? *b : *a;
    p->src_r = transposed ? *a : *b;
    const int32_t *l_target = transposed ? b_col : a_row;
    const int32_t *r_target = transposed ? a_col : b_row;
    if ((rc = rp_plan(&p->src_l, l_target, &p->rp_l, max_bits)) != LCO_OK) { delete p; return rc; }
    if ((rc = rp_plan(&p->src_r, r_target, &p->rp_r, max_bits)) != LCO_OK) { delete p; return rc; }
    p->rp_l.lsd_only = p->rp_r.lsd_only = tune ? tune->radix_order : 0;
    p->need_l = !same_sig(p->src_l.order, p->src_l.sig, l_target);
    p->need_r = !same_sig(p->src_r.order, p->src_r.sig, r_target);
    p->rows_h = transposed ? n : m;
    p->mL = H * p->rows_h;
    p->nR = transposed ? m : n;
    p->k = k;
    p->kr = H * k;
    p->nnz_l = p->src_l.nnz;
    p->nnz_r = p->src_r.nnz;
    p->colbits = bits_host((uint64_t)p->nR);
    p->acc = (alg == LCO_ALG_SOP) ? 2 : ((alg == LCO_ALG_CSRNA || alg == LCO_ALG_CSCNA) ? 0 : 1);
    p->lookup = (alg == LCO_ALG_DCSR || alg == LCO_ALG_DCSC || alg == LCO_ALG_SOP) ? kLookupDcsr : kLookupCsr;
    // keys of the chunk kernel pack (local row < 2^11, column): wide columns go to SOP
    if (p->acc != 2 && p->colbits > 52) {
        p->acc = 2;
        p->lookup = kLookupDcsr;
    }
    p->sop_bits = bits_host((uint64_t)p->mL * (uint64_t)p->nR);
    {
        uint64_t na = 1;
        while (na < (uint64_t)(p->nnz_r > 0 ? p->nnz_r : 1)) na <<= 1;
        const int kb = bits_host((uint64_t)p->kr);
        const int nb = bits_host(na);
        p->aux_shift = kb > nb ? kb - nb : 0;
        p->naux = (int64_t)(((uint64_t)(p->kr - 1) >> p->aux_shift) + 1);
    }
    // info
    p->info.alg = alg;
    p->info.transposed = transposed;
    p->info.class_a = ca;
    p->info.class_b = cb;
    p->info.permute_a = transposed ? p->need_r : p->need_l;
    p->info.permute_b = transposed ? p->need_l : p->need_r;
    p->info.m = m;
    p->info.k = k;
    p->info.n = n;
    {
        // C's modes: the entrywise pairs, A's free modes, B's free modes
        lco_shape &cs = p->info.c_shape;
        cs.order = nentry + nfa + nfb;
        int q = 0;
        for (int i = 0; i < nentry; ++i) cs.dims[q++] = a->dims[emodes_a[i]];
        for (int i = 0; i < nfa; ++i) cs.dims[q++] = a->dims[free_a[i]];
        for (int i = 0; i < nfb; ++i) cs.dims[q++] = b->dims[free_b[i]];
        if (cs.order == 0) {
            cs.order = 1;
            cs.dims[0] = 1;
            cs.sig[0] = 0;
        } else if (!transposed) {
            for (int i = 0; i < cs.order; ++i) cs.sig[i] = cs.order - 1 - i;
        } else {
            // most significant first: the entrywise modes, B's free modes,
            // then A's free modes
            int32_t msf[kMaxOrder];
            int t = 0;
            for (int i = 0; i < nentry; ++i) msf[t++] = i;
            for (int i = 0; i < nfb; ++i) msf[t++] = nentry + nfa + i;
            for (int i = 0; i < nfa; ++i) msf[t++] = nentry + i;
            for (int i = 0; i < cs.order; ++i) cs.sig[i] = msf[cs.order - 1 - i];
        }
        cs.nnz = 0;
    }
    // workspace layout, phase 1
    size_t off = kWsHeaderBytes;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes ? bytes : 1); return o; };
    const int64_t nl = p->nnz_l > 0 ? p->nnz_l : 1, nr = p->nnz_r > 0 ? p->nnz_r : 1;
    // the phase-1 look-back words follow the header, so one memset resets both
    {
        const size_t scan_tiles = (size_t)((nl + kScanTile - 1) / kScanTile) + 1;
        const size_t dcsr_tiles = (size_t)((nr + kScanTile - 1) / kScanTile) + 1;
        p->off_p1state = take((2 * scan_tiles + dcsr_tiles) * 8);
        p->p1state_bytes = align_up((2 * scan_tiles + dcsr_tiles) * 8);
    }
    p->off_l_liv = p->need_l ? take((size_t)nl * 8) : 0;
    p->off_l_val = p->need_l ? take((size_t)nl * 8) : 0;
    p->off_r_liv = p->need_r ? take((size_t)nr * 8) : 0;
    p->off_r_val = p->need_r ? take((size_t)nr * 8) : 0;
    {
        size_t rb = 0;
        if (p->need_l) rb = rp_region_bytes(p->rp_l, p->nnz_l);
        if (p->need_r) { size_t x = rp_region_bytes(p->rp_r, p->nnz_r); if (x > rb) rb = x; }
        p->off_rp = take(rb);
    }
    if (p->lookup == kLookupCsr) {
        p->off_mdt_rowptr = take((size_t)(p->kr + 1) * 8);
    } else {
        p->off_mdt_rowptr = take((size_t)(nr + 1) * 8);
        p->off_mdt_rowid = take((size_t)nr * 8);
        p->off_mdt_aux = take((size_t)(p->naux + 1) * 8);
    }
    p->off_P = p->acc == 2 ? take((size_t)(nl + 1) * 8) : 0;
    // DCSR: the scan keeps every entry's lookup so that phase 2 reads it
    // instead of searching R's row ids again
    p->off_ec = p->lookup == kLookupDcsr ? take((size_t)nl * 8) : 0;
    p->off_row_start = take((size_t)(nl + 1) * 8);
    p->off_row_id = take((size_t)nl * 8);
    p->off_row_work = take((size_t)(nl + 1) * 8);
    p->off_row_hout = take((size_t)nl * 8);
    p->off_heavy = take((size_t)nl * 8);
    p->phase1_end = off;
    *plan_out = p;
    return LCO_OK;
}

int32_t lco_plan_get_info(const lco_plan *plan, lco_plan_info *info) {
    if (!plan || !info) return LCO_ERR_INVALID;
    *info = plan->info;
    return LCO_OK;
}

int32_t lco_plan_destroy(lco_plan *plan) {
    delete plan;
    return LCO_OK;
}

int32_t lco_contract_workspace(const lco_plan *plan, int64_t cap, size_t *ws_bytes) {
    if (!plan || !ws_bytes || cap < 0) return LCO_ERR_INVALID;
    *ws_bytes = plan->phase1_end + contract_phase2_bytes(plan, cap);
    return LCO_OK;
}

}  // extern "C"

namespace lco {
namespace {

struct Operands {
    const int64_t *l_liv;
    const double *l_val;
    const int64_t *r_liv;
    const double *r_val;
};

Operands operands(const lco_plan *p, const int64_t *a_liv, const double *a_val, const int64_t *b_liv,
                  const double *b_val, char *ws) {
    Operands o;
    const int64_t *src_l_liv = p->l_is_a ? a_liv : b_liv;
    const double *src_l_val = p->l_is_a ? a_val : b_val;
    const int64_t *src_r_liv = p->l_is_a ? b_liv : a_liv;
    const double *src_r_val = p->l_is_a ? b_val : a_val;
    o.l_liv = p->need_l ? reinterpret_cast<int64_t *>(ws + p->off_l_liv) : src_l_liv;
    o.l_val = p->need_l ? reinterpret_cast<double *>(ws + p->off_l_val) : src_l_val;
    o.r_liv = p->need_r ? reinterpret_cast<int64_t *>(ws + p->off_r_liv) : src_r_liv;
    o.r_val = p->need_r ? reinterpret_cast<double *>(ws + p->off_r_val) : src_r_val;
    return o;
}

Mdt make_mdt(const lco_plan *p, char *ws) {
    Mdt m{};
    m.kind = p->lookup;
    m.k = p->kr;
    m.nnz = p->nnz_r;
    m.row_ptr = reinterpret_cast<int64_t *>(ws + p->off_mdt_rowptr);
    if (p->lookup == kLookupDcsr) {
        m.row_id = reinterpret_cast<int64_t *>(ws + p->off_mdt_rowid);
        m.aux = reinterpret_cast<int64_t *>(ws + p->off_mdt_aux);
        m.aux_shift = p->aux_shift;
        m.naux = p->naux;
        m.ec = reinterpret_cast<const uint64_t *>(ws + p->off_ec);
    }
    return m;
}

bool check_ptrs(const lco_plan *p, const int64_t *a_liv, const double *a_val, const int64_t *b_liv,
                const double *b_val) {
    const int64_t na = p->l_is_a ? p->nnz_l : p->nnz_r;
    const int64_t nb = p->l_is_a ? p->nnz_r : p->nnz_l;
    if (na > 0 && (!a_liv || !a_val)) return false;
    if (nb > 0 && (!b_liv || !b_val)) return false;
    return true;
}

int32_t symbolic_enqueue(const lco_plan *p, const int64_t *a_liv, const double *a_val, const int64_t *b_liv,
                         const double *b_val, char *ws, cudaStream_t s) {
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    // reset header (status, results, counters) and the phase-1 look-back
    // state, which follows it
    if (cudaMemsetAsync(ws, 0, p->off_p1state + p->p1state_bytes, s) != cudaSuccess) return LCO_ERR_CUDA;
    if (p->nnz_l == 0 || p->nnz_r == 0) {
        LCO_LAUNCH("k_set_empty", s, k_set_empty<<<1, 1, 0, s>>>(hdr, p->info.alg));
        return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
    }
    const int64_t *src_l_liv = p->l_is_a ? a_liv : b_liv;
    const double *src_l_val = p->l_is_a ? a_val : b_val;
    const int64_t *src_r_liv = p->l_is_a ? b_liv : a_liv;
    const double *src_r_val = p->l_is_a ? b_val : a_val;
    Operands o = operands(p, a_liv, a_val, b_liv, b_val, ws);
    char *rp_region = ws + p->off_rp;
    if (p->need_l) {
        if (rp_enqueue(p->rp_l, p->nnz_l, src_l_liv, src_l_val, const_cast<int64_t *>(o.l_liv),
                       const_cast<double *>(o.l_val), rp_region, hdr, s) != cudaSuccess)
            return LCO_ERR_CUDA;
    }
    if (p->need_r) {
        if (rp_enqueue(p->rp_r, p->nnz_r, src_r_liv, src_r_val, const_cast<int64_t *>(o.r_liv),
                       const_cast<double *>(o.r_val), rp_region, hdr, s) != cudaSuccess)
            return LCO_ERR_CUDA;
    }
    const int sms = sm_count();
    Mdt mdt = make_mdt(p, ws);
    const DivU64 div_n = make_div((uint64_t)p->nR);
    uint64_t *scan_state = reinterpret_cast<uint64_t *>(ws + p->off_p1state);
    uint64_t *dcsr_state = scan_state + 2 * (((p->nnz_l + kScanTile - 1) / kScanTile) + 1);
    if (p->lookup == kLookupCsr) {
        int64_t grid = (std::max<int64_t>(p->nnz_r, p->kr + 1) + 255) / 256;
        if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
        LCO_LAUNCH("k_csr_rowptr", s, k_csr_rowptr<<<(unsigned)grid, 256, 0, s>>>(o.r_liv, p->nnz_r, div_n, p->kr,
                                                    const_cast<int64_t *>(mdt.row_ptr)));
    } else {
        DcsrArgs d{};
        d.liv = o.r_liv;
        d.nnz = p->nnz_r;
        d.div_n = div_n;
        d.row_id = const_cast<int64_t *>(mdt.row_id);
        d.row_ptr = const_cast<int64_t *>(mdt.row_ptr);
        d.state = dcsr_state;
        d.hdr = hdr;
        const int64_t tiles = (p->nnz_r + kScanTile - 1) / kScanTile;
        LCO_LAUNCH("k_dcsr_build", s, k_dcsr_build<<<(unsigned)tiles, kCT, 0, s>>>(d));
        int64_t grid = (p->nnz_r + 1 + 255) / 256;
        if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
        LCO_LAUNCH("k_dcsr_aux", s, k_dcsr_aux<<<(unsigned)grid, 256, 0, s>>>(mdt.row_id, hdr, p->aux_shift, p->naux,
                                                  const_cast<int64_t *>(mdt.aux), p->nnz_r));
    }
    ScanArgs sa{};
    sa.alg = p->info.alg;
    sa.l_liv = o.l_liv;
    sa.nnz_l = p->nnz_l;
    sa.div_k = make_div((uint64_t)p->k);
    sa.k = p->k;
    sa.div_h = make_div((uint64_t)p->rows_h);
    sa.mdt = mdt;
    sa.P = p->acc == 2 ? reinterpret_cast<int64_t *>(ws + p->off_P) : nullptr;
    if (p->lookup == kLookupDcsr) {
        Mdt m0 = mdt;
        m0.ec = nullptr;
        int64_t grid = (p->nnz_l + 255) / 256;
        if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
        LCO_LAUNCH("k_entry_lookup", s, k_entry_lookup<<<(unsigned)grid, 256, 0, s>>>(
                                            o.l_liv, p->nnz_l, sa.div_k, p->k, sa.div_h, m0,
                                            reinterpret_cast<uint64_t *>(ws + p->off_ec)));
    }
    sa.row_start = reinterpret_cast<int64_t *>(ws + p->off_row_start);
    sa.row_id = reinterpret_cast<int64_t *>(ws + p->off_row_id);
    sa.row_work = reinterpret_cast<int64_t *>(ws + p->off_row_work);
    sa.state_w = scan_state;
    sa.state_h = scan_state + ((p->nnz_l + kScanTile - 1) / kScanTile) + 1;
    sa.hdr = hdr;
    const int64_t tiles = (p->nnz_l + kScanTile - 1) / kScanTile;
    // after a kernel (the row-pointer, DCSR or lookup launch): dependent launch
    LCO_LAUNCH("k_work_scan", s, launch_dependent(k_work_scan, (unsigned)tiles, kCT, 0, s, sa));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

int32_t numeric_enqueue(const lco_plan *p, const int64_t *a_liv, const double *a_val, const int64_t *b_liv,
                        const double *b_val, int64_t *c_liv, double *c_val, int64_t cap, char *ws,
                        cudaStream_t s) {
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    if (p->nnz_l == 0 || p->nnz_r == 0) {
        LCO_LAUNCH("k_set_empty", s, k_set_empty<<<1, 1, 0, s>>>(hdr, p->info.alg));
        return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
    }
    Operands o = operands(p, a_liv, a_val, b_liv, b_val, ws);
    const P2Layout L = p2_layout(p, cap);
    const int64_t capc = L.capc;
    const int64_t nchunks_max = L.nchunks_max;
    char *p2 = ws + p->phase1_end;
    uint64_t *chunk_state = reinterpret_cast<uint64_t *>(p2 + L.chunk_state);
    uint32_t *chunk_ctr = reinterpret_cast<uint32_t *>(p2 + L.chunk_ctr);
    uint64_t *reduce_state = reinterpret_cast<uint64_t *>(p2 + L.reduce_state);
    uint64_t *sk0 = reinterpret_cast<uint64_t *>(p2 + L.arr[0]);
    double *sv0 = reinterpret_cast<double *>(p2 + L.arr[1]);
    uint64_t *sk1 = reinterpret_cast<uint64_t *>(p2 + L.arr[2]);
    double *sv1 = reinterpret_cast<double *>(p2 + L.arr[3]);
    uint64_t *sk2 = reinterpret_cast<uint64_t *>(p2 + L.arr[4]);
    double *sv2 = reinterpret_cast<double *>(p2 + L.arr[5]);
    char *sop_region = p2 + L.sop_radix;
    if (cudaMemsetAsync(p2, 0, L.zero_bytes, s) != cudaSuccess) return LCO_ERR_CUDA;
    Mdt mdt = make_mdt(p, ws);
    const int sms = sm_count();
    const int64_t *P = reinterpret_cast<const int64_t *>(ws + p->off_P);
    if (p->acc != 2) {
        int64_t *row_start = reinterpret_cast<int64_t *>(ws + p->off_row_start);
        int64_t *row_id = reinterpret_cast<int64_t *>(ws + p->off_row_id);
        int64_t *row_work = reinterpret_cast<int64_t *>(ws + p->off_row_work);
        int64_t *row_hout = reinterpret_cast<int64_t *>(ws + p->off_row_hout);
        int64_t *heavy = reinterpret_cast<int64_t *>(ws + p->off_heavy);
        unsigned long long *nheavy = reinterpret_cast<unsigned long long *>(chunk_ctr + 4);
        int64_t *act_rows = reinterpret_cast<int64_t *>(p2 + L.act_rows);
        unsigned long long *nact = reinterpret_cast<unsigned long long *>(chunk_ctr + 10);
        TableArgs ta{};
        ta.row_start = row_start;
        ta.row_work = row_work;
        ta.heavy_list = heavy;
        ta.nheavy = nheavy;
        ta.act_rows = act_rows;
        ta.nact = nact;
        ta.state = reinterpret_cast<uint64_t *>(p2 + L.table_state);
        ta.tile_ctr = chunk_ctr + 8;
        ta.cap = cap;
        ta.hdr = hdr;
        // Rows with no product are dropped from the light-row kernel's tiles
        // only when R is row-sparse (DCSR): then many L entries miss R.
        // Otherwise nearly every row is active and the ordered compaction,
        // a chain of look-backs, would cost more than it saves.
        const bool compact = p->lookup == kLookupDcsr;
        if (compact) {
            // persistent CTAs over tiles of rows (the rows are at most L's entries)
            int64_t grid = (p->nnz_l + kTabTile - 1) / kTabTile;
            if (grid > (int64_t)sms * 2) grid = (int64_t)sms * 2;
            LCO_LAUNCH("k_row_table", s, k_row_table<<<(unsigned)(grid > 0 ? grid : 1), kCT, 0, s>>>(ta));
        } else {
            int64_t grid = (p->nnz_l + 1 + 255) / 256;
            if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
            LCO_LAUNCH("k_row_heavy", s, k_row_heavy<<<(unsigned)grid, 256, 0, s>>>(ta));
        }
        HeavyArgs ha{};
        ha.l_liv = o.l_liv;
        ha.l_val = o.l_val;
        ha.r_liv = o.r_liv;
        ha.r_val = o.r_val;
        ha.div_k = make_div((uint64_t)p->k);
        ha.k = p->k;
        ha.div_h = make_div((uint64_t)p->rows_h);
        ha.div_n = make_div((uint64_t)p->nR);
        ha.nR = p->nR;
        ha.colbits = p->colbits;
        ha.mdt = mdt;
        ha.row_start = row_start;
        ha.row_work = row_work;
        ha.heavy_list = heavy;
        ha.nheavy = nheavy;
        ha.row_hout = row_hout;
        ha.cap = cap;
        ha.sk0 = sk0;
        ha.sv0 = sv0;
        ha.sk1 = sk1;
        ha.sv1 = sv1;
        ha.ctr = chunk_ctr + 2;
        ha.hdr = hdr;
        ha.acc = p->acc;
        // function attributes are per device: set them once on each
        static std::atomic<uint64_t> attr_done{0};
        int dev = 0;
        cudaGetDevice(&dev);
        const uint64_t bit = 1ull << (dev & 63);
        if (!(attr_done.load() & bit)) {
            cudaFuncSetAttribute(k_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeavySmemBytes);
            const int rows_smem = (int)sizeof(RowsSmem) * (kRowsThreads / 32);
            cudaFuncSetAttribute(k_rows<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem);
            cudaFuncSetAttribute(k_rows<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem);
            cudaFuncSetAttribute(k_rows<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem);
            cudaFuncSetAttribute(k_rows<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem);
            attr_done.fetch_or(bit);
        }
        // this and the launches below follow a kernel: dependent launches
        LCO_LAUNCH("k_heavy", s, launch_dependent(k_heavy, (unsigned)sms, kCT, kHeavySmemBytes, s, ha));
        RowsArgs ra{};
        ra.l_liv = o.l_liv;
        ra.l_val = o.l_val;
        ra.r_liv = o.r_liv;
        ra.r_val = o.r_val;
        ra.k = p->k;
        ra.div_h = make_div((uint64_t)p->rows_h);
        ra.div_n = make_div((uint64_t)p->nR);
        ra.nR = p->nR;
        ra.mdt = mdt;
        ra.row_start = row_start;
        ra.row_id = row_id;
        ra.row_work = row_work;
        ra.row_hout = row_hout;
        ra.act_rows = compact ? act_rows : nullptr;
        ra.nact = nact;
        ra.copy_list = heavy;
        ra.ncopy = reinterpret_cast<unsigned long long *>(chunk_ctr + 6);
        ra.nlist = p->nnz_l;
        ra.c_liv = c_liv;
        ra.c_val = c_val;
        ra.cap = cap;
        ra.sk0 = sk0;
        ra.sv0 = sv0;
        ra.sk1 = sk1;
        ra.sv1 = sv1;
        ra.tile_state = chunk_state;
        ra.tile_ctr = chunk_ctr;
        ra.hdr = hdr;
        const bool scratch = rows_scratch(p);
        if (scratch) {
            ra.c_liv = reinterpret_cast<int64_t *>(p2 + L.arr[4]);
            ra.c_val = reinterpret_cast<double *>(p2 + L.arr[5]);
            ra.tile_cnt = reinterpret_cast<int64_t *>(p2 + L.tile_cnt);
            ra.tile_base = reinterpret_cast<int64_t *>(p2 + L.tile_base);
            ra.blk_tot = reinterpret_cast<unsigned long long *>(p2 + L.blk_tot);
            ra.sup_tot = reinterpret_cast<unsigned long long *>(p2 + L.sup_tot);
        }
        const int warps = kRowsThreads / 32;
        // persistent: one wave of resident CTAs takes every tile (CTAs of a
        // later wave would only find the tile counter exhausted)
        int64_t grid = (nchunks_max + warps - 1) / warps;
        if (grid > (int64_t)sms * kRowsCtas) grid = (int64_t)sms * kRowsCtas;
        const size_t rows_smem = sizeof(RowsSmem) * warps;
        const bool narrow = p->nR <= (int64_t)0xfffffffell;
        if (scratch) {
            if (narrow) {
                LCO_LAUNCH("k_rows", s, launch_dependent(k_rows<uint32_t, true>, (unsigned)grid, kRowsThreads, rows_smem, s, ra));
            } else {
                LCO_LAUNCH("k_rows", s, launch_dependent(k_rows<uint64_t, true>, (unsigned)grid, kRowsThreads, rows_smem, s, ra));
            }
        } else {
            if (narrow) {
                LCO_LAUNCH("k_rows", s, launch_dependent(k_rows<uint32_t, false>, (unsigned)grid, kRowsThreads, rows_smem, s, ra));
            } else {
                LCO_LAUNCH("k_rows", s, launch_dependent(k_rows<uint64_t, false>, (unsigned)grid, kRowsThreads, rows_smem, s, ra));
            }
        }
        LCO_LAUNCH("k_copy_rows", s, launch_dependent(k_copy_rows, (unsigned)(sms * 2), 256, 0, s, ra));
        if (scratch) {
            CompactArgs ca{};
            ca.s_liv = ra.c_liv;
            ca.s_val = ra.c_val;
            ca.tile_cnt = ra.tile_cnt;
            ca.tile_base = ra.tile_base;
            ca.blk_tot = ra.blk_tot;
            ca.sup_tot = ra.sup_tot;
            ca.act_rows = ra.act_rows;
            ca.nact = nact;
            ca.c_liv = c_liv;
            ca.c_val = c_val;
            ca.cap = cap;
            ca.hdr = hdr;
            const int64_t nblk = (nchunks_max + 7) / 8;
            int64_t cgrid = nblk < (int64_t)sms * kCompactCtas ? nblk : (int64_t)sms * kCompactCtas;
            LCO_LAUNCH("k_compact", s,
                       launch_dependent(k_compact, (unsigned)(cgrid > 0 ? cgrid : 1), kCompactThreads, 0, s, ca));
        }
    } else {
        SopArgs sa{};
        sa.l_liv = o.l_liv;
        sa.l_val = o.l_val;
        sa.r_liv = o.r_liv;
        sa.r_val = o.r_val;
        sa.nnz_l = p->nnz_l;
        sa.div_k = make_div((uint64_t)p->k);
        sa.k = p->k;
        sa.div_h = make_div((uint64_t)p->rows_h);
        sa.nR = p->nR;
        sa.mdt = mdt;
        sa.P = P;
        sa.cap = cap;
        sa.out_liv = reinterpret_cast<int64_t *>(sk0);
        sa.out_val = sv0;
        sa.hdr = hdr;
        int64_t grid = (p->nnz_l + 255) / 256;
        if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
        LCO_LAUNCH("k_sop_expand", s, k_sop_expand<<<(unsigned)grid, 256, 0, s>>>(sa));
        // sort products by output LIV with the radix engine (device-side count f)
        RadixJob j{};
        j.relin.nseg = 1;
        j.relin.identity = 1;
        j.key_div = make_div(1);
        j.D = L.sop_D;
        j.P = L.sop_P;
        j.n_host = 0;
        j.n_dev = &hdr->f;
        j.n_cap = capc;
        j.src_liv = reinterpret_cast<int64_t *>(sk0);
        j.src_val = sv0;
        j.dst_liv = reinterpret_cast<int64_t *>(sk1);
        j.dst_val = sv1;
        j.tmp_liv = reinterpret_cast<int64_t *>(sk2);
        j.tmp_val = sv2;
        radix_carve(j, sop_region);
        j.counters = hdr->counters;
        j.status = &hdr->status;
        if (radix_enqueue(j, s) != cudaSuccess) return LCO_ERR_CUDA;
        ReduceArgs ra{};
        ra.key = reinterpret_cast<int64_t *>(sk1);
        ra.val = sv1;
        ra.cap = cap;
        ra.c_liv = c_liv;
        ra.c_val = c_val;
        ra.state = reduce_state;
        ra.ctr = chunk_ctr + 1;
        ra.hdr = hdr;
        const int64_t tiles = (capc + kScanTile - 1) / kScanTile;
        LCO_LAUNCH("k_reduce_by_key", s, k_reduce_by_key<<<(unsigned)(tiles > 0 ? tiles : 1), kCT, 0, s>>>(ra));
    }
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

P2Layout p2_layout(const lco_plan *p, int64_t cap) {
    P2Layout L{};
    L.capc = cap > 0 ? cap : 1;
    L.nchunks_max = (p->nnz_l + 31) / 32 + 2;   // row tiles of the light-row kernel
    size_t off = 0;
    L.chunk_state = off;
    // counters: [0] row tiles, [1] reduce tiles, [2] heavy rows, [4..5] heavy
    // count, [6..7] long copies, [8] row-table tiles, [10..11] active rows
    L.chunk_ctr = (size_t)L.nchunks_max * 8;
    off += align_up((size_t)L.nchunks_max * 8 + 64);
    L.reduce_state = off;
    off += align_up((size_t)((L.capc + kScanTile - 1) / kScanTile + 2) * 8);
    L.table_state = off;
    off += align_up((size_t)((p->nnz_l + kTabTile - 1) / kTabTile + 2) * 8);
    L.blk_tot = off;
    off += align_up((size_t)(L.nchunks_max / kBlkTiles + 2) * 8);
    L.sup_tot = off;
    off += align_up((size_t)(L.nchunks_max / kSupTiles + 2) * 8);
    L.zero_bytes = off;
    L.act_rows = off;
    off += align_up((size_t)(p->nnz_l > 0 ? p->nnz_l : 1) * 8);
    // SOP: products, sorted products and the radix tmp buffer (6 arrays);
    // row kernels: heavy-row scratch and its ping-pong buffer (4 arrays)
    const bool scratch = rows_scratch(p);
    const int narr = (p->acc == 2 || scratch) ? 6 : 4;
    for (int i = 0; i < 6; ++i) {
        L.arr[i] = off;
        if (i < narr) off += align_up((size_t)L.capc * 8);
    }
    L.tile_cnt = off;
    if (scratch) off += align_up((size_t)L.nchunks_max * 8);
    L.tile_base = off;
    if (scratch) off += align_up((size_t)L.nchunks_max * 8);
    L.sop_radix = off;
    radix_digits(p->sop_bits, &L.sop_D, &L.sop_P);
    if (p->acc == 2) off += radix_state_bytes(L.capc, L.sop_D, L.sop_P);
    L.total = off;
    return L;
}

}  // namespace

// The parts of a contraction workspace that must be zero before its first
// use (everything else is written before it is read, or reset by the phases
// themselves): the radix engines' digit-histogram tables.  Lets a caller run
// on recycled memory without clearing the whole workspace.
cudaError_t contract_ws_init(const lco_plan *p, void *ws, int64_t cap, cudaStream_t s) {
    char *w = reinterpret_cast<char *>(ws);
    if (p->need_l || p->need_r) {
        cudaError_t e = cudaMemsetAsync(w + p->off_rp, 0, radix_hist_table_bytes(), s);
        if (e != cudaSuccess) return e;
    }
    if (p->acc == 2 && cap >= 0) {
        const P2Layout L = p2_layout(p, cap);
        return cudaMemsetAsync(w + p->phase1_end + L.sop_radix, 0, radix_hist_table_bytes(), s);
    }
    return cudaSuccess;
}

size_t contract_phase1_bytes(const lco_plan *p) { return p->phase1_end; }

void plan_view(const lco_plan *p, PlanView *v) {
    v->l_is_a = p->l_is_a;
    v->need_l = p->need_l;
    v->need_r = p->need_r;
    v->alg = p->info.alg;
    v->lookup = p->lookup;
    v->mL = p->mL;
    v->k = p->k;
    v->nR = p->nR;
    v->nnz_l = p->nnz_l;
    v->nnz_r = p->nnz_r;
    v->relin_l = p->rp_l.relin;
    v->relin_r = p->rp_r.relin;
}

void plan_row_table(const lco_plan *p, const void *ws, const int64_t **row_start, const int64_t **row_id,
                    const int64_t **row_work) {
    const char *w = reinterpret_cast<const char *>(ws);
    *row_start = reinterpret_cast<const int64_t *>(w + p->off_row_start);
    *row_id = reinterpret_cast<const int64_t *>(w + p->off_row_id);
    *row_work = reinterpret_cast<const int64_t *>(w + p->off_row_work);
}

namespace {

int32_t check_ws(const lco_plan *p, void *ws, size_t ws_bytes, int64_t cap) {
    if (!ws) return LCO_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    size_t need = p->phase1_end + (cap >= 0 ? contract_phase2_bytes(p, cap) : 0);
    if (ws_bytes < need) return LCO_ERR_OOM;
    return LCO_OK;
}

}  // namespace
}  // namespace lco

extern "C" {

int32_t lco_contract_symbolic(const lco_plan *plan, const int64_t *a_liv, const double *a_val,
                              const int64_t *b_liv, const double *b_val, void *ws, size_t ws_bytes,
                              void *stream) {
    NvtxRange nvtx("lco_contract_symbolic");
    if (!plan) return LCO_ERR_INVALID;
    int32_t rc = check_ws(plan, ws, ws_bytes, -1);
    if (rc != LCO_OK) return rc;
    if (!check_ptrs(plan, a_liv, a_val, b_liv, b_val)) return LCO_ERR_INVALID;
    return symbolic_enqueue(plan, a_liv, a_val, b_liv, b_val, reinterpret_cast<char *>(ws),
                            (cudaStream_t)stream);
}

int32_t lco_contract_numeric(const lco_plan *plan, const int64_t *a_liv, const double *a_val,
                             const int64_t *b_liv, const double *b_val, int64_t *c_liv, double *c_val,
                             int64_t cap, void *ws, size_t ws_bytes, void *stream) {
    NvtxRange nvtx("lco_contract_numeric");
    if (!plan || cap < 0) return LCO_ERR_INVALID;
    int32_t rc = check_ws(plan, ws, ws_bytes, cap);
    if (rc != LCO_OK) return rc;
    if (!check_ptrs(plan, a_liv, a_val, b_liv, b_val)) return LCO_ERR_INVALID;
    if (cap > 0 && (!c_liv || !c_val)) return LCO_ERR_INVALID;
    return numeric_enqueue(plan, a_liv, a_val, b_liv, b_val, c_liv, c_val, cap, reinterpret_cast<char *>(ws),
                           (cudaStream_t)stream);
}

int32_t lco_contract(const lco_plan *plan, const int64_t *a_liv, const double *a_val, const int64_t *b_liv,
                     const double *b_val, int64_t *c_liv, double *c_val, int64_t cap, void *ws, size_t ws_bytes,
                     void *stream) {
    int32_t rc = lco_contract_symbolic(plan, a_liv, a_val, b_liv, b_val, ws, ws_bytes, stream);
    if (rc != LCO_OK) return rc;
    return lco_contract_numeric(plan, a_liv, a_val, b_liv, b_val, c_liv, c_val, cap, ws, ws_bytes, stream);
}

int32_t lco_contract_result_get(const void *ws, lco_contract_result *out, void *stream) {
    if (!ws || !out) return LCO_ERR_INVALID;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCO_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(WsHeader), cudaMemcpyDeviceToHost) != cudaSuccess) return LCO_ERR_CUDA;
    out->status = h.status;
    out->alg = h.alg;
    out->nnz_c = h.nnz_c;
    out->f = h.f;
    out->nzr_b = h.nzr_b;
    return LCO_OK;
}

}  // extern "C"
