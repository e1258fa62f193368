// lco_radix.cu -- histogram, offset-scan and scatter kernels of the stable LSD radix engine.
#include <atomic>

#include "lco_radix.cuh"

namespace lco {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUpItems = 8;       // histogram kernels: loads in flight per thread
// direct-form scatter CTAs resident per SM (80 registers each, no spills;
// measured 46.6 us per pass on the 3.4M-entry product permutation vs 48.3
// at four per SM with spills); a build may
// override it (and the bulk-form threshold below) to measure other shapes
#ifndef LCO_SCATTER_CTAS
#define LCO_SCATTER_CTAS 3
#endif
constexpr int kScatterCtas = LCO_SCATTER_CTAS;
constexpr int kScanItems = 16;    // offset scan: counts per thread
constexpr int kScanTile = kRadixThreads * kScanItems;
constexpr int kCtrUpsweep = 8;    // header counter: upsweep blocks finished
constexpr int kCtrScan = 12;      // header counters [12, 12 + kMaxPasses): offset-scan tiles

// Element count; a device-side count never exceeds the capacity the
// buffers were sized for.
__device__ __forceinline__ int64_t job_n(const RadixJob &j) {
    if (!j.n_dev) return j.n_host;
    const int64_t n = *j.n_dev;
    return n < j.n_cap ? n : j.n_cap;
}

// Range r of the G ranges: tiles [r T / G, (r + 1) T / G) of the T tiles
// of n elements, so that ranges differ by at most one tile; the last tile
// of the input is ragged.
__device__ __forceinline__ void range_of(const RadixJob &j, int64_t n, int64_t r, int64_t &lo, int64_t &hi) {
    const int64_t T = (n + kRadixTile - 1) / kRadixTile;
    lo = (r * T / j.G) * kRadixTile;
    hi = ((r + 1) * T / j.G) * kRadixTile;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
}

// Which buffers a pass reads and writes.  Active passes ping-pong between
// dst and tmp so that the last active pass writes dst; the first active pass
// reads the source (and re-linearises it).  With no active pass, the last
// pass copies the re-linearised source to dst.
struct PassIO {
    const int64_t *sl;
    const double *sv;
    int64_t *dl;
    double *dv;
    bool run, first, copy;
};

__device__ __forceinline__ PassIO pass_io(const RadixJob &j, int pass) {
    PassIO io{};
    const int Q = j.active[16];
    const bool act = j.active[pass] != 0;
    io.copy = (Q == 0) && (pass == j.P - 1);
    io.run = act || io.copy;
    int q = 0;
    for (int p = 0; p < pass; ++p) q += j.active[p] != 0;
    io.first = io.copy || q == 0;
    const bool prev_in_dst = q > 0 && ((Q - 1 - (q - 1)) & 1) == 0;
    io.sl = io.first ? j.src_liv : (prev_in_dst ? j.dst_liv : j.tmp_liv);
    io.sv = io.first ? j.src_val : (prev_in_dst ? j.dst_val : j.tmp_val);
    const bool to_dst = io.copy || ((Q - 1 - q) & 1) == 0;
    io.dl = to_dst ? j.dst_liv : j.tmp_liv;
    io.dv = to_dst ? j.dst_val : j.tmp_val;
    return io;
}

// Look-back words of one offset scan: its tiles over the NB x G table.
__host__ __device__ __forceinline__ int64_t scan_tiles(int NB, int G) {
    return ((int64_t)NB * G + kScanTile - 1) / kScanTile;
}

// ---------------------------------------------------------------------------
// One read of the source keys: every pass's digit histogram per range
// (counts_src) and, per range and pass, the one digit the range holds (-1
// when it holds several, -2 when it is empty).  The last block to finish
// marks the passes whose digit is the same over all the data (nothing to
// do) and resets its counter.  Block 0 first clears the offset scans'
// look-back words and tile counters (the scans run after this launch).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const __grid_constant__ RadixJob j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ int s_last;
    __shared__ int s_nz[kMaxPasses], s_dig[kMaxPasses];
    const int NB = 1 << j.D;
    const int nh = j.P * NB;
    if (blockIdx.x == 0) {
        const int64_t nst = (int64_t)kMaxPasses * scan_tiles(NB, j.G);
        for (int64_t i = threadIdx.x; i < nst; i += blockDim.x) j.scan_state[i] = 0;
        if (threadIdx.x < kMaxPasses) j.counters[kCtrScan + threadIdx.x] = 0;
    }
    for (int i = threadIdx.x; i < nh; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x < kMaxPasses) {
        s_nz[threadIdx.x] = 0;
        s_dig[threadIdx.x] = 0;
    }
    __syncthreads();

    const int64_t n = job_n(j);
    int64_t lo, hi;
    range_of(j, n, blockIdx.x, lo, hi);
    const uint32_t mask = (uint32_t)NB - 1;
    // kUpItems independent loads in flight per thread
    for (int64_t e0 = lo; e0 < hi; e0 += (int64_t)kUpItems * kRadixThreads) {
        int64_t v[kUpItems];
#pragma unroll
        for (int i = 0; i < kUpItems; ++i) {
            const int64_t e = e0 + i * kRadixThreads + threadIdx.x;
            v[i] = e < hi ? j.src_liv[e] : -1;
        }
#pragma unroll
        for (int i = 0; i < kUpItems; ++i) {
            if (v[i] >= 0) {
                const uint64_t key = divu(j.key_div, (uint64_t)relin(j.relin, v[i]));
                for (int p = 0; p < j.P; ++p)
                    atomicAdd(&s_hist[p * NB + (uint32_t)((key >> (p * j.D)) & mask)], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
        const int p = i / NB, d = i - p * NB;
        const uint32_t c = s_hist[i];
        j.counts_src[((int64_t)p * NB + d) * j.G + blockIdx.x] = c;
        if (c) {
            atomicAdd(&s_nz[p], 1);
            s_dig[p] = d;   // read only when exactly one digit is present
        }
    }
    __syncthreads();
    if (threadIdx.x < j.P) {
        const int p = threadIdx.x;
        j.cdig[(int64_t)p * j.G + blockIdx.x] = lo >= hi ? -2 : (s_nz[p] == 1 ? s_dig[p] : -1);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&j.counters[kCtrUpsweep], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: a pass is skipped when every non-empty range holds the same
    // single digit
    __shared__ int s_several[kMaxPasses], s_lo[kMaxPasses], s_hi[kMaxPasses];
    if (threadIdx.x < kMaxPasses) {
        s_several[threadIdx.x] = 0;
        s_lo[threadIdx.x] = 1 << 30;
        s_hi[threadIdx.x] = -1;
    }
    __syncthreads();
    for (int p = 0; p < j.P; ++p) {
        int several = 0, dlo = 1 << 30, dhi = -1;
        for (int r = threadIdx.x; r < j.G; r += blockDim.x) {
            const int c = *reinterpret_cast<volatile const int32_t *>(j.cdig + (int64_t)p * j.G + r);
            if (c == -1) several = 1;
            if (c >= 0) {
                dlo = c < dlo ? c : dlo;
                dhi = c > dhi ? c : dhi;
            }
        }
        if (several) s_several[p] = 1;
        if (dhi >= 0) {
            atomicMin(&s_lo[p], dlo);
            atomicMax(&s_hi[p], dhi);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nactive = 0;
        for (int p = 0; p < j.P; ++p) {
            const int act = (n > 0) && (s_several[p] || s_lo[p] != s_hi[p]);
            j.active[p] = act;
            nactive += act;
        }
        j.active[16] = nactive;
        j.counters[kCtrUpsweep] = 0;
    }
}

// Per-range digit histogram of the buffer a later pass reads.
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const __grid_constant__ RadixJob j, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    const PassIO io = pass_io(j, pass);
    if (!io.run || io.first) return;
    const int NB = 1 << j.D;
    for (int i = threadIdx.x; i < NB; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const int64_t n = job_n(j);
    int64_t lo, hi;
    range_of(j, n, blockIdx.x, lo, hi);
    const uint32_t mask = (uint32_t)NB - 1;
    const int shift = pass * j.D;
    for (int64_t e0 = lo; e0 < hi; e0 += (int64_t)kUpItems * kRadixThreads) {
        int64_t v[kUpItems];
#pragma unroll
        for (int i = 0; i < kUpItems; ++i) {
            const int64_t e = e0 + i * kRadixThreads + threadIdx.x;
            v[i] = e < hi ? io.sl[e] : -1;
        }
#pragma unroll
        for (int i = 0; i < kUpItems; ++i)
            if (v[i] >= 0) atomicAdd(&s_hist[(uint32_t)(divu(j.key_div, (uint64_t)v[i]) >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < NB; d += blockDim.x) j.counts_hist[(int64_t)d * j.G + blockIdx.x] = s_hist[d];
}

// roffs[d][r] = the number of elements with a smaller digit, plus those with
// digit d in ranges before r: the exclusive prefix sum of the digit-major
// count table.  One single-pass scan (tiles taken in launch order, each
// summing the tiles before it by decoupled look-back).
__global__ void __launch_bounds__(kRadixThreads) k_radix_offsets(const __grid_constant__ RadixJob j, int pass) {
    const PassIO io = pass_io(j, pass);
    if (!io.run || io.copy) return;
    __shared__ uint64_t s_wsum[kRadixWarps + 1];
    __shared__ uint32_t s_tile;
    const int NB = 1 << j.D;
    const int64_t M = (int64_t)NB * j.G;
    const uint32_t *cnt = io.first ? j.counts_src + (int64_t)pass * M : j.counts_hist;
    uint64_t *state = j.scan_state + (int64_t)pass * scan_tiles(NB, j.G);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&j.counters[kCtrScan + pass], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + (int64_t)tid * kScanItems;
    uint32_t c[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) c[i] = base + i < M ? cnt[base + i] : 0u;
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) sum += c[i];
    uint64_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint64_t wex = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
        const uint64_t v = s_wsum[w];
        wex += w < warp ? v : 0;
        tot += v;
    }
    if (warp == 0) {
        if (lane == 0) lb_store(state + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | tot);
        uint64_t ex = 0;
        if (tile > 0) ex = lookback_warp(state, tile, j.status);
        if (lane == 0) {
            if (tile > 0) lb_store(state + tile, kFlagIncl | (ex + tot));
            s_wsum[kRadixWarps] = ex;
        }
    }
    __syncthreads();
    uint64_t run = s_wsum[kRadixWarps] + wex + x - sum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < M) j.roffs[base + i] = run;
        run += c[i];
    }
}

// Shared memory of a scatter CTA: the staging buffer (key, value pairs), the
// per-tile global base and running offset of every digit, the per-warp digit
// counts (16 bits, warp-major: [warp][digit]) and the digit of every staged
// element (used when a digit is not a plain shift of the key), rounded up to
// 128 bytes (the bulk form's input buffers follow: copy destinations must be
// aligned).
__host__ __device__ constexpr size_t scatter_smem_bytes_base(int D) {
    return ((size_t)kRadixTile * 18 + ((size_t)1 << D) * 16 + ((size_t)1 << D) * 2 * kRadixWarps + 64 + 127) &
           ~(size_t)127;
}

// Digit of a key in a pass: a shift when the key divisor is a power of two
// (kShift: the divisor's shift plus the pass's digit offset, precomputed),
// else the invariant division first.
template <bool kShift>
__device__ __forceinline__ uint32_t key_digit(const RadixJob &j, int64_t key, int shift, uint32_t mask) {
    if constexpr (kShift) return (uint32_t)((uint64_t)key >> shift) & mask;
    else return (uint32_t)(divu(j.key_div, (uint64_t)key) >> shift) & mask;
}

// ---------------------------------------------------------------------------
// One stable scatter pass: CTA r walks range r tile by tile (kRadixTile
// elements, warp w holding elements w*256 + 32 i + lane of the tile), placing
// each tile from running per-digit offsets.  Per tile:
//   1. each warp ranks its items in element order: lanes with equal digits
//      find each other with one match instruction, and the lowest of them
//      reads and advances the warp's count of that digit; an item's rank is
//      the count before it plus its peers in lower lanes;
//   2. each thread turns the counts of its digits into per-warp slots (the
//      tile-local start of that warp's run of the digit), the tile's global
//      base of the digit and the running offset for the next tile -- one
//      block scan over the digit totals;
//   3. every item is staged, as one 16-byte (key, value) store, at slot +
//      rank: the tile sorted by digit, stably;
//   4. the staged tile is written out in order: each digit's run is a
//      contiguous stretch of the output.
// The count table is warp-major (a warp's counts are one row, so the random
// digits of a warp spread over all shared-memory banks) and each thread of
// step 2 owns pairs of digits (one 32-bit word per warp row).
// Two forms:
//   kBulk: the next input tile comes in by bulk copy while the current one is
//     processed (double-buffered input, two CTAs per SM) -- ranges of many
//     tiles;
//   otherwise: tiles are loaded directly and kScatterCtas CTAs share an SM, filling
//     each other's barrier gaps -- ranges of few tiles.
// ---------------------------------------------------------------------------
template <bool kBulk, bool kShift>
__global__ void __launch_bounds__(kRadixThreads, kBulk ? 2 : kScatterCtas)
    k_radix_scatter(const __grid_constant__ RadixJob j, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PassIO io = pass_io(j, pass);
    if (!io.run) return;
    const int D = j.D;
    const int NB = 1 << D;
    double2 *s_kv = reinterpret_cast<double2 *>(smem_raw);                                 // [kRadixTile]
    int64_t *s_run = reinterpret_cast<int64_t *>(s_kv + kRadixTile);
    int64_t *s_gb = s_run + NB;
    uint16_t *s_cnt = reinterpret_cast<uint16_t *>(s_gb + NB);                            // [8][NB]
    uint16_t *s_dig = s_cnt + (size_t)NB * kRadixWarps;                                    // [kRadixTile]
    uint32_t *s_wtot = reinterpret_cast<uint32_t *>(s_dig + kRadixTile);                  // [8]
    // bulk form only: the input buffers and their barrier, after the tables
    int64_t *in_key = reinterpret_cast<int64_t *>(smem_raw + scatter_smem_bytes_base(D));
    double *in_val = reinterpret_cast<double *>(in_key + kRadixTile);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(in_val + kRadixTile);

    const int64_t n = job_n(j);
    int64_t lo, hi;
    range_of(j, n, blockIdx.x, lo, hi);
    if (io.copy) {
        for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            io.dl[e] = relin(j.relin, io.sl[e]);
            io.dv[e] = io.sv[e];
        }
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t mask = (uint32_t)NB - 1;
    const int shift = kShift ? (int)j.key_div.shift + pass * D : pass * D;
    // count-table words owned by this thread in step 2: [w0, w0 + wpt) of
    // each warp row (word k holds digits 2k and 2k + 1)
    const int nwords = NB >= 2 ? NB / 2 : 1;
    const int wpt = nwords > kRadixThreads ? nwords / kRadixThreads : 1;
    const int w0 = tid * wpt;
    uint32_t *cnt_words = reinterpret_cast<uint32_t *>(s_cnt);
    for (int d = tid; d < NB; d += kRadixThreads) s_run[d] = (int64_t)j.roffs[(int64_t)d * j.G + blockIdx.x];
    for (int i = tid; i < NB * kRadixWarps / 2; i += kRadixThreads) cnt_words[i] = 0;
    const unsigned lt = lanemask_lt();
    uint16_t *wcnt = s_cnt + (size_t)warp * NB;
    // bulk form: the next tile is copied in while the current one is
    // processed, when both input arrays are 16-byte aligned (tile starts are
    // even element offsets); an odd last element is read directly
    const bool bulk = kBulk && ((reinterpret_cast<uintptr_t>(io.sl) | reinterpret_cast<uintptr_t>(io.sv)) & 15) == 0;
    uint32_t parity = 0;
    auto issue = [&](int64_t base) {
        const int64_t m = (hi - base < (int64_t)kRadixTile ? hi - base : (int64_t)kRadixTile) & ~(int64_t)1;
        if (m <= 0) return;
        const uint32_t bytes = (uint32_t)(m * 8);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(s_bar, 2 * bytes);
        bulk_copy_g2s(in_key, io.sl + base, bytes, s_bar);
        bulk_copy_g2s(in_val, io.sv + base, bytes, s_bar);
    };
    if (bulk && tid == 0) {
        mbar_init(s_bar, 1);
        if (lo < hi) issue(lo);
    }
    __syncthreads();

    for (int64_t tile_base = lo; tile_base < hi; tile_base += kRadixTile) {
        const int tile_n = (int)((hi - tile_base) < (int64_t)kRadixTile ? (hi - tile_base) : (int64_t)kRadixTile);
        // this warp's valid items: i * 32 + lane < wn
        const int wn = tile_n - warp * (32 * kRadixItems);
        const int bulk_n = bulk ? (tile_n & ~1) : 0;     // elements that arrived by bulk copy
        if (bulk && bulk_n > 0) {
            const bool ok = mbar_wait_bounded(s_bar, parity);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_error(j.status, LCO_ERR_TIMEOUT);
                return;
            }
        }
        // ---- 1. load, digits, stable ranks within the warp ----
        int64_t keys[kRadixItems];
        double vals[kRadixItems];
        uint32_t dr[kRadixItems];    // digit | rank within the warp's run << 16
        const int wofs = warp * (32 * kRadixItems) + lane;    // tile-local index of item 0
        const int64_t *kp = io.sl + tile_base + wofs;
        const double *vp = io.sv + tile_base + wofs;
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const int li = wofs + i * 32;
            keys[i] = 0;
            vals[i] = 0.0;
            if (li < bulk_n) {
                keys[i] = in_key[li];
                vals[i] = in_val[li];
            } else if (i * 32 + lane < wn) {
                keys[i] = __ldg(kp + i * 32);
                vals[i] = __ldg(vp + i * 32);
            }
        }
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const bool valid = i * 32 + lane < wn;
            uint32_t d = 0;
            if (valid) {
                if (io.first) keys[i] = relin(j.relin, keys[i]);
                d = key_digit<kShift>(j, keys[i], shift, mask);
            }
            // lanes holding the same digit (invalid lanes carry labels no
            // valid lane has: digits are < 2^11).  One match instruction;
            // measured against one ballot per digit bit, it is faster on
            // keys whose warps hold few distinct digits (the 3.4M-entry
            // product of the 64^3 Laplacian and a derivative: 48 vs 54 us
            // per pass) and slower on uniform random keys (69 vs 64).
            const unsigned peers = __match_any_sync(kFull, valid ? d : 0x10000u | (uint32_t)lane);
            const int leader = __ffs(peers) - 1;
            uint32_t c = 0;
            if (valid && lane == leader) {
                c = wcnt[d];
                wcnt[d] = (uint16_t)(c + (uint32_t)__popc(peers));
            }
            c = __shfl_sync(kFull, c, leader);
            dr[i] = d | ((c + (uint32_t)__popc(peers & lt)) << 16);
            __syncwarp();
        }
        __syncthreads();
        // the input buffer is free: fetch the next tile behind this one's work
        if (bulk && tid == 0 && tile_base + kRadixTile < hi) issue(tile_base + kRadixTile);
        // ---- 2. per-warp slots, the tile's global bases, running offsets ----
        {
            uint32_t tsum = 0;
            for (int q = 0; q < wpt; ++q) {
                const int k = w0 + q;
                if (k < nwords) {
                    uint32_t s2 = 0;
#pragma unroll
                    for (int w = 0; w < kRadixWarps; ++w) s2 += cnt_words[w * nwords + k];
                    tsum += (s2 & 0xffffu) + (s2 >> 16);    // a half never carries (< 2^12 per word)
                }
            }
            // exclusive scan of the thread sums (digits are owned in order)
            uint32_t x = tsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += u;
            }
            if (lane == 31) s_wtot[warp] = x;
            __syncthreads();
            uint32_t run = x - tsum;
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) run += w < warp ? s_wtot[w] : 0u;
            for (int q = 0; q < wpt; ++q) {
                const int k = w0 + q;
                if (k < nwords) {
                    // low halves (digit 2k) become slots in one sweep down the
                    // warp rows, high halves (digit 2k + 1) in a second
                    const uint32_t ts_lo = run;
#pragma unroll
                    for (int w = 0; w < kRadixWarps; ++w) {
                        const uint32_t v = cnt_words[w * nwords + k];
                        cnt_words[w * nwords + k] = (v & 0xffff0000u) | run;
                        run += v & 0xffffu;
                    }
                    const uint32_t ts_hi = run;
#pragma unroll
                    for (int w = 0; w < kRadixWarps; ++w) {
                        const uint32_t v = cnt_words[w * nwords + k];
                        cnt_words[w * nwords + k] = (v & 0xffffu) | (run << 16);
                        run += v >> 16;
                    }
                    const int dlo = 2 * k;
                    if (dlo < NB) {
                        const int64_t r0 = s_run[dlo];
                        s_gb[dlo] = r0 - (int64_t)ts_lo;
                        s_run[dlo] = r0 + (int64_t)(ts_hi - ts_lo);
                    }
                    if (dlo + 1 < NB) {
                        const int64_t r1 = s_run[dlo + 1];
                        s_gb[dlo + 1] = r1 - (int64_t)ts_hi;
                        s_run[dlo + 1] = r1 + (int64_t)(run - ts_hi);
                    }
                }
            }
        }
        __syncthreads();
        // ---- 3. staging at the sorted tile-local position ----
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            if (i * 32 + lane < wn) {
                const uint32_t d = dr[i] & 0xffffu;
                const uint32_t pos = (uint32_t)wcnt[d] + (dr[i] >> 16);
                s_kv[pos] = make_double2(__longlong_as_double(keys[i]), vals[i]);
                if (!kShift) s_dig[pos] = (uint16_t)d;
            }
        }
        __syncthreads();
        // ---- 4. write-out in staged order; reset this thread's count words ----
#pragma unroll
        for (int q = 0; q < kRadixItems; ++q) {
            const int i = tid + q * kRadixThreads;
            if (i < tile_n) {
                const double2 kv = s_kv[i];
                const int64_t k = __double_as_longlong(kv.x);
                const uint32_t d = kShift ? key_digit<true>(j, k, shift, mask) : (uint32_t)s_dig[i];
                const int64_t g = s_gb[d] + i;
                io.dl[g] = k;
                io.dv[g] = kv.y;
            }
        }
        for (int q = 0; q < wpt; ++q) {
            const int k = w0 + q;
            if (k < nwords) {
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) cnt_words[w * nwords + k] = 0;
            }
        }
        __syncthreads();
    }
}

size_t scatter_smem_bytes(int D, bool bulk) {
    return scatter_smem_bytes_base(D) + (bulk ? (size_t)kRadixTile * 16 + 16 : 0);
}

size_t upsweep_smem_bytes(int D, int P) { return (size_t)P * ((size_t)1 << D) * 4; }

}  // namespace

int radix_sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Up to kBulkMinTiles tiles per CTA of a full direct-form wave, the direct
// scatter runs; beyond, the bulk-copy form (two CTAs per SM, at least eight
// tiles per range).
#ifndef LCO_BULK_MIN_TILES
#define LCO_BULK_MIN_TILES 4
#endif
constexpr int64_t kBulkMinTiles = LCO_BULK_MIN_TILES;

bool radix_bulk(int64_t n_cap) {
    const int64_t tiles = (n_cap + kRadixTile - 1) / kRadixTile;
    return tiles > kBulkMinTiles * kScatterCtas * (int64_t)radix_sm_count();
}

// One range per scatter CTA of a full wave (or one per tile, when there are
// fewer tiles than that).
int radix_ranges(int64_t n_cap) {
    const int64_t tiles = (n_cap + kRadixTile - 1) / kRadixTile;
    const int64_t gmax = (radix_bulk(n_cap) ? 2 : kScatterCtas) * (int64_t)radix_sm_count();
    int64_t g = tiles < gmax ? tiles : gmax;
    if (g < 1) g = 1;
    return (int)g;
}

size_t radix_state_bytes(int64_t n_cap, int D, int P) {
    const size_t NB = (size_t)1 << D;
    const size_t G = (size_t)radix_ranges(n_cap);
    size_t b = 0;
    b += align_up(32 * 4);                                                  // active
    b += align_up((size_t)kMaxPasses * G * 4);                              // cdig
    b += align_up((size_t)kMaxPasses * scan_tiles((int)NB, (int)G) * 8);   // scan_state
    b += align_up((size_t)P * G * NB * 4);                                  // counts_src
    b += align_up(G * NB * 4);                                              // counts_hist
    b += align_up(G * NB * 8);                                              // roffs
    return b;
}

// Nothing in the engine's region needs to be zero before a call (the
// upsweep clears what the scans wait on); callers that clear this many
// leading bytes of it only reset the pass flags, which every call rewrites.
size_t radix_hist_table_bytes() { return align_up(32 * 4); }

void radix_carve(RadixJob &job, char *region) {
    const size_t NB = (size_t)1 << job.D;
    job.G = radix_ranges(job.n_cap);
    const size_t G = (size_t)job.G;
    char *p = region;
    job.active = reinterpret_cast<int32_t *>(p); p += align_up(32 * 4);
    job.cdig = reinterpret_cast<int32_t *>(p); p += align_up((size_t)kMaxPasses * G * 4);
    job.scan_state = reinterpret_cast<uint64_t *>(p);
    p += align_up((size_t)kMaxPasses * scan_tiles((int)NB, (int)G) * 8);
    job.counts_src = reinterpret_cast<uint32_t *>(p); p += align_up((size_t)job.P * G * NB * 4);
    job.counts_hist = reinterpret_cast<uint32_t *>(p); p += align_up(G * NB * 4);
    job.roffs = reinterpret_cast<uint64_t *>(p);
}

namespace {

template <bool kBulk, bool kShift>
void launch_scatter(const RadixJob &job, int p, cudaStream_t stream) {
    LCO_LAUNCH("k_radix_scatter", stream,
               (k_radix_scatter<kBulk, kShift><<<(unsigned)job.G, kRadixThreads, scatter_smem_bytes(job.D, kBulk),
                                                  stream>>>(job, p)));
}

}  // namespace

cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream) {
    // function attributes are per device: set them once on each
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        const int bulk_bytes = (int)scatter_smem_bytes(kMaxDigitBits, true);
        const int direct_bytes = (int)scatter_smem_bytes(kMaxDigitBits, false);
        cudaFuncSetAttribute(k_radix_scatter<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bulk_bytes);
        cudaFuncSetAttribute(k_radix_scatter<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bulk_bytes);
        cudaFuncSetAttribute(k_radix_scatter<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_bytes);
        cudaFuncSetAttribute(k_radix_scatter<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_bytes);
        cudaFuncSetAttribute(k_radix_upsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upsweep_smem_bytes(kMaxDigitBits, kMaxPasses));
        attr_done.fetch_or(bit);
    }
    if (job.n_cap <= 0) return cudaSuccess;
    const unsigned G = (unsigned)job.G;
    const int NB = 1 << job.D;
    const unsigned scan_grid = (unsigned)scan_tiles(NB, job.G);
    LCO_LAUNCH("k_radix_upsweep", stream,
               k_radix_upsweep<<<G, kRadixThreads, upsweep_smem_bytes(job.D, job.P), stream>>>(job));
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const bool bulk = radix_bulk(job.n_cap);
    const bool shift = job.key_div.pow2 != 0;
    for (int p = 0; p < job.P; ++p) {
        if (p > 0) {
            LCO_LAUNCH("k_radix_hist", stream,
                       k_radix_hist<<<G, kRadixThreads, (size_t)NB * 4, stream>>>(job, p));
        }
        LCO_LAUNCH("k_radix_offsets", stream, k_radix_offsets<<<scan_grid, kRadixThreads, 0, stream>>>(job, p));
        if (bulk) {
            if (shift) launch_scatter<true, true>(job, p, stream);
            else launch_scatter<true, false>(job, p, stream);
        } else {
            if (shift) launch_scatter<false, true>(job, p, stream);
            else launch_scatter<false, false>(job, p, stream);
        }
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace lco
