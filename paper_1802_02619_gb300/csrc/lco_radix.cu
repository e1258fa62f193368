// lco_radix.cu -- counting and single-sweep scatter kernels of the stable LSD radix engine.
#include <atomic>

#include "lco_radix.cuh"

namespace lco {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUpItems = 8;       // counting kernel: consecutive keys per thread and round
// scatter CTAs resident per SM; a build may override it to measure others
#ifndef LCO_SCATTER_CTAS
#define LCO_SCATTER_CTAS 3
#endif
constexpr int kScatterCtas = LCO_SCATTER_CTAS;
#ifndef LCO_UPSWEEP_CTAS
#define LCO_UPSWEEP_CTAS 4
#endif
constexpr int kUpsweepCtasPerSm = LCO_UPSWEEP_CTAS;   // counting CTAs per SM; a build may override it
constexpr int kCtrUpsweep = 8;    // header counter: counting blocks finished
constexpr int kCtrTile = 12;      // header counters [12, 12 + kMaxPasses): tiles taken by the q-th run pass
// Two-pass keys whose high-digit buckets all fit one CTA's shared memory are
// sorted high digit first: one global scatter by the high digit, then each
// bucket sorted by the low digit inside one CTA (contiguous read and write).
// The upsweep decides it on the device from the digit counts.
#ifndef LCO_RADIX_LOCAL
#define LCO_RADIX_LOCAL 1
#endif
constexpr int kLocalThreads = 512;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kLocalCap = 8192;                            // elements of one bucket
constexpr int kLocalItems = kLocalCap / kLocalThreads;     // per thread
constexpr int kLocalMaxBits = 9;                           // digit widths the local sort takes
// pass flags: [p] pass p runs, [16] passes that run, [17] high digit first,
// [18] its high pass, [19] its low pass
constexpr int kFlagQ = 16, kFlagMsd = 17, kFlagHi = 18, kFlagLo = 19;

// Element count; a device-side count never exceeds the capacity the
// buffers were sized for.
__device__ __forceinline__ int64_t job_n(const RadixJob &j) {
    if (!j.n_dev) return j.n_host;
    const int64_t n = *j.n_dev;
    return n < j.n_cap ? n : j.n_cap;
}

__host__ __device__ __forceinline__ int64_t tiles_of(int64_t n) { return (n + kRadixTile - 1) / kRadixTile; }

// Range r of the G counting ranges: tiles [r T / G, (r + 1) T / G) of the
// T tiles of n elements, so that ranges differ by at most one tile.
__device__ __forceinline__ void range_of(const RadixJob &j, int64_t n, int64_t r, int64_t &lo, int64_t &hi) {
    const int64_t T = tiles_of(n);
    lo = (r * T / j.G) * kRadixTile;
    hi = ((r + 1) * T / j.G) * kRadixTile;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
}

// Which buffers a pass reads and writes.  Passes that run ping-pong between
// dst and tmp so that the last one writes dst; the first one reads the
// source (and re-linearises it).  With no pass to run, the last pass copies
// the re-linearised source to dst.  q is the pass's rank among those that
// run (it selects the look-back region and the tile counter).
struct PassIO {
    const int64_t *sl;
    const double *sv;
    int64_t *dl;
    double *dv;
    int q;
    bool run, first, copy;
};

__device__ __forceinline__ PassIO pass_io(const RadixJob &j, int pass) {
    PassIO io{};
    if (j.active[kFlagMsd]) {
        // high digit first: only the high pass scatters, source -> tmp
        io.run = pass == j.active[kFlagHi];
        io.first = true;
        io.copy = false;
        io.q = 0;
        io.sl = j.src_liv;
        io.sv = j.src_val;
        io.dl = j.tmp_liv;
        io.dv = j.tmp_val;
        return io;
    }
    const int Q = j.active[kFlagQ];
    const bool act = j.active[pass] != 0;
    io.copy = (Q == 0) && (pass == j.P - 1);
    io.run = act || io.copy;
    int q = 0;
    for (int p = 0; p < pass; ++p) q += j.active[p] != 0;
    io.q = q;
    io.first = io.copy || q == 0;
    const bool prev_in_dst = q > 0 && ((Q - 1 - (q - 1)) & 1) == 0;
    io.sl = io.first ? j.src_liv : (prev_in_dst ? j.dst_liv : j.tmp_liv);
    io.sv = io.first ? j.src_val : (prev_in_dst ? j.dst_val : j.tmp_val);
    const bool to_dst = io.copy || ((Q - 1 - q) & 1) == 0;
    io.dl = to_dst ? j.dst_liv : j.tmp_liv;
    io.dv = to_dst ? j.dst_val : j.tmp_val;
    return io;
}

// Look-back words, [flag:2 | value]: flag 0 = not yet published, 1 = the
// tile's own count of the digit, 2 = the count over the tile and every tile
// before it.  32-bit words when fewer than 2^30 elements can occur.  A
// thread owns digits 2k and 2k + 1, whose words are adjacent: they are
// published and read as one pair (each word is still written whole, so a
// pair read may see one word newer than the other; each is judged by its
// own flag).
template <typename W>
struct LbWord;

template <>
struct LbWord<uint32_t> {
    static constexpr uint32_t kAgg = 1u << 30;
    static constexpr uint32_t kIncl = 2u << 30;
    static constexpr uint32_t kMask = (1u << 30) - 1;
    __device__ static __forceinline__ uint32_t flag(uint32_t v) { return v >> 30; }
    __device__ static __forceinline__ void store(uint32_t *p, uint32_t v) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
    }
    __device__ static __forceinline__ void store2(uint32_t *p, uint32_t a, uint32_t b) {
        asm volatile("st.relaxed.gpu.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(a), "r"(b) : "memory");
    }
    __device__ static __forceinline__ void load2(const uint32_t *p, uint32_t &a, uint32_t &b) {
        asm volatile("ld.relaxed.gpu.global.v2.u32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "l"(p) : "memory");
    }
#ifndef LCO_LB_BATCH
#define LCO_LB_BATCH 4
#endif
    // predecessor pairs fetched per look-back round (measured on the 3.4M-entry
    // product: 4 and 6 alike, 8 slower, 16 much slower); a build may override it
    static constexpr int kBatch = LCO_LB_BATCH;
};

template <>
struct LbWord<uint64_t> {
    static constexpr uint64_t kAgg = 1ull << 62;
    static constexpr uint64_t kIncl = 2ull << 62;
    static constexpr uint64_t kMask = (1ull << 62) - 1;
    __device__ static __forceinline__ uint64_t flag(uint64_t v) { return v >> 62; }
    __device__ static __forceinline__ void store2(uint64_t *p, uint64_t a, uint64_t b) {
        asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
    }
    __device__ static __forceinline__ void load2(const uint64_t *p, uint64_t &a, uint64_t &b) {
        asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
    }
    static constexpr int kBatch = 4;
};

// ---------------------------------------------------------------------------
// One read of the source keys: every pass's digit counts over the whole
// input (per-CTA counts in shared memory, added into the global table).
// The last block to finish turns each pass's counts into the start of every
// digit's run in that pass's output (an exclusive scan over the digits) and
// marks the passes whose digit is the same over all the data (nothing to
// do).  Block 0 resets the scatter passes' tile counters; all blocks clear
// the look-back words the first scatter pass to run will use.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const __grid_constant__ RadixJob j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ int s_last;
    __shared__ unsigned long long s_part[kRadixWarps + 1];
    const int NB = 1 << j.D;
    const int nh = j.P * NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid < kMaxPasses) j.counters[kCtrTile + tid] = 0;
    for (int i = tid; i < nh; i += blockDim.x) s_hist[i] = 0;
    const int64_t n = job_n(j);
    {
        const int64_t words = tiles_of(n) * NB * (j.wide_lb ? 2 : 1);   // 32-bit words of region 0 in use
        uint32_t *z = reinterpret_cast<uint32_t *>(j.lb);
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < words; i += (int64_t)gridDim.x * blockDim.x)
            z[i] = 0;
    }
    __syncthreads();

    int64_t lo, hi;
    range_of(j, n, blockIdx.x, lo, hi);
    const uint32_t mask = (uint32_t)NB - 1;
    // Each thread counts kUpItems consecutive keys per round and adds a run
    // of equal digits with one shared atomic: keys sorted in their old order
    // repeat digits in runs, and lanes at different places of such runs
    // rarely hit the same counter at once (with one key per lane, a warp of
    // neighbouring keys would serialise on a handful of counters).
    // the next round's keys are loaded before this round's are counted
    constexpr int64_t kStride = (int64_t)kUpItems * kRadixThreads;
    int64_t e0 = lo + (int64_t)tid * kUpItems;
    int64_t nxt[kUpItems];
#pragma unroll
    for (int i = 0; i < kUpItems; ++i) nxt[i] = e0 + i < hi ? __ldg(j.src_liv + e0 + i) : 0;
    for (; e0 < hi; e0 += kStride) {
        uint64_t key[kUpItems];
        const int m = hi - e0 < (int64_t)kUpItems ? (int)(hi - e0) : kUpItems;
#pragma unroll
        for (int i = 0; i < kUpItems; ++i) key[i] = (uint64_t)nxt[i];
        const int64_t e1 = e0 + kStride;
#pragma unroll
        for (int i = 0; i < kUpItems; ++i) nxt[i] = e1 + i < hi ? __ldg(j.src_liv + e1 + i) : 0;
#pragma unroll
        for (int i = 0; i < kUpItems; ++i)
            if (i < m) key[i] = divu(j.key_div, (uint64_t)relin(j.relin, (int64_t)key[i]));
        for (int p = 0; p < j.P; ++p) {
            uint32_t *h = s_hist + p * NB;
            const int sh = p * j.D;
            uint32_t cur = (uint32_t)(key[0] >> sh) & mask, cnt = 0;
#pragma unroll
            for (int i = 0; i < kUpItems; ++i) {
                if (i < m) {
                    const uint32_t d = (uint32_t)(key[i] >> sh) & mask;
                    if (d != cur) {
                        atomicAdd(&h[cur], cnt);
                        cur = d;
                        cnt = 0;
                    }
                    ++cnt;
                }
            }
            if (cnt) atomicAdd(&h[cur], cnt);
        }
    }
    __syncthreads();
    for (int i = tid; i < nh; i += blockDim.x) {
        const uint32_t c = s_hist[i];
        if (c) atomicAdd(&j.hist[i], (unsigned long long)c);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&j.counters[kCtrUpsweep], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: per pass, thread t owns digits [t * per, (t + 1) * per)
    const int per = NB > kRadixThreads ? NB / kRadixThreads : 1;
    const int d0 = tid * per;
    int nactive = 0, p_hi = -1, p_lo = -1, hi_big = 0;
    for (int p = 0; p < j.P; ++p) {
        volatile const unsigned long long *h = j.hist + (int64_t)p * NB;
        unsigned long long c[8];
        unsigned long long sum = 0;
        int nz = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = (i < per && d0 + i < NB) ? h[d0 + i] : 0ull;
            sum += c[i];
            nz += c[i] != 0;
        }
        unsigned long long x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) s_part[warp] = x;
        // a pass runs when more than one digit occurs
        const int holders = __syncthreads_count(nz > 0);
        const int multi = __syncthreads_or(nz > 1);
        unsigned long long run = x - sum;
        for (int w = 0; w < warp; ++w) run += s_part[w];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < per && d0 + i < NB) {
                j.dstart[(int64_t)p * NB + d0 + i] = run;
                run += c[i];
            }
        }
        unsigned long long cmax = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) cmax = c[i] > cmax ? c[i] : cmax;
        const int big = __syncthreads_or(cmax > (unsigned long long)kLocalCap);
        const int act = (n > 0) && (holders > 1 || multi);
        if (tid == 0) j.active[p] = act;
        if (act) {
            p_lo = p_hi;
            p_hi = p;
            hi_big = big;
        }
        nactive += act;
        __syncthreads();
    }
    if (tid == 0) {
        j.active[kFlagQ] = nactive;
        const int msd = LCO_RADIX_LOCAL && !j.lsd_only && nactive == 2 && j.D <= kLocalMaxBits && !hi_big;
        j.active[kFlagMsd] = msd;
        j.active[kFlagHi] = p_hi;
        j.active[kFlagLo] = p_lo;
        j.counters[kCtrUpsweep] = 0;
    }
}

// Shared memory of a scatter CTA: the staged tile (key, value pairs), the
// global base of every digit, the per-warp digit counts (16 bits,
// warp-major: [warp][digit]) and the digit of every staged element (used
// when a digit is not a plain shift of the key).
__host__ __device__ constexpr size_t scatter_smem_bytes(int D) {
    return (size_t)kRadixTile * 16 + ((size_t)1 << D) * 8 + ((size_t)1 << D) * 2 * kRadixWarps +
           (size_t)kRadixTile * 2;
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
// One stable scatter pass.  Each CTA takes the next tile (kRadixTile
// elements, in order of a global counter; warp w holds elements
// w * 256 + 32 i + lane of the tile) and:
//   1. ranks its items within the warp in element order: lanes with equal
//      digits find each other with one match instruction per item, and the
//      lowest of them reads and advances the warp's count of that digit (the
//      matches of all items first, then the chain of count updates);
//   2. turns the per-warp counts into per-warp slots (the tile-local start
//      of that warp's run of each digit) by one block scan over the digit
//      totals, and publishes each digit's count in the tile;
//   3. stages every item, as one 16-byte (key, value) store, at slot + rank:
//      the tile sorted by digit, stably;
//   2b. sums each digit's counts in the tiles before it by decoupled
//      look-back (predecessors read a few at a time, the nearest inclusive
//      word ends the walk) and publishes the inclusive count; the digit's
//      global base is the start of its run in the pass's output plus that
//      prefix (the staging of step 3 overlaps the wait);
//   4. writes the staged tile out in order: each digit's run is a contiguous
//      stretch of the output.
// Every CTA also clears its slice of the look-back words of the next pass to
// run (the previous pass that used them has finished).
// ---------------------------------------------------------------------------
template <bool kShift, typename W>
__global__ void __launch_bounds__(kRadixThreads, kScatterCtas)
    k_radix_scatter(const __grid_constant__ RadixJob j, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_wtot[kRadixWarps];
    using LB = LbWord<W>;
    grid_dep_wait();
    const PassIO io = pass_io(j, pass);
    if (!io.run) return;
    const int D = j.D;
    const int NB = 1 << D;
    double2 *s_kv = reinterpret_cast<double2 *>(smem_raw);                 // [kRadixTile]
    int64_t *s_gb = reinterpret_cast<int64_t *>(s_kv + kRadixTile);        // [NB]
    uint16_t *s_cnt = reinterpret_cast<uint16_t *>(s_gb + NB);             // [warps][NB]
    uint16_t *s_dig = s_cnt + (size_t)NB * kRadixWarps;                    // [kRadixTile]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = job_n(j);
    const int64_t T = tiles_of(n);
    if (io.copy) {
        const int64_t t = blockIdx.x;
        if (t >= T) return;
        const int64_t lo = t * kRadixTile, hi = lo + kRadixTile < n ? lo + kRadixTile : n;
        for (int64_t e = lo + tid; e < hi; e += kRadixThreads) {
            io.dl[e] = relin(j.relin, io.sl[e]);
            io.dv[e] = io.sv[e];
        }
        return;
    }
    const size_t region = (size_t)tiles_of(j.n_cap) * (size_t)NB;
    W *lb_cur = reinterpret_cast<W *>(j.lb) + (size_t)(io.q & 1) * region;
    W *lb_next = reinterpret_cast<W *>(j.lb) + (size_t)((io.q + 1) & 1) * region;
    if ((int64_t)blockIdx.x < T)
        for (int d = tid; d < NB; d += kRadixThreads) lb_next[(size_t)blockIdx.x * NB + d] = 0;
    if (tid == 0) s_tile = atomicAdd(&j.counters[kCtrTile + io.q], 1u);
    uint32_t *cnt_words = reinterpret_cast<uint32_t *>(s_cnt);
    const int nwords = NB / 2;    // word k holds the counts of digits 2k and 2k + 1
    for (int i = tid; i < nwords * kRadixWarps; i += kRadixThreads) cnt_words[i] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= T) return;
    const int64_t tbase = tile * kRadixTile;
    const int tile_n = (int)(n - tbase < (int64_t)kRadixTile ? n - tbase : (int64_t)kRadixTile);
    const int wofs = warp * (32 * kRadixItems) + lane;    // tile-local index of item 0
    const int lim = tile_n - wofs;                        // item i is valid iff 32 i < lim

    // ---- 1. load, digits, stable ranks within the warp ----
    int64_t keys[kRadixItems];
    double vals[kRadixItems];
    {
        const int64_t *kp = io.sl + tbase + wofs;
        const double *vp = io.sv + tbase + wofs;
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const bool valid = i * 32 < lim;
            keys[i] = valid ? __ldg(kp + i * 32) : 0;
            vals[i] = valid ? __ldg(vp + i * 32) : 0.0;
        }
    }
    const uint32_t mask = (uint32_t)NB - 1;
    const int shift = kShift ? (int)j.key_div.shift + pass * D : pass * D;
    uint32_t lab[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const bool valid = i * 32 < lim;
        if (valid && io.first) keys[i] = relin(j.relin, keys[i]);
        // invalid lanes carry labels no valid lane has (digits are < 2^11)
        lab[i] = valid ? key_digit<kShift>(j, keys[i], shift, mask) : (0x10000u | (uint32_t)lane);
    }
    unsigned peers[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) peers[i] = __match_any_sync(kFull, lab[i]);
    uint16_t *wcnt = s_cnt + (size_t)warp * NB;
    uint32_t cb[kRadixItems];
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        uint32_t c = 0;
        if (lane == __ffs(peers[i]) - 1 && lab[i] < 0x10000u) {
            c = wcnt[lab[i]];
            wcnt[lab[i]] = (uint16_t)(c + (uint32_t)__popc(peers[i]));
        }
        cb[i] = c;
        __syncwarp();
    }
    const unsigned lt = lanemask_lt();
    uint32_t dr[kRadixItems];    // digit | rank within the warp's run of the digit << 16
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const uint32_t c = __shfl_sync(kFull, cb[i], __ffs(peers[i]) - 1);
        dr[i] = (lab[i] & 0xffffu) | ((c + (uint32_t)__popc(peers[i] & lt)) << 16);
    }
    __syncthreads();

    // ---- 2. per-warp slots and tile counts; the counts are published ----
    const int wpt = nwords > kRadixThreads ? nwords / kRadixThreads : 1;   // 1, 2 or 4
    const int w0 = tid * wpt;
    {
        uint32_t tsum = 0;
        for (int q = 0; q < wpt; ++q) {
            const int k = w0 + q;
            if (k < nwords) {
                uint32_t s2 = 0;
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) s2 += cnt_words[w * nwords + k];
                tsum += (s2 & 0xffffu) + (s2 >> 16);    // a half never carries (<= 2048 per digit)
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
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = w0 + q;
            if (q >= wpt || k >= nwords) break;
            uint32_t v[kRadixWarps];
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) v[w] = cnt_words[w * nwords + k];
            uint32_t r = run;
            uint32_t sl[kRadixWarps];
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) {
                sl[w] = r;
                r += v[w] & 0xffffu;
            }
            const uint32_t ts_hi = r;
#pragma unroll
            for (int w = 0; w < kRadixWarps; ++w) {
                cnt_words[w * nwords + k] = sl[w] | (r << 16);
                r += v[w] >> 16;
            }
            const uint32_t c_lo = ts_hi - run, c_hi = r - ts_hi;
            // until step 2b, a digit's base slot holds its tile-local start and count
            s_gb[2 * k] = (int64_t)((run << 16) | c_lo);
            s_gb[2 * k + 1] = (int64_t)((ts_hi << 16) | c_hi);
            run = r;
            const W flag = tile == 0 ? LB::kIncl : LB::kAgg;
            LB::store2(lb_cur + (size_t)tile * NB + 2 * k, flag | (W)c_lo, flag | (W)c_hi);
        }
    }
    __syncthreads();
    // ---- 3. staging at the sorted tile-local position ----
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        if (i * 32 < lim) {
            const uint32_t d = dr[i] & 0xffffu;
            const uint32_t pos = (uint32_t)wcnt[d] + (dr[i] >> 16);
            s_kv[pos] = make_double2(__longlong_as_double(keys[i]), vals[i]);
            if (!kShift) s_dig[pos] = (uint16_t)d;
        }
    }
    // ---- 2b. counts of the tiles before (look-back), global bases ----
    {
        const unsigned long long *dst = j.dstart + (int64_t)pass * NB;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = w0 + q;
            if (q >= wpt || k >= nwords) break;
            const uint32_t x_lo = (uint32_t)s_gb[2 * k], x_hi = (uint32_t)s_gb[2 * k + 1];
            W e_lo = 0, e_hi = 0;
            if (tile > 0) {
                // Predecessors are read kBatch pairs at a time; in each round a
                // digit's walk ends at the nearest inclusive word, found with
                // bit masks over the batch (no branch per word; 50.8 vs 53.2 us
                // per pass with a branch per word).
                constexpr int B = LB::kBatch;
                W *my = lb_cur + (size_t)tile * NB + 2 * k;
                bool f_lo = false, f_hi = false;
                const long long t0 = clock64();
                for (int64_t t = tile - 1; !(f_lo && f_hi); t -= B) {
                    W a[B], b[B];
                    uint32_t need_lo = 0, need_hi = 0;
                    for (;;) {
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            a[i] = LB::kIncl;
                            b[i] = LB::kIncl;
                            if (t - i >= 0) LB::load2(lb_cur + (size_t)(t - i) * NB + 2 * k, a[i], b[i]);
                        }
                        uint32_t il = 0, ih = 0, zl = 0, zh = 0;
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            il |= (uint32_t)(LB::flag(a[i]) == 2) << i;
                            ih |= (uint32_t)(LB::flag(b[i]) == 2) << i;
                            zl |= (uint32_t)(LB::flag(a[i]) == 0) << i;
                            zh |= (uint32_t)(LB::flag(b[i]) == 0) << i;
                        }
                        need_lo = f_lo ? 0u : (il ? (2u << (__ffs(il) - 1)) - 1u : (1u << B) - 1u);
                        need_hi = f_hi ? 0u : (ih ? (2u << (__ffs(ih) - 1)) - 1u : (1u << B) - 1u);
                        if (!((zl & need_lo) | (zh & need_hi))) {
                            if (!f_lo) f_lo = il != 0;
                            if (!f_hi) f_hi = ih != 0;
                            break;
                        }
                        if (clock64() - t0 > kSpinBudgetCycles) {
                            set_error(j.status, LCO_ERR_TIMEOUT);
                            need_lo = need_hi = 0;
                            f_lo = f_hi = true;
                            break;
                        }
                        __nanosleep(32);
                    }
#pragma unroll
                    for (int i = 0; i < B; ++i) {
                        e_lo += ((need_lo >> i) & 1u) ? (a[i] & LB::kMask) : (W)0;
                        e_hi += ((need_hi >> i) & 1u) ? (b[i] & LB::kMask) : (W)0;
                    }
                }
                LB::store2(my, LB::kIncl | (e_lo + (W)(x_lo & 0xffffu)), LB::kIncl | (e_hi + (W)(x_hi & 0xffffu)));
            }
            s_gb[2 * k] = (int64_t)dst[2 * k] + (int64_t)e_lo - (int64_t)(x_lo >> 16);
            s_gb[2 * k + 1] = (int64_t)dst[2 * k + 1] + (int64_t)e_hi - (int64_t)(x_hi >> 16);
        }
    }
    __syncthreads();
    // ---- 4. write-out in staged order ----
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
}

// ---------------------------------------------------------------------------
// High digit first, second step: CTA b sorts bucket b of the high digit (a
// contiguous stretch of tmp, at most kLocalCap elements, in source order
// since the high-digit scatter is stable) stably by the low digit and writes
// it to the same stretch of dst.  The bucket's keys are held in shared
// memory; warp w ranks elements [512 w, 512 (w + 1)) in order; one scan
// over the digits turns the per-warp counts into slots; each element's
// sorted position receives its index; the bucket is written out in sorted
// order (coalesced stores; values gathered from the stretch, which the
// scatter has just left in L2).  Keys, indices and counts take 96 KB, so
// two CTAs share an SM (measured on the 3.4M-entry product permutation: 45
// us, against 55 us with keys and values in shared memory at one CTA per
// SM and 57 us for the second global scatter pass it replaces).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t local_smem_bytes() {
    return (size_t)kLocalCap * 10 + (size_t)kLocalWarps * ((size_t)1 << kLocalMaxBits) * 2;
}

template <bool kShift>
__global__ void __launch_bounds__(kLocalThreads, 2) k_radix_local(const __grid_constant__ RadixJob j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_wtot[kLocalWarps];
    grid_dep_wait();
    if (!j.active[kFlagMsd]) return;
    const int D = j.D, NB = 1 << D;
    const int b = blockIdx.x;
    if (b >= NB) return;
    const int p_hi = j.active[kFlagHi], p_lo = j.active[kFlagLo];
    const int64_t s = (int64_t)j.dstart[(int64_t)p_hi * NB + b];
    const int m = (int)j.hist[(int64_t)p_hi * NB + b];   // at most kLocalCap (checked by the upsweep)
    if (m <= 0) return;
    int64_t *s_key = reinterpret_cast<int64_t *>(smem_raw);     // [kLocalCap]
    uint16_t *s_idx = reinterpret_cast<uint16_t *>(s_key + kLocalCap);
    uint16_t *s_cnt = s_idx + kLocalCap;                         // [warps][NB]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t *kin = j.tmp_liv + s;
    const double *vin = j.tmp_val + s;
    uint32_t *cw = reinterpret_cast<uint32_t *>(s_cnt);
    for (int i = tid; i < kLocalWarps * NB / 2; i += kLocalThreads) cw[i] = 0;
    const uint32_t mask = (uint32_t)NB - 1;
    const int shift = kShift ? (int)j.key_div.shift + p_lo * D : p_lo * D;
    const int wbase = warp * (kLocalItems * 32);
    // each warp loads its own elements' keys (every load in flight at once)
    uint32_t dr[kLocalItems];
    {
        int64_t k[kLocalItems];
#pragma unroll
        for (int it = 0; it < kLocalItems; ++it) {
            const int i = wbase + it * 32 + lane;
            k[it] = i < m ? __ldcg(kin + i) : 0;
        }
#pragma unroll
        for (int it = 0; it < kLocalItems; ++it) {
            const int i = wbase + it * 32 + lane;
            if (i < m) s_key[i] = k[it];
            dr[it] = i < m ? key_digit<kShift>(j, k[it], shift, mask) : (0x10000u | (uint32_t)lane);
        }
    }
    __syncthreads();
    uint16_t *wc = s_cnt + warp * NB;
    const unsigned lt = lanemask_lt();
    // lanes with equal digits: one ballot per digit bit (the low digits of a
    // bucket in source order are nearly all distinct within a warp, where a
    // match instruction is slow: 17k vs 11k cycles a bucket alone, but the
    // match unit is shared by the CTAs of an SM)
#pragma unroll
    for (int it = 0; it < kLocalItems; ++it) {
        const bool valid = dr[it] < 0x10000u;
        unsigned peers = __ballot_sync(kFull, valid);
        if (peers) {
#pragma unroll
            for (int bt = 0; bt < kLocalMaxBits; ++bt) {
                if (bt < D) {
                    const bool bit = (dr[it] >> bt) & 1u;
                    const unsigned bb = __ballot_sync(kFull, bit);
                    peers &= bit ? bb : ~bb;
                }
            }
            const int leader = __ffs(peers) - 1;
            uint32_t c = 0;
            if (valid && lane == leader) {
                c = wc[dr[it]];
                wc[dr[it]] = (uint16_t)(c + (uint32_t)__popc(peers));
            }
            __syncwarp();
            c = __shfl_sync(kFull, c, valid ? leader : lane);
            if (valid) dr[it] |= (c + (uint32_t)__popc(peers & lt)) << 16;
        }
    }
    __syncthreads();
    // digit tid: its total over the warps, the exclusive scan over digits,
    // then per-warp slots in place of the counts
    uint32_t tot = 0;
    if (tid < NB) {
#pragma unroll
        for (int w = 0; w < kLocalWarps; ++w) tot += s_cnt[w * NB + tid];
    }
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_wtot[warp] = x;
    __syncthreads();
    uint32_t run = x - tot;
#pragma unroll
    for (int w = 0; w < kLocalWarps; ++w) run += w < warp ? s_wtot[w] : 0u;
    if (tid < NB) {
#pragma unroll
        for (int w = 0; w < kLocalWarps; ++w) {
            const uint32_t v = s_cnt[w * NB + tid];
            s_cnt[w * NB + tid] = (uint16_t)run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kLocalItems; ++it) {
        const int i = wbase + it * 32 + lane;
        if (i < m) s_idx[wc[dr[it] & 0xffffu] + (dr[it] >> 16)] = (uint16_t)i;
    }
    __syncthreads();
    int64_t *kout = j.dst_liv + s;
    double *vout = j.dst_val + s;
#pragma unroll
    for (int h = 0; h < kLocalItems; h += 8) {
        double v[8];
        int idx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int p = tid + (h + u) * kLocalThreads;
            idx[u] = p < m ? s_idx[p] : 0;
            v[u] = p < m ? __ldcg(vin + idx[u]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int p = tid + (h + u) * kLocalThreads;
            if (p < m) {
                kout[p] = s_key[idx[u]];
                vout[p] = v[u];
            }
        }
    }
}

size_t upsweep_smem_bytes(int D, int P) { return (size_t)P * ((size_t)1 << D) * 4; }

// Look-back words are 32-bit below this many elements.
constexpr int64_t kNarrowLbMax = (int64_t)1 << 30;

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

// One counting CTA per range of whole tiles, up to kUpsweepCtasPerSm per SM.
int radix_ranges(int64_t n_cap) {
    const int64_t tiles = tiles_of(n_cap);
    const int64_t gmax = (int64_t)kUpsweepCtasPerSm * radix_sm_count();
    int64_t g = tiles < gmax ? tiles : gmax;
    if (g < 1) g = 1;
    return (int)g;
}

size_t radix_state_bytes(int64_t n_cap, int D, int P) {
    const size_t NB = (size_t)1 << D;
    const size_t wsz = n_cap >= kNarrowLbMax ? 8 : 4;
    size_t b = 0;
    b += align_up(32 * 4);                                   // active
    b += align_up((size_t)P * NB * 8);                       // hist
    b += align_up((size_t)P * NB * 8);                       // dstart
    b += align_up(2 * (size_t)tiles_of(n_cap) * NB * wsz);   // look-back regions
    return b;
}

size_t radix_hist_table_bytes() { return align_up(32 * 4); }

void radix_carve(RadixJob &job, char *region) {
    const size_t NB = (size_t)1 << job.D;
    job.G = radix_ranges(job.n_cap);
    job.wide_lb = job.n_cap >= kNarrowLbMax ? 1 : 0;
    char *p = region;
    job.active = reinterpret_cast<int32_t *>(p); p += align_up(32 * 4);
    job.hist = reinterpret_cast<unsigned long long *>(p); p += align_up((size_t)job.P * NB * 8);
    job.dstart = reinterpret_cast<unsigned long long *>(p); p += align_up((size_t)job.P * NB * 8);
    job.lb = p;
}

namespace {

template <bool kShift, typename W>
void launch_scatter(const RadixJob &job, int p, unsigned grid, cudaStream_t stream) {
    // after the counting launch or the previous pass: a dependent launch
    LCO_LAUNCH("k_radix_scatter", stream,
               launch_dependent(k_radix_scatter<kShift, W>, grid, kRadixThreads, scatter_smem_bytes(job.D), stream,
                                job, p));
}

}  // namespace

cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream) {
    // function attributes are per device: set them once on each
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        const int bytes = (int)scatter_smem_bytes(kMaxDigitBits);
        cudaFuncSetAttribute(k_radix_scatter<true, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_radix_scatter<false, uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_radix_scatter<true, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_radix_scatter<false, uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_radix_upsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upsweep_smem_bytes(kMaxDigitBits, kMaxPasses));
        cudaFuncSetAttribute(k_radix_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)local_smem_bytes());
        cudaFuncSetAttribute(k_radix_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)local_smem_bytes());
        attr_done.fetch_or(bit);
    }
    if (job.n_cap <= 0) return cudaSuccess;
    const int NB = 1 << job.D;
    // the counting launch adds into the digit table: clear it first
    cudaError_t err = cudaMemsetAsync(job.hist, 0, (size_t)job.P * NB * 8, stream);
    if (err != cudaSuccess) return err;
    LCO_LAUNCH("k_radix_upsweep", stream,
               k_radix_upsweep<<<(unsigned)job.G, kRadixThreads, upsweep_smem_bytes(job.D, job.P), stream>>>(job));
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const unsigned grid = (unsigned)tiles_of(job.n_cap);
    const bool shift = job.key_div.pow2 != 0;
    for (int p = 0; p < job.P; ++p) {
        if (job.wide_lb) {
            if (shift) launch_scatter<true, uint64_t>(job, p, grid, stream);
            else launch_scatter<false, uint64_t>(job, p, grid, stream);
        } else {
            if (shift) launch_scatter<true, uint32_t>(job, p, grid, stream);
            else launch_scatter<false, uint32_t>(job, p, grid, stream);
        }
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    // high digit first (decided on the device; a no-op otherwise): possible
    // only for digit widths the local sort takes and two or more passes
    if (LCO_RADIX_LOCAL && !job.lsd_only && job.P >= 2 && job.D <= kLocalMaxBits) {
        // after the last pass: a dependent launch
        if (shift) LCO_LAUNCH("k_radix_local", stream,
                              launch_dependent(k_radix_local<true>, (unsigned)NB, kLocalThreads, local_smem_bytes(),
                                               stream, job));
        else LCO_LAUNCH("k_radix_local", stream,
                        launch_dependent(k_radix_local<false>, (unsigned)NB, kLocalThreads, local_smem_bytes(),
                                         stream, job));
        err = cudaGetLastError();
    }
    return err;
}

}  // namespace lco
