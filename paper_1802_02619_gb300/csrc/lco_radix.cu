// lco_radix.cu -- histogram and scatter kernels of the stable LSD radix engine.
#include <atomic>

#include "lco_radix.cuh"

namespace lco {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUpItems = 8;   // histogram kernels: loads in flight per thread
constexpr int kOffItems = 16; // offsets kernel: ranges per lane (G <= 512)
constexpr int kScatterCtas = 4; // scatter CTAs resident per SM (9-bit digits)

// In-place exclusive scan of n (<= 256 * 8) 32-bit values held in shared
// memory, by a block of kRadixThreads threads.  Returns the total.
__device__ uint32_t block_exscan_u32(uint32_t *a, int n) {
    __shared__ uint32_t s_warp[kRadixWarps];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kRadixThreads - 1) / kRadixThreads;
    const int start = tid * per;
    uint32_t local = 0;
    for (int i = 0; i < per; ++i)
        if (start + i < n) local += a[start + i];
    uint32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kRadixWarps ? s_warp[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += v;
        }
        if (lane < kRadixWarps) s_warp[lane] = wi - w;
        if (lane == kRadixWarps - 1) s_total = wi;
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + incl - local;
    for (int i = 0; i < per; ++i) {
        if (start + i < n) {
            uint32_t v = a[start + i];
            a[start + i] = run;
            run += v;
        }
    }
    __syncthreads();
    return s_total;
}

// Exclusive scan of n (<= 256 * 8) 64-bit values in shared memory.
__device__ void block_exscan_u64(uint64_t *a, int n) {
    __shared__ uint64_t s_warp64[kRadixWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + kRadixThreads - 1) / kRadixThreads;
    const int start = tid * per;
    uint64_t local = 0;
    for (int i = 0; i < per; ++i)
        if (start + i < n) local += a[start + i];
    uint64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp64[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kRadixWarps ? s_warp64[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t v = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += v;
        }
        if (lane < kRadixWarps) s_warp64[lane] = wi - w;
    }
    __syncthreads();
    uint64_t run = s_warp64[warp] + incl - local;
    for (int i = 0; i < per; ++i) {
        if (start + i < n) {
            uint64_t v = a[start + i];
            a[start + i] = run;
            run += v;
        }
    }
    __syncthreads();
}

// Element count; a device-side count never exceeds the capacity the
// buffers were sized for.
__device__ __forceinline__ int64_t job_n(const RadixJob &j) {
    if (!j.n_dev) return j.n_host;
    const int64_t n = *j.n_dev;
    return n < j.n_cap ? n : j.n_cap;
}

// Range r of the G ranges: a whole number of tiles, the last one ragged.
__device__ __forceinline__ void range_of(const RadixJob &j, int64_t n, int64_t r, int64_t &lo, int64_t &hi) {
    int64_t per = (n + j.G - 1) / j.G;
    per = (per + kRadixTile - 1) / kRadixTile * kRadixTile;
    lo = r * per;
    hi = lo + per;
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

// ---------------------------------------------------------------------------
// One read of the source keys: every pass's digit histogram, per range
// (counts_src) and in total (ghist).  The last block to finish turns the
// totals into exclusive digit offsets, flags passes whose digit is constant
// (nothing to do) and leaves ghist zeroed for the next call.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const __grid_constant__ RadixJob j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ int s_last;
    const int NB = 1 << j.D;
    const int nh = j.P * NB;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) s_hist[i] = 0;
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
        j.counts_src[((int64_t)p * NB + d) * j.G + blockIdx.x] = s_hist[i];
        if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&j.ghist[i]), (unsigned long long)s_hist[i]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&j.counters[8], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: exclusive scans, pass activity, counter reset
    uint64_t *s_h64 = reinterpret_cast<uint64_t *>(smem_raw);   // NB entries
    __shared__ int s_triv;
    int nactive = 0;
    for (int p = 0; p < j.P; ++p) {
        if (threadIdx.x == 0) s_triv = 0;
        __syncthreads();
        for (int d = threadIdx.x; d < NB; d += blockDim.x) {
            uint64_t c = atomicAdd(reinterpret_cast<unsigned long long *>(&j.ghist[p * NB + d]), 0ull);
            s_h64[d] = c;
            if ((int64_t)c == n) s_triv = 1;
            j.ghist[p * NB + d] = 0;
        }
        __syncthreads();
        block_exscan_u64(s_h64, NB);
        for (int d = threadIdx.x; d < NB; d += blockDim.x) j.offs[p * NB + d] = s_h64[d];
        int act = (n > 0) && !s_triv;
        if (threadIdx.x == 0) j.active[p] = act;
        nactive += act;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        j.active[16] = nactive;
        j.counters[8] = 0;
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

// roffs[r][d] = offs[pass][d] + sum of counts[r'][d] over ranges r' < r.
// One warp per digit.  The count tables are digit-major ([d][G]), so a warp
// reads 32 consecutive ranges per load; lane l holds ranges i * 32 + l.
__global__ void __launch_bounds__(kRadixThreads) k_radix_offsets(const __grid_constant__ RadixJob j, int pass) {
    const PassIO io = pass_io(j, pass);
    if (!io.run || io.copy) return;
    const int NB = 1 << j.D;
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * kRadixWarps + (threadIdx.x >> 5);
    if (d >= NB) return;
    const uint32_t *cnt = (io.first ? j.counts_src + (int64_t)pass * NB * j.G : j.counts_hist) + (int64_t)d * j.G;
    // all loads issued before the scans (G <= 32 * kOffItems)
    uint32_t c[kOffItems];
#pragma unroll
    for (int i = 0; i < kOffItems; ++i) {
        const int r = i * 32 + lane;
        c[i] = r < j.G ? cnt[r] : 0u;
    }
    uint64_t run = j.offs[pass * NB + d];
#pragma unroll
    for (int i = 0; i < kOffItems; ++i) {
        uint64_t x = c[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += u;
        }
        const int r = i * 32 + lane;
        if (r < j.G) j.roffs[(int64_t)r * NB + d] = run + x - c[i];
        run += __shfl_sync(kFull, x, 31);
    }
}

// Staging buffer and digit tables of a scatter CTA, rounded up to 128 bytes
// (the bulk form's input buffers follow: copy destinations must be aligned).
__host__ __device__ constexpr size_t scatter_smem_bytes_base(int D) {
    return ((size_t)kRadixTile * 16 + ((size_t)1 << D) * 16 + ((size_t)1 << D) * 4 +
            (size_t)kRadixWarps * ((size_t)1 << D) * 2 + 127) & ~(size_t)127;
}

// ---------------------------------------------------------------------------
// One stable scatter pass: CTA r walks range r tile by tile (kRadixTile
// elements), ranking each tile with warp match instructions and placing it
// from running per-digit offsets; the tile is staged in shared memory so
// that the writes of each digit's run are contiguous.  Digit tables use
// 16-bit warp counts and digits are recomputed at write-out, to keep shared
// memory small.  Two forms:
//   kBulk: the next input tile comes in by bulk copy while the current one
//     is ranked (double-buffered input, two CTAs per SM) -- for ranges of
//     many tiles;
//   otherwise: tiles are loaded directly and only the staging buffer and
//     the digit tables are in shared memory, so four CTAs fit on an SM and
//     their tiles fill each other's barrier gaps -- for ranges of few tiles.
// ---------------------------------------------------------------------------
template <bool kBulk>
__global__ void __launch_bounds__(kRadixThreads, kBulk ? 2 : kScatterCtas)
    k_radix_scatter(const __grid_constant__ RadixJob j, int pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PassIO io = pass_io(j, pass);
    if (!io.run) return;
    const int NB = 1 << j.D;
    int64_t *s_key = reinterpret_cast<int64_t *>(smem_raw);
    double *s_val = reinterpret_cast<double *>(s_key + kRadixTile);
    int64_t *s_run = reinterpret_cast<int64_t *>(s_val + kRadixTile);
    int64_t *s_gbase = s_run + NB;
    uint32_t *s_tstart = reinterpret_cast<uint32_t *>(s_gbase + NB);
    uint16_t *s_whist = reinterpret_cast<uint16_t *>(s_tstart + NB);
    // bulk form only: the input buffers and their barrier, after the tables
    int64_t *in_key = reinterpret_cast<int64_t *>(smem_raw + scatter_smem_bytes_base(j.D));
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
    const int shift = pass * j.D;
    for (int d = tid; d < NB; d += kRadixThreads) s_run[d] = (int64_t)j.roffs[(int64_t)blockIdx.x * NB + d];
    const unsigned lt = lanemask_lt();
    uint16_t *wh = s_whist + warp * NB;
    // bulk form: the next tile is copied in while the current one is ranked
    // and scattered, when both input arrays are 16-byte aligned (tile starts
    // are even element offsets); an odd last element is read directly
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
    if (bulk) {
        if (tid == 0) {
            mbar_init(s_bar, 1);
            if (lo < hi) issue(lo);
        }
        __syncthreads();
    }

    for (int64_t tile_base = lo; tile_base < hi; tile_base += kRadixTile) {
        const int tile_n = (int)((hi - tile_base) < (int64_t)kRadixTile ? (hi - tile_base) : (int64_t)kRadixTile);
        const int64_t bulk_end = bulk ? tile_base + (tile_n & ~1) : tile_base;
        for (int i = tid; i < kRadixWarps * NB / 2; i += kRadixThreads) reinterpret_cast<uint32_t *>(s_whist)[i] = 0;
        if (bulk && bulk_end > tile_base) {
            const bool ok = mbar_wait_bounded(s_bar, parity);
            parity ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) set_error(j.status, LCO_ERR_TIMEOUT);
                return;
            }
        }
        int64_t keys[kRadixItems];
        double vals[kRadixItems];
        uint32_t digs[kRadixItems];
        const int64_t wbase = tile_base + warp * (32 * kRadixItems);
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const int64_t e = wbase + i * 32 + lane;
            keys[i] = 0;
            vals[i] = 0.0;
            if (e < bulk_end) {
                keys[i] = in_key[e - tile_base];
                vals[i] = in_val[e - tile_base];
            } else if (e < hi) {
                keys[i] = __ldg(io.sl + e);
                vals[i] = __ldg(io.sv + e);
            }
        }
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const int64_t e = wbase + i * 32 + lane;
            if (io.first && e < hi) keys[i] = relin(j.relin, keys[i]);
            digs[i] = e < hi ? (uint32_t)((divu(j.key_div, (uint64_t)keys[i]) >> shift) & mask) : 0u;
        }
        __syncthreads();
        // the input buffer is free: fetch the next tile behind this one's work
        if (bulk && tid == 0 && tile_base + kRadixTile < hi) issue(tile_base + kRadixTile);
        // warp-level stable ranking: the lanes holding the same digit find each
        // other with one match instruction (invalid lanes carry a digit no
        // valid lane has); the rank is packed above the digit (digit < 2^11,
        // rank < 2^13) to keep registers low
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const int64_t e = wbase + i * 32 + lane;
            const bool valid = e < hi;
            const uint32_t d = digs[i];
            const unsigned peers = __match_any_sync(kFull, valid ? d : 0xffffu);
            const int leader = valid ? (__ffs(peers) - 1) : lane;
            uint32_t basev = 0;
            if (valid && lane == leader) {
                basev = wh[d];
                wh[d] = (uint16_t)(basev + (uint32_t)__popc(peers));
            }
            basev = __shfl_sync(kFull, basev, leader);
            digs[i] = d | ((basev + (uint32_t)__popc(peers & lt)) << 16);
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive offsets of the warps, tile count
        for (int d = tid; d < NB; d += kRadixThreads) {
            uint32_t run = 0;
            for (int w = 0; w < kRadixWarps; ++w) {
                const uint32_t c = s_whist[w * NB + d];
                s_whist[w * NB + d] = (uint16_t)run;
                run += c;
            }
            s_tstart[d] = run;
        }
        __syncthreads();
        // global start of each digit's run in this tile, then local starts
        for (int d = tid; d < NB; d += kRadixThreads) {
            s_gbase[d] = s_run[d];
            s_run[d] += s_tstart[d];
        }
        __syncthreads();
        block_exscan_u32(s_tstart, NB);
        for (int d = tid; d < NB; d += kRadixThreads) s_gbase[d] -= (int64_t)s_tstart[d];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kRadixItems; ++i) {
            const int64_t e = wbase + i * 32 + lane;
            if (e < hi) {
                const uint32_t d = digs[i] & 0xffffu;
                const uint32_t lp = s_tstart[d] + wh[d] + (digs[i] >> 16);
                s_key[lp] = keys[i];
                s_val[lp] = vals[i];
            }
        }
        __syncthreads();
        for (int i = tid; i < tile_n; i += kRadixThreads) {
            const int64_t k = s_key[i];
            const uint32_t d = (uint32_t)((divu(j.key_div, (uint64_t)k) >> shift) & mask);
            const int64_t g = s_gbase[d] + i;
            io.dl[g] = k;
            io.dv[g] = s_val[i];
        }
        __syncthreads();
    }
}

size_t scatter_smem_bytes(int D, bool bulk) {
    return scatter_smem_bytes_base(D) + (bulk ? (size_t)kRadixTile * 16 + 16 : 0);
}

size_t upsweep_smem_bytes(int D, int P) {
    size_t NB = (size_t)1 << D;
    size_t a = (size_t)P * NB * 4, b = NB * 8;
    return a > b ? a : b;
}

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

// The histogram and offset tables have a fixed size (the largest digit plan)
// so that jobs with different plans can share one region: every job leaves
// the histogram table zeroed, and a zero-filled region starts that way.
constexpr size_t kHistTableBytes = (size_t)kMaxPasses * ((size_t)1 << kMaxDigitBits) * 8;

// Up to kBulkMinTiles tiles per CTA of a four-per-SM wave, the direct
// scatter runs (at least two tiles per range); beyond, the bulk-copy form
// (two CTAs per SM, at least four tiles per range).
constexpr int64_t kBulkMinTiles = 4;

bool radix_bulk(int64_t n_cap) {
    const int64_t tiles = (n_cap + kRadixTile - 1) / kRadixTile;
    return tiles > kBulkMinTiles * kScatterCtas * (int64_t)radix_sm_count();
}

int radix_ranges(int64_t n_cap) {
    const int64_t tiles = (n_cap + kRadixTile - 1) / kRadixTile;
    const bool bulk = radix_bulk(n_cap);
    int64_t g = bulk ? (tiles + 3) / 4 : (tiles + 1) / 2;
    int64_t gmax = (bulk ? 2 : kScatterCtas) * (int64_t)radix_sm_count();   // one wave of scatter CTAs
    if (gmax > 32 * kOffItems) gmax = 32 * kOffItems;
    if (g > gmax) g = gmax;
    if (g < 1) g = 1;
    return (int)g;
}

size_t radix_state_bytes(int64_t n_cap, int D, int P) {
    const size_t NB = (size_t)1 << D;
    const size_t G = (size_t)radix_ranges(n_cap);
    size_t b = 0;
    b += align_up(kHistTableBytes);      // ghist
    b += align_up(kHistTableBytes);      // offs
    b += align_up(32 * 4);               // active
    b += align_up((size_t)P * G * NB * 4);   // counts_src
    b += align_up(G * NB * 4);           // counts_hist
    b += align_up(G * NB * 8);           // roffs
    return b;
}

size_t radix_hist_table_bytes() { return align_up(kHistTableBytes); }

void radix_carve(RadixJob &job, char *region) {
    const size_t NB = (size_t)1 << job.D;
    job.G = radix_ranges(job.n_cap);
    const size_t G = (size_t)job.G;
    char *p = region;
    job.ghist = reinterpret_cast<uint64_t *>(p); p += align_up(kHistTableBytes);
    job.offs = reinterpret_cast<uint64_t *>(p); p += align_up(kHistTableBytes);
    job.active = reinterpret_cast<int32_t *>(p); p += align_up(32 * 4);
    job.counts_src = reinterpret_cast<uint32_t *>(p); p += align_up((size_t)job.P * G * NB * 4);
    job.counts_hist = reinterpret_cast<uint32_t *>(p); p += align_up(G * NB * 4);
    job.roffs = reinterpret_cast<uint64_t *>(p);
}

cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream) {
    // function attributes are per device: set them once on each
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        cudaFuncSetAttribute(k_radix_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem_bytes(kMaxDigitBits, true));
        cudaFuncSetAttribute(k_radix_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem_bytes(kMaxDigitBits, false));
        cudaFuncSetAttribute(k_radix_upsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upsweep_smem_bytes(kMaxDigitBits, kMaxPasses));
        attr_done.fetch_or(bit);
    }
    if (job.n_cap <= 0) return cudaSuccess;
    const unsigned G = (unsigned)job.G;
    const int NB = 1 << job.D;
    LCO_LAUNCH("k_radix_upsweep", stream,
               k_radix_upsweep<<<G, kRadixThreads, upsweep_smem_bytes(job.D, job.P), stream>>>(job));
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    for (int p = 0; p < job.P; ++p) {
        if (p > 0) {
            LCO_LAUNCH("k_radix_hist", stream,
                       k_radix_hist<<<G, kRadixThreads, (size_t)NB * 4, stream>>>(job, p));
        }
        LCO_LAUNCH("k_radix_offsets", stream,
                   k_radix_offsets<<<(unsigned)((NB + kRadixWarps - 1) / kRadixWarps), kRadixThreads, 0, stream>>>(job, p));
        if (radix_bulk(job.n_cap)) {
            LCO_LAUNCH("k_radix_scatter", stream,
                       k_radix_scatter<true><<<G, kRadixThreads, scatter_smem_bytes(job.D, true), stream>>>(job, p));
        } else {
            LCO_LAUNCH("k_radix_scatter", stream,
                       k_radix_scatter<false><<<G, kRadixThreads, scatter_smem_bytes(job.D, false), stream>>>(job, p));
        }
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace lco
