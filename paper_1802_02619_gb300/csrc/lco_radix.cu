// lco_radix.cu -- histogram and scatter kernels of the stable LSD radix engine.
#include "lco_radix.cuh"

namespace lco {

namespace {

constexpr unsigned kFull = 0xffffffffu;

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

// ---------------------------------------------------------------------------
// One read of the keys: every pass's digit histogram.  Also clears the
// look-back state of all passes.  The last block to finish turns the
// histograms into exclusive digit offsets, flags passes whose digit is
// constant (nothing to do), and resets the counters for the next call.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const __grid_constant__ RadixJob j, int64_t state_words) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ int s_last;
    const int NB = 1 << j.D;
    const int nh = j.P * NB;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();

    const int64_t n = job_n(j);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
    const uint32_t mask = (uint32_t)NB - 1;
    for (int64_t e = gtid; e < n; e += gsz) {
        int64_t liv = relin(j.relin, j.src_liv[e]);
        uint64_t key = divu(j.key_div, (uint64_t)liv);
        for (int p = 0; p < j.P; ++p)
            atomicAdd(&s_hist[p * NB + (uint32_t)((key >> (p * j.D)) & mask)], 1u);
    }
    // clear look-back state for the scatter passes
    for (int64_t w = gtid; w < state_words; w += gsz) j.state[w] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nh; i += blockDim.x)
        if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&j.ghist[i]),
                                 (unsigned long long)s_hist[i]);
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
        for (int p = 0; p < kMaxPasses; ++p) j.counters[p] = 0;
        j.counters[8] = 0;
    }
}

// ---------------------------------------------------------------------------
// One stable scatter pass over a tile of kRadixTile elements.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRadixThreads, 1) k_radix_scatter(const __grid_constant__ RadixJob j, int pass, int64_t tiles_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NB = 1 << j.D;
    int64_t *s_key = reinterpret_cast<int64_t *>(smem_raw);
    double *s_val = reinterpret_cast<double *>(s_key + kRadixTile);
    int64_t *s_gbase = reinterpret_cast<int64_t *>(s_val + kRadixTile);
    uint32_t *s_whist = reinterpret_cast<uint32_t *>(s_gbase + NB);
    uint32_t *s_tstart = s_whist + kRadixWarps * NB;
    uint16_t *s_dig = reinterpret_cast<uint16_t *>(s_tstart + NB);
    __shared__ int64_t s_tile;

    const int Q = j.active[16];
    const bool act = j.active[pass] != 0;
    const bool copy_mode = (Q == 0) && (pass == j.P - 1);
    if (!act && !copy_mode) return;
    int q = 0;
    for (int p = 0; p < pass; ++p) q += j.active[p] != 0;

    const int64_t n = job_n(j);
    const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    if (threadIdx.x == 0) s_tile = atomicAdd(&j.counters[pass], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) return;

    const bool first = copy_mode || q == 0;
    const int64_t *src_liv = first ? j.src_liv : (((Q - 1 - (q - 1)) & 1) == 0 ? j.dst_liv : j.tmp_liv);
    const double *src_val = first ? j.src_val : (((Q - 1 - (q - 1)) & 1) == 0 ? j.dst_val : j.tmp_val);
    int64_t *dst_liv = copy_mode || (((Q - 1 - q) & 1) == 0) ? j.dst_liv : j.tmp_liv;
    double *dst_val = copy_mode || (((Q - 1 - q) & 1) == 0) ? j.dst_val : j.tmp_val;

    const int64_t tile_base = tile * kRadixTile;
    const int tile_n = (int)((n - tile_base) < (int64_t)kRadixTile ? (n - tile_base) : (int64_t)kRadixTile);

    if (copy_mode) {
        for (int i = threadIdx.x; i < tile_n; i += blockDim.x) {
            int64_t e = tile_base + i;
            dst_liv[e] = relin(j.relin, src_liv[e]);
            dst_val[e] = src_val[e];
        }
        return;
    }

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t mask = (uint32_t)NB - 1;
    const int shift = pass * j.D;

    for (int i = tid; i < kRadixWarps * NB; i += kRadixThreads) s_whist[i] = 0;

    int64_t keys[kRadixItems];
    double vals[kRadixItems];
    uint32_t digs[kRadixItems];
    const int64_t wbase = tile_base + warp * (32 * kRadixItems);
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        int64_t e = wbase + i * 32 + lane;
        if (e < n) {
            int64_t k = src_liv[e];
            if (first) k = relin(j.relin, k);
            keys[i] = k;
            vals[i] = src_val[e];
            digs[i] = (uint32_t)((divu(j.key_div, (uint64_t)k) >> shift) & mask);
        } else {
            keys[i] = 0;
            vals[i] = 0.0;
            digs[i] = 0;
        }
    }
    __syncthreads();

    // warp-level stable ranking (multi-split by ballots); the rank is packed
    // above the digit (digit < 2^11, rank < 2^13) to keep registers low
    uint32_t *wh = s_whist + warp * NB;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = wbase + i * 32 + lane;
        const bool valid = e < n;
        const unsigned vmask = __ballot_sync(kFull, valid);
        unsigned peers = vmask;
        const uint32_t d = digs[i];
        for (int b = 0; b < j.D; ++b) {
            const unsigned bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(kFull, bit);
            peers &= bit ? bal : ~bal;
        }
        const int leader = valid ? (__ffs(peers) - 1) : lane;
        uint32_t basev = 0;
        if (valid && lane == leader) {
            basev = wh[d];
            wh[d] = basev + (uint32_t)__popc(peers);
        }
        basev = __shfl_sync(kFull, basev, leader);
        digs[i] = d | ((basev + (uint32_t)__popc(peers & lt)) << 16);
        __syncwarp();
    }
    __syncthreads();

    // per-digit counts: exclusive over warps, total per tile; publish aggregates
    uint64_t *st_pass = j.state + (int64_t)pass * tiles_cap * NB;
    for (int d = tid; d < NB; d += kRadixThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kRadixWarps; ++w) {
            uint32_t c = s_whist[w * NB + d];
            s_whist[w * NB + d] = run;
            run += c;
        }
        s_tstart[d] = run;
        lb_store(st_pass + tile * NB + d, (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)run);
    }
    __syncthreads();
    for (int d = tid; d < NB; d += kRadixThreads) {
        uint64_t excl = 0;
        if (tile > 0) {
            excl = lookback(st_pass + d, tile, NB, j.status);
            lb_store(st_pass + tile * NB + d, kFlagIncl | (excl + s_tstart[d]));
        }
        s_gbase[d] = (int64_t)(j.offs[pass * NB + d] + excl);
    }
    __syncthreads();
    block_exscan_u32(s_tstart, NB);
    for (int d = tid; d < NB; d += kRadixThreads) s_gbase[d] -= (int64_t)s_tstart[d];
    __syncthreads();

#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const int64_t e = wbase + i * 32 + lane;
        if (e < n) {
            const uint32_t d = digs[i] & 0xffffu;
            const uint32_t lp = s_tstart[d] + wh[d] + (digs[i] >> 16);
            s_key[lp] = keys[i];
            s_val[lp] = vals[i];
            s_dig[lp] = (uint16_t)d;
        }
    }
    __syncthreads();
    for (int i = tid; i < tile_n; i += kRadixThreads) {
        const uint32_t d = s_dig[i];
        const int64_t g = s_gbase[d] + i;
        dst_liv[g] = s_key[i];
        dst_val[g] = s_val[i];
    }
}

size_t scatter_smem_bytes(int D) {
    size_t NB = (size_t)1 << D;
    return (size_t)kRadixTile * 16 + NB * 8 + (size_t)kRadixWarps * NB * 4 + NB * 4 +
           (size_t)kRadixTile * 2;
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

size_t radix_state_bytes(int64_t n_cap, int D, int P) {
    const size_t NB = (size_t)1 << D;
    const size_t tiles = (size_t)((n_cap + kRadixTile - 1) / kRadixTile);
    size_t b = 0;
    b += align_up(kHistTableBytes);      // ghist
    b += align_up(kHistTableBytes);      // offs
    b += align_up(32 * 4);               // active
    b += align_up((size_t)P * (tiles ? tiles : 1) * NB * 8);   // look-back state
    return b;
}

size_t radix_hist_table_bytes() { return align_up(kHistTableBytes); }

void radix_carve(RadixJob &job, char *region) {
    char *p = region;
    job.ghist = reinterpret_cast<uint64_t *>(p); p += align_up(kHistTableBytes);
    job.offs = reinterpret_cast<uint64_t *>(p); p += align_up(kHistTableBytes);
    job.active = reinterpret_cast<int32_t *>(p); p += align_up(32 * 4);
    job.state = reinterpret_cast<uint64_t *>(p);
}

cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream) {
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem_bytes(kMaxDigitBits));
        cudaFuncSetAttribute(k_radix_upsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upsweep_smem_bytes(kMaxDigitBits, kMaxPasses));
        attr_done = true;
    }
    if (job.n_cap <= 0) return cudaSuccess;
    const int64_t tiles_cap = (job.n_cap + kRadixTile - 1) / kRadixTile;
    const int64_t NB = (int64_t)1 << job.D;
    const int64_t state_words = (int64_t)job.P * tiles_cap * NB;
    int up_grid = radix_sm_count() * kUpsweepCtasPerSm;
    const int64_t want = (job.n_cap + kRadixThreads * 8 - 1) / (kRadixThreads * 8);
    if (want < up_grid) up_grid = (int)(want > 0 ? want : 1);
    LCO_LAUNCH("k_radix_upsweep", stream, k_radix_upsweep<<<up_grid, kRadixThreads, upsweep_smem_bytes(job.D, job.P), stream>>>(job, state_words));
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    for (int p = 0; p < job.P; ++p) {
        LCO_LAUNCH("k_radix_scatter", stream, k_radix_scatter<<<(unsigned)tiles_cap, kRadixThreads, scatter_smem_bytes(job.D), stream>>>(job, p, tiles_cap));
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace lco
