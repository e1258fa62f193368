// lco_internal.cuh -- device helpers shared by the LCO kernels (not part of the ABI).
#pragma once

#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include "lco.h"
#include <nvtx3/nvToolsExt.h>

namespace lco {

constexpr int kMaxOrder = LCO_MAX_ORDER;
constexpr int kWsHeaderBytes = 256;
// Bounded device waits: a look-back spin gives up after this many SM clock
// cycles (about one second at 2 GHz), records LCO_ERR_TIMEOUT and continues
// with a zero contribution so that the kernel always terminates.  The wait
// helpers take the budget as an argument (default kSpinBudgetCycles); only
// the wait self-test passes a smaller one, to its own kernel.
constexpr long long kSpinBudgetCycles = 2000000000LL;

// ---------------------------------------------------------------------------
// Unsigned 64-bit division by an invariant divisor.
//
// Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), Fig. 4.1: for a divisor d >= 1 let
// l = ceil(log2 d) and m' = floor(2^64 (2^l - d) / d) + 1; then for every
// 64-bit n, q = (t1 + ((n - t1) >> 1)) >> (l - 1) with t1 = mulhi(m', n).
// Powers of two use a plain shift.
// ---------------------------------------------------------------------------
struct DivU64 {
    uint64_t d;
    uint64_t m;
    uint32_t shift;
    uint32_t pow2;
};

inline DivU64 make_div(uint64_t d) {
    DivU64 v{};
    v.d = d;
    if ((d & (d - 1)) == 0) {
        v.pow2 = 1;
        v.shift = (uint32_t)__builtin_ctzll(d);
        v.m = 0;
        return v;
    }
    uint32_t l = 64u - (uint32_t)__builtin_clzll(d - 1);   // ceil(log2 d), 2 <= l <= 63
    unsigned __int128 num = ((unsigned __int128)((1ull << l) - d)) << 64;
    v.m = (uint64_t)(num / d) + 1u;
    v.shift = l - 1;
    v.pow2 = 0;
    return v;
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ uint64_t divu(const DivU64 &v, uint64_t n) {
    if (v.pow2) return n >> v.shift;
    uint64_t t1 = mulhi64(v.m, n);
    return (t1 + ((n - t1) >> 1)) >> v.shift;
}

// ---------------------------------------------------------------------------
// Unsigned 128-bit dividend, 64-bit invariant divisor (wide LIVs).
//
// The high word goes through DivU64; the rest is one "2-by-1" step of
// Moeller & Granlund, "Improved division by invariant integers" (IEEE
// Trans. Computers 60(2), 2011), Algorithm 4: with the divisor normalised
// (d_n = d << s, top bit set) and its reciprocal v = floor((2^128 - 1) /
// d_n) - 2^64, a two-word numerator (u1, u0) with u1 < d_n gives q and r
// from one 64x64 product, a two-word add and at most two corrections.
// ---------------------------------------------------------------------------
struct DivU128by64 {
    DivU64 hi;     // for the high word
    uint64_t dn;   // d << s
    uint64_t v;    // reciprocal of dn
    uint32_t s;    // normalisation shift
    uint32_t pad;
};

inline DivU128by64 make_div128(uint64_t d) {
    DivU128by64 w{};
    w.hi = make_div(d);
    w.s = (uint32_t)__builtin_clzll(d);
    w.dn = d << w.s;
    const unsigned __int128 all = ~(unsigned __int128)0;
    w.v = (uint64_t)(all / w.dn - ((unsigned __int128)1 << 64));
    return w;
}

// x = q * d + r, 0 <= r < d; returns q, writes r.
__host__ __device__ __forceinline__ unsigned __int128 divu128(const DivU128by64 &w, unsigned __int128 x,
                                                             uint64_t &r) {
    const uint64_t xh = (uint64_t)(x >> 64), xl = (uint64_t)x;
    const uint64_t d = w.hi.d;
    const uint64_t qh = divu(w.hi, xh);
    const uint64_t rh = xh - qh * d;
    // normalise the two-word remainder (rh, xl): rh < d, so u1 < dn
    const uint64_t u1 = w.s ? (rh << w.s) | (xl >> (64 - w.s)) : rh;
    const uint64_t u0 = xl << w.s;
    const unsigned __int128 p = (unsigned __int128)w.v * u1;
    const unsigned __int128 qq = p + ((((unsigned __int128)(u1 + 1)) << 64) | u0);
    uint64_t q1 = (uint64_t)(qq >> 64);
    const uint64_t q0 = (uint64_t)qq;
    uint64_t rr = u0 - q1 * w.dn;
    if (rr > q0) {
        --q1;
        rr += w.dn;
    }
    if (rr >= w.dn) {
        ++q1;
        rr -= w.dn;
    }
    r = rr >> w.s;
    return ((unsigned __int128)qh << 64) | q1;
}

// ---------------------------------------------------------------------------
// Re-linearisation (Sec. 3.1 "LIV shuffle").  Modes that are adjacent and in
// the same relative order in both the old and the new order are merged into
// one "segment" on the host, so an order-N shuffle costs (segments - 1)
// divisions.  Segments are listed in old significance order (least
// significant first); seg_div[t] is the range of segment t and seg_stride[t]
// its stride in the new LIV.
// ---------------------------------------------------------------------------
struct RelinParams {
    int32_t nseg;
    int32_t identity;
    DivU64 seg_div[kMaxOrder];
    int64_t seg_stride[kMaxOrder];
    // every segment range and stride a power of two (every dimension is):
    // a segment is a bit field, moved by masks and shifts -- segment t is
    // bits [in_shift[t], in_shift[t] + width) of the old LIV (seg_mask[t] =
    // 2^width - 1) and lands at bit stride_shift[t] of the new one
    int32_t all_pow2;
    uint32_t stride_shift[kMaxOrder];
    uint32_t in_shift[kMaxOrder];
    uint64_t seg_mask[kMaxOrder];
};

__host__ __device__ __forceinline__ int64_t relin(const RelinParams &p, int64_t liv) {
    if (p.identity) return liv;
    if (p.all_pow2) {
        // independent fields (no chain through the remaining LIV); the loop
        // is unrolled so that every segment's constants are direct operands
        const uint64_t x = (uint64_t)liv;
        uint64_t out = 0;
#pragma unroll
        for (int t = 0; t < kMaxOrder; ++t) {
            if (t >= p.nseg) break;
            out |= ((x >> p.in_shift[t]) & p.seg_mask[t]) << p.stride_shift[t];
        }
        return (int64_t)out;
    }
    uint64_t r = (uint64_t)liv;
    int64_t out = 0;
#pragma unroll 1
    for (int t = 0; t < p.nseg - 1; ++t) {
        uint64_t q = divu(p.seg_div[t], r);
        uint64_t c = r - q * p.seg_div[t].d;
        out += (int64_t)c * p.seg_stride[t];
        r = q;
    }
    out += (int64_t)r * p.seg_stride[p.nseg - 1];
    return out;
}

// ---------------------------------------------------------------------------
// Workspace header (first 256 bytes of every workspace).
// ---------------------------------------------------------------------------
struct WsHeader {
    int32_t status;      // first device error (0 = none)
    int32_t alg;
    int64_t nnz_c;
    int64_t f;
    int64_t nzr_b;
    int64_t nchunks;
    int64_t work_total;
    int64_t nrows_l;         // non-empty rows of the left matrix operand
    uint32_t counters[32];   // tile/chunk counters and "last block" counters
};
static_assert(sizeof(WsHeader) <= kWsHeaderBytes, "header too large");

__device__ __forceinline__ void set_error(int32_t *status, int32_t err) {
    atomicCAS(status, 0, err);
}

// ---------------------------------------------------------------------------
// Decoupled look-back state words: [flag:2 | value:62].
// flag 0 = not yet published, 1 = aggregate of the tile only, 2 = inclusive
// prefix through the tile.
// ---------------------------------------------------------------------------
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ void lb_store(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t lb_load(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of the tiles before `tile` for one counter column; `state`
// is laid out [tile][stride].  Waits (bounded) for predecessors to publish.
// The predecessors' words are fetched kLookbackBatch at a time (independent
// loads in flight) and consumed nearest first until an inclusive prefix is met.
constexpr int kLookbackBatch = 8;

__device__ __forceinline__ uint64_t lookback(const uint64_t *state, int64_t tile, int64_t stride,
                                             int32_t *status, long long budget = kSpinBudgetCycles) {
    uint64_t excl = 0;
    const long long t0 = clock64();
    for (int64_t t = tile - 1; t >= 0; t -= kLookbackBatch) {
        uint64_t s[kLookbackBatch];
#pragma unroll
        for (int i = 0; i < kLookbackBatch; ++i) s[i] = t - i >= 0 ? lb_load(state + (t - i) * stride) : 0;
#pragma unroll
        for (int i = 0; i < kLookbackBatch; ++i) {
            if (t - i < 0) return excl;
            while ((s[i] >> 62) == 0) {
                if (clock64() - t0 > budget) {
                    set_error(status, LCO_ERR_TIMEOUT);
                    return excl;
                }
                __nanosleep(64);
                s[i] = lb_load(state + (t - i) * stride);
            }
            excl += s[i] & kValueMask;
            if ((s[i] >> 62) == 2) return excl;
        }
    }
    return excl;
}

// The same exclusive prefix computed by a whole warp (all 32 lanes must
// call it; every lane gets the result).  Each round fetches 32 x
// kLookbackBlocks predecessor words at once; the nearest inclusive word ends
// the walk.  A word that is needed but not yet published is re-read (bounded
// wait).  Positions before tile 0 count as an inclusive prefix of zero.
constexpr int kLookbackBlocks = 1;

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t lookback_warp(const uint64_t *state, int64_t tile, int32_t *status,
                                                  long long budget = kSpinBudgetCycles) {
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    const long long t0 = clock64();
    for (int64_t base = tile - 1; base >= 0; base -= 32 * kLookbackBlocks) {
        uint64_t w[kLookbackBlocks];
#pragma unroll
        for (int j = 0; j < kLookbackBlocks; ++j) {
            const int64_t idx = base - 32 * j - lane;
            w[j] = idx >= 0 ? lb_load(state + idx) : kFlagIncl;
        }
#pragma unroll
        for (int j = 0; j < kLookbackBlocks; ++j) {
            const int64_t idx = base - 32 * j - lane;
            for (;;) {
                const unsigned incl = __ballot_sync(0xffffffffu, (w[j] >> 62) == 2);
                const int first = incl ? __ffs(incl) - 1 : 31;
                const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
                const unsigned notready = __ballot_sync(0xffffffffu, (w[j] >> 62) == 0) & need;
                if (!notready) {
                    excl += warp_sum_u64(lane <= first ? (w[j] & kValueMask) : 0);
                    if (incl) return excl;
                    break;
                }
                // warp-uniform decision, so that all lanes leave together
                if (__any_sync(0xffffffffu, clock64() - t0 > budget)) {
                    if (lane == 0) set_error(status, LCO_ERR_TIMEOUT);
                    return excl;
                }
                // back off briefly so that spinning warps do not crowd the L2
                // lines their predecessors are about to publish to
                __nanosleep(64);
                if ((notready >> lane) & 1u) w[j] = lb_load(state + idx);
            }
        }
    }
    return excl;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, 1-D form) completing on a shared-memory
// mbarrier.  Addresses must be 16-byte aligned and sizes multiples of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity; false once the spin budget is
// spent (the caller records the error and leaves).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long budget = kSpinBudgetCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// NVTX range over a public entry point (visible in ncu/nsys timelines; a
// no-op when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Kernel timing / launch counting (implemented in lco_api.cu).
void timing_begin(const char *name, cudaStream_t s);
void timing_end(cudaStream_t s);

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched by launch_dependent() is
// scheduled while the kernel before it in the stream drains, instead of
// after that kernel has completed; its CTAs then wait in grid_dep_wait()
// until the predecessor has completed and its writes are visible.  Every
// kernel launched this way calls grid_dep_wait() before any other memory
// access, so that (by induction along the stream) it also sees the writes of
// every earlier operation.  launch_dependent() is used only where the
// operation before the launch in the stream is a kernel launch.  In a kernel
// launched normally the wait returns at once.  LCO_PDL=0 in the environment
// turns the programmatic launches into ordinary ones.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

inline bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("LCO_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lco

// Launch a kernel through the timing hooks: LCO_LAUNCH("name", stream, kernel<<<g, b, sm, stream>>>(args));
#define LCO_LAUNCH(name, stream, ...)        \
    do {                                     \
        ::lco::timing_begin((name), (stream)); \
        __VA_ARGS__;                         \
        ::lco::timing_end((stream));         \
    } while (0)

namespace lco {

}  // namespace lco
