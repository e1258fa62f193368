// lco_radix.cuh -- stable LSD radix engine over (int64 LIV, double value) pairs.
//
// Used for the permutation of Sec. 4 (keys are re-linearised LIVs shaved by
// the resting suffix, Sec. 4.1) and for sorting product lists by output LIV
// (SOP, Sec. 5.2.5).  The input's tiles are split into G contiguous ranges
// of whole tiles, one CTA each.  One launch reads the keys once and computes
// every pass's digit histogram per range, and marks passes whose digit is
// the same for every element (those are skipped on the device).  A pass is
// then: the start of every (digit, range) run in the output -- one exclusive
// scan over the digit-major count table -- and a scatter in which each CTA
// walks its range tile by tile, ranking each tile with warp match
// instructions and advancing running per-digit offsets, so no CTA waits on
// another.  Passes after the first one that runs histogram the intermediate
// buffer first.
#pragma once

#include "lco_internal.cuh"

namespace lco {

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kMaxDigitBits = 11;
// Default cap on the digit width.  A scatter tile holds 2048 elements; with
// 2^11 buckets a random key leaves about one element per bucket per tile and
// the scattered writes no longer coalesce (measured: an 11-bit pass cost 3x
// an 8-bit pass on 32-bit random keys), so wider digits only pay when they
// remove a pass and the keys are clustered.  A tuning hint may raise it.
#ifndef LCO_DEFAULT_DIGIT_BITS
#define LCO_DEFAULT_DIGIT_BITS 9
#endif
constexpr int kDefaultDigitBits = LCO_DEFAULT_DIGIT_BITS;   // a build may override it to measure others
constexpr int kMaxPasses = 6;
constexpr int kUpsweepCtasPerSm = 4;

struct RadixJob {
    RelinParams relin;     // applied to source keys on first read (identity allowed)
    DivU64 key_div;        // key = relin(liv) div key_div
    int32_t D;             // digit bits
    int32_t P;             // passes
    int32_t G;             // input ranges (one CTA each), fixed from n_cap
    int64_t n_host;        // element count, or
    const int64_t *n_dev;  // device element count (overrides n_host when set)
    int64_t n_cap;         // upper bound on the element count (sizes grids and tables)
    const int64_t *src_liv;
    const double *src_val;
    int64_t *dst_liv;
    double *dst_val;
    int64_t *tmp_liv;
    double *tmp_val;
    // workspace pieces (digit-major tables: entry [d][r] at d * G + r)
    int32_t *active;       // [kMaxPasses] pass runs (digit not constant) + count at [16]
    int32_t *cdig;         // [kMaxPasses][G] the one digit of a range, -1 several, -2 empty range
    uint32_t *counts_src;  // [P][NB][G] per-range counts over the source order
    uint32_t *counts_hist; // [NB][G] per-range counts before a later pass
    uint64_t *roffs;       // [NB][G] start of each (digit, range) run in the output of a pass
    uint64_t *scan_state;  // [kMaxPasses][scan tiles] look-back words of the offset scans
    uint32_t *counters;    // header counters: [8] upsweep "last block", [12 + p] scan tiles of pass p
    int32_t *status;
};

// Digit plan for a key range of `key_bits` bits, digits at most max_bits wide.
inline void radix_digits(int key_bits, int *D, int *P, int max_bits = kDefaultDigitBits) {
    if (max_bits < 1 || max_bits > kMaxDigitBits) max_bits = kDefaultDigitBits;
    if (key_bits <= 0) { *D = 1; *P = 1; return; }
    int p = (key_bits + max_bits - 1) / max_bits;
    if (p > kMaxPasses) p = kMaxPasses;
    int d = (key_bits + p - 1) / p;
    *D = d;
    *P = p;
}

// Number of input ranges for up to n_cap elements.
int radix_ranges(int64_t n_cap);
// Bytes of workspace the engine needs for up to n_cap elements (excluding the
// header and excluding the tmp buffers when those are supplied elsewhere).
size_t radix_state_bytes(int64_t n_cap, int D, int P);
// Lays the engine's pieces out in `region` (which must hold
// radix_state_bytes bytes); counters/status live in the caller's header.
void radix_carve(RadixJob &job, char *region);
// Enqueues the histogram launch and P scatter launches.
cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream);
// Bytes of the digit-histogram table at the start of a carved region.
size_t radix_hist_table_bytes();
int radix_sm_count();

}  // namespace lco
