// lco_radix.cuh -- stable LSD radix engine over (int64 LIV, double value) pairs.
//
// Used for the permutation of Sec. 4 (keys are re-linearised LIVs shaved by
// the resting suffix, Sec. 4.1) and for sorting product lists by output LIV
// (SOP, Sec. 5.2.5).  One launch reads the keys once and counts every
// pass's digits over the whole input; its last block turns the counts into
// the start of every digit's run in each pass's output and marks passes
// whose digit is the same for every element (those are skipped on the
// device).  A pass is then a single scatter launch: each CTA takes the next
// 2048-element tile in order, ranks it with warp match instructions,
// publishes its per-digit counts and finds the counts of the tiles before it
// by decoupled look-back, so that the tile's runs land at their final place
// without a separate counting or offset launch.  When two passes remain and
// every high-digit bucket fits one CTA, the high digit goes first and a
// local-sort launch orders each bucket by the low digit.
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

struct RadixJob {
    RelinParams relin;     // applied to source keys on first read (identity allowed)
    DivU64 key_div;        // key = relin(liv) div key_div
    int32_t D;             // digit bits
    int32_t P;             // passes
    int32_t G;             // counting CTAs (contiguous ranges of whole tiles), fixed from n_cap
    int32_t wide_lb;       // look-back words are 64-bit (capacity of 2^30 elements or more)
    int32_t lsd_only;      // never high digit first (a tuning choice)
    int64_t n_host;        // element count, or
    const int64_t *n_dev;  // device element count (overrides n_host when set)
    int64_t n_cap;         // upper bound on the element count (sizes grids and tables)
    const int64_t *src_liv;
    const double *src_val;
    int64_t *dst_liv;
    double *dst_val;
    int64_t *tmp_liv;
    double *tmp_val;
    // workspace pieces
    int32_t *active;               // [kMaxPasses] pass runs (digit not constant) + count at [16]
    unsigned long long *hist;      // [P][NB] digit counts over the input (cleared by radix_enqueue)
    unsigned long long *dstart;    // [P][NB] start of digit d's run in the output of pass p
    void *lb;                      // [2][tiles][NB] look-back words (two alternating regions)
    uint32_t *counters;            // header counters: [8] counting "last block", [12 + q] tiles of the q-th run pass
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

// Number of counting CTAs for up to n_cap elements.
int radix_ranges(int64_t n_cap);
// Bytes of workspace the engine needs for up to n_cap elements (excluding the
// header and excluding the tmp buffers when those are supplied elsewhere).
size_t radix_state_bytes(int64_t n_cap, int D, int P);
// Lays the engine's pieces out in `region` (which must hold
// radix_state_bytes bytes); counters/status live in the caller's header.
void radix_carve(RadixJob &job, char *region);
// Enqueues the counting launch and P scatter launches (and clears the digit
// counts before them).
cudaError_t radix_enqueue(const RadixJob &job, cudaStream_t stream);
// Leading bytes of a carved region that a caller may clear before a call
// (the pass flags; every call rewrites them, so clearing is optional).
size_t radix_hist_table_bytes();
int radix_sm_count();

}  // namespace lco
