// lco_host.h -- host-side planning shared by the permutation and contraction entry points.
#pragma once

#include <cuda_runtime.h>

#include "lco_internal.cuh"
#include "lco_radix.cuh"

namespace lco {

int32_t check_sig(int32_t order, const int32_t *sig);
// Validates order, sig and dims; *total receives the product of the dims.
int32_t check_shape(const lco_shape *t, int64_t *total);

// How a permutation of one tensor is carried out (Sec. 4.1).
struct RpPlan {
    lco_rp_info info;
    RelinParams relin;   // old LIV -> new LIV
    DivU64 key_div;      // key = newLIV div m_low
    int64_t total;       // product of dims
    int32_t identity;    // new order equals old order
    int32_t lsd_only;    // never high digit first (a tuning choice)
};

int32_t rp_plan(const lco_shape *t, const int32_t *new_sig, RpPlan *out, int max_digit_bits = kDefaultDigitBits);
// Bytes the radix engine needs for this plan on nnz elements (state + tmp buffers),
// excluding the workspace header.
size_t rp_region_bytes(const RpPlan &plan, int64_t nnz);
// Enqueues the permutation.  `region` holds rp_region_bytes bytes; `hdr` is
// the workspace header whose counters and status word the kernels use.
cudaError_t rp_enqueue(const RpPlan &plan, int64_t nnz, const int64_t *in_liv, const double *in_val,
                       int64_t *out_liv, double *out_val, char *region, WsHeader *hdr,
                       cudaStream_t stream);

// Re-linearisation parameters from old to new order (modes merged into
// segments when they stay adjacent and in the same relative order).
RelinParams make_relin(int32_t order, const int64_t *dims, const int32_t *sig_old,
                       const int32_t *sig_new);

cudaError_t relin_enqueue(const RelinParams &p, int64_t n, const int64_t *in, int64_t *out,
                          cudaStream_t stream);

// Zeroes the parts of a contraction workspace (sized for capacity `cap`,
// cap < 0: phase 1 only) that must start zeroed.
cudaError_t contract_ws_init(const lco_plan *p, void *ws, int64_t cap, cudaStream_t s);
// Bytes of the phase-1 region at the start of a contraction workspace.
size_t contract_phase1_bytes(const lco_plan *p);

// The matrix view a plan multiplies (row variants: L = A, R = B; column
// variants: L = B, R = A): L is mL x k, R is k x nR, and relin_l / relin_r
// map an operand's source LIV to its matrix-order LIV (row * k + column for
// L, row * nR + column for R).
struct PlanView {
    int32_t l_is_a, need_l, need_r, alg, lookup;
    int64_t mL, k, nR, nnz_l, nnz_r;
    RelinParams relin_l, relin_r;
};
void plan_view(const lco_plan *p, PlanView *v);

// L's row table of a contraction after its phase 1, in workspace `ws`:
// row_start[r] / row_work[r] are the first entry and the work prefix of
// L's r-th non-empty row (both with one closing element), row_id[r] its
// row index; the number of rows is the header's nrows_l.
void plan_row_table(const lco_plan *p, const void *ws, const int64_t **row_start, const int64_t **row_id,
                    const int64_t **row_work);

}  // namespace lco
