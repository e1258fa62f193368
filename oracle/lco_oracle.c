/*
 * lco_oracle.c -- CPU oracle for the LCO sparse-tensor hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of what the hot path computes, written from the paper
 * (Harrison & Joseph, "High Performance Rearrangement and Multiplication
 * Routines for Sparse Tensor Arithmetic").  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through seeded inputs made by the `synth` package.
 *
 * All index arithmetic is signed 64-bit (Sec. 3.1: LIVs are signed 64-bit
 * and the product of the dimensions stays below 2^63).  Values are IEEE
 * double.
 *
 * Functions and the passage each follows:
 *   lco_oracle_linearise / _delinearise  Sec. 3.1, the LIV formula
 *                                        LIV = i + n_i (j + n_j k) and
 *                                        Table 1.
 *   lco_oracle_relinearise               Sec. 3.1, "LIV shuffle".
 *   lco_oracle_permute                   Sec. 3.2 / Sec. 4: permutation is
 *                                        re-ordering sorted data into a new
 *                                        lexicographic order (definition:
 *                                        relinearise, then sort).
 *   lco_oracle_rp_classify               Sec. 4.1, Fig. 2: rearrangement vs
 *                                        resting indices.
 *   lco_oracle_rp_keyspec                Sec. 4.1: region size (the top
 *                                        resting prefix) and the divisor for
 *                                        the resting suffix.
 *   lco_oracle_rp_permute                Sec. 4.1: the RP algorithm --
 *                                        regions by linear scan, stable sort
 *                                        of each region on the shaved key.
 *   lco_oracle_contract                  Sec. 5 (eq. for a_ijkl x_kl and the
 *                                        inner/outer products of Sec. 5.2):
 *                                        C = sum over matched contracted
 *                                        coordinates of a * b (definition).
 *   lco_oracle_contract_ew               Sec. 5: the same with entrywise
 *                                        (shared, unsummed) mode pairs --
 *                                        one matrix product per value of the
 *                                        shared indices (definition).
 *   lco_oracle_dispatch                  Sec. 5.2, Table 4 and the ratio
 *                                        test dim/nnz > 3 (Secs. 5.2.3-5.2.5)
 *                                        with the n > m orientation rule of
 *                                        Sec. 5.2.2.
 *   lco_oracle_sort                      Sec. 3.2: sorting non-zeros into
 *                                        lexicographic (LIV) order
 *                                        (definition: stable sort by LIV).
 *   lco_oracle_add                       Sec. 3.2 / Fig. 3c: the sum of two
 *                                        tensors in one order, as in Eq. 4
 *                                        (definition: union of entries,
 *                                        values added).
 *   lco_oracle_relinearise_wide /        Sec. 3.1 and Sec. 7 (future work:
 *   lco_oracle_permute_wide /            LIVs past 2^63 - 1): the same LIV
 *   lco_oracle_contract_wide             formula and the same definitions of
 *                                        a permutation and a contraction,
 *                                        with unsigned 128-bit LIVs (dims
 *                                        multiply to at most 2^127 - 1); a
 *                                        wide LIV is two uint64 words, low
 *                                        word first.
 *
 * Parity pins for every function live under tests/ (test_oracle_*.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAX_ORDER 16

enum {
    ORC_OK = 0,
    ORC_ERR_INVALID = 1,
    ORC_ERR_OVERFLOW = 2,
    ORC_ERR_OOM = 4
};

/* ------------------------------------------------------------------ */
/* Validation helpers                                                  */
/* ------------------------------------------------------------------ */

/* Product of dims must stay <= 2^63 - 1 (Sec. 3.1). */
static int checked_product(int order, const int64_t *dims, int64_t *out)
{
    int64_t p = 1;
    for (int t = 0; t < order; ++t) {
        if (dims[t] < 1) return ORC_ERR_INVALID;
        if (p > INT64_MAX / dims[t]) return ORC_ERR_OVERFLOW;
        p *= dims[t];
    }
    *out = p;
    return ORC_OK;
}

/* sig must be a permutation of 0..order-1 */
static int valid_sig(int order, const int32_t *sig)
{
    int seen[ORC_MAX_ORDER] = {0};
    if (order < 1 || order > ORC_MAX_ORDER) return 0;
    for (int t = 0; t < order; ++t) {
        if (sig[t] < 0 || sig[t] >= order || seen[sig[t]]) return 0;
        seen[sig[t]] = 1;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: linearisation.  sig[0] is the least significant mode.    */
/* The LIV is built by Horner's rule from the most significant mode:  */
/* for sig {0,1,2} this is i + n_i (j + n_j k).                        */
/* ------------------------------------------------------------------ */

static int64_t linearise_one(int order, const int64_t *dims, const int32_t *sig,
                             const int64_t *coord)
{
    int64_t liv = 0;
    for (int t = order - 1; t >= 0; --t) {
        int mode = sig[t];
        liv = liv * dims[mode] + coord[mode];
    }
    return liv;
}

/* Peel the digits off least significant first with % and /. */
static void delinearise_one(int order, const int64_t *dims, const int32_t *sig,
                            int64_t liv, int64_t *coord)
{
    int64_t r = liv;
    for (int t = 0; t < order; ++t) {
        int mode = sig[t];
        coord[mode] = r % dims[mode];
        r = r / dims[mode];
    }
}

int lco_oracle_linearise(int32_t order, const int64_t *dims, const int32_t *sig,
                         int64_t nnz, const int64_t *coords, int64_t *liv)
{
    int64_t total;
    int rc;
    if (!valid_sig(order, sig)) return ORC_ERR_INVALID;
    if ((rc = checked_product(order, dims, &total)) != ORC_OK) return rc;
    for (int64_t e = 0; e < nnz; ++e) {
        const int64_t *c = coords + e * order;
        for (int t = 0; t < order; ++t)
            if (c[t] < 0 || c[t] >= dims[t]) return ORC_ERR_INVALID;
        liv[e] = linearise_one(order, dims, sig, c);
    }
    return ORC_OK;
}

int lco_oracle_delinearise(int32_t order, const int64_t *dims, const int32_t *sig,
                           int64_t nnz, const int64_t *liv, int64_t *coords)
{
    int64_t total;
    int rc;
    if (!valid_sig(order, sig)) return ORC_ERR_INVALID;
    if ((rc = checked_product(order, dims, &total)) != ORC_OK) return rc;
    for (int64_t e = 0; e < nnz; ++e) {
        if (liv[e] < 0 || liv[e] >= total) return ORC_ERR_INVALID;
        delinearise_one(order, dims, sig, liv[e], coords + e * order);
    }
    return ORC_OK;
}

/* Sec. 3.1, "LIV shuffle": recompute every LIV for a new lexicographic
 * order by decomposing it into coordinates and recomposing them. */
int lco_oracle_relinearise(int32_t order, const int64_t *dims, const int32_t *sig_old,
                           const int32_t *sig_new, int64_t nnz, const int64_t *liv_in,
                           int64_t *liv_out)
{
    int64_t total;
    int rc;
    int64_t coord[ORC_MAX_ORDER];
    if (!valid_sig(order, sig_old) || !valid_sig(order, sig_new)) return ORC_ERR_INVALID;
    if ((rc = checked_product(order, dims, &total)) != ORC_OK) return rc;
    for (int64_t e = 0; e < nnz; ++e) {
        if (liv_in[e] < 0 || liv_in[e] >= total) return ORC_ERR_INVALID;
        delinearise_one(order, dims, sig_old, liv_in[e], coord);
        liv_out[e] = linearise_one(order, dims, sig_new, coord);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Permutation by definition: relinearise, then sort by the new LIV.  */
/* LIVs of a valid tensor are distinct, so the sort order is unique.  */
/* ------------------------------------------------------------------ */

typedef struct { int64_t key; int64_t idx; } keyidx_t;

static int cmp_keyidx(const void *pa, const void *pb)
{
    const keyidx_t *a = (const keyidx_t *)pa, *b = (const keyidx_t *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->idx < b->idx) return -1;   /* ties broken by input position: stable */
    if (a->idx > b->idx) return 1;
    return 0;
}

int lco_oracle_permute(int32_t order, const int64_t *dims, const int32_t *sig_old,
                       const int32_t *sig_new, int64_t nnz, const int64_t *liv_in,
                       const double *val_in, int64_t *liv_out, double *val_out)
{
    int rc;
    int64_t *newliv;
    keyidx_t *ki;
    if (nnz == 0) return valid_sig(order, sig_old) && valid_sig(order, sig_new) ? ORC_OK : ORC_ERR_INVALID;
    newliv = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    ki = (keyidx_t *)malloc(sizeof(keyidx_t) * (size_t)nnz);
    if (!newliv || !ki) { free(newliv); free(ki); return ORC_ERR_OOM; }
    rc = lco_oracle_relinearise(order, dims, sig_old, sig_new, nnz, liv_in, newliv);
    if (rc != ORC_OK) { free(newliv); free(ki); return rc; }
    for (int64_t e = 0; e < nnz; ++e) { ki[e].key = newliv[e]; ki[e].idx = e; }
    qsort(ki, (size_t)nnz, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t e = 0; e < nnz; ++e) {
        liv_out[e] = ki[e].key;
        val_out[e] = val_in[ki[e].idx];
    }
    free(newliv);
    free(ki);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1: RP index classification.                                  */
/* An index is a rearrangement index when, going from the old to the   */
/* new order, it moves above an index that used to be more significant */
/* than it (its edge crosses that index's edge in Fig. 2).  All other  */
/* indices are resting.  is_rearr[mode] receives 1 or 0.               */
/* ------------------------------------------------------------------ */

int lco_oracle_rp_classify(int32_t order, const int32_t *sig_old, const int32_t *sig_new,
                           int32_t *is_rearr)
{
    int pos_old[ORC_MAX_ORDER], pos_new[ORC_MAX_ORDER];
    if (!valid_sig(order, sig_old) || !valid_sig(order, sig_new)) return ORC_ERR_INVALID;
    /* position = significance rank, 0 = least significant */
    for (int t = 0; t < order; ++t) { pos_old[sig_old[t]] = t; pos_new[sig_new[t]] = t; }
    for (int x = 0; x < order; ++x) {
        int r = 0;
        for (int y = 0; y < order; ++y) {
            if (y == x) continue;
            /* y was more significant than x, and is now less significant */
            if (pos_old[y] > pos_old[x] && pos_new[y] < pos_new[x]) r = 1;
        }
        is_rearr[x] = r;
    }
    return ORC_OK;
}

/* Sec. 4.1: the shaving parameters.  Working down the new order from its
 * most significant index, the leading resting indices split the data into
 * independent regions; m_top is the number of index values in one region
 * (the product of the dims below that prefix; 30 in Fig. 2).  The resting
 * indices below the lowest rearrangement index need no sorting; m_low is
 * the product of their dims (3 in Fig. 2).  The shaved key of an element is
 * (newLIV mod m_top) div m_low.  n_rearr receives the number of
 * rearrangement indices (0 means the new order needs no data movement). */
int lco_oracle_rp_keyspec(int32_t order, const int64_t *dims, const int32_t *sig_old,
                          const int32_t *sig_new, int64_t *m_top, int64_t *m_low,
                          int32_t *n_rearr)
{
    int32_t rearr[ORC_MAX_ORDER];
    int64_t total;
    int rc, t, lowest = -1, nr = 0;
    if ((rc = lco_oracle_rp_classify(order, sig_old, sig_new, rearr)) != ORC_OK) return rc;
    if ((rc = checked_product(order, dims, &total)) != ORC_OK) return rc;
    /* lowest rearrangement index in the new order (smallest significance) */
    for (t = 0; t < order; ++t) {
        if (rearr[sig_new[t]]) { if (lowest < 0) lowest = t; ++nr; }
    }
    *n_rearr = nr;
    if (nr == 0) { *m_top = total; *m_low = total; return ORC_OK; }
    /* resting suffix below the lowest rearrangement index */
    {
        int64_t p = 1;
        for (t = 0; t < lowest; ++t) p *= dims[sig_new[t]];
        *m_low = p;
    }
    /* leading resting indices of the new order, from the top down */
    {
        int64_t p = total;
        for (t = order - 1; t >= 0; --t) {
            if (rearr[sig_new[t]]) break;
            p /= dims[sig_new[t]];
        }
        *m_top = p;
    }
    return ORC_OK;
}

/* Sec. 4.1, the RP algorithm, in the paper's steps:
 *  1. recompute the LIVs in the new order;
 *  2. find the regions where the leading resting indices are constant by a
 *     linear scan against the largest LIV of the current region;
 *  3. stably sort each region on the shaved key (newLIV mod m_top) div m_low.
 * Stability (ties kept in input order) supplies the resting suffix. */
int lco_oracle_rp_permute(int32_t order, const int64_t *dims, const int32_t *sig_old,
                          const int32_t *sig_new, int64_t nnz, const int64_t *liv_in,
                          const double *val_in, int64_t *liv_out, double *val_out)
{
    int64_t m_top, m_low;
    int32_t nr;
    int rc;
    int64_t *newliv;
    keyidx_t *ki;
    if ((rc = lco_oracle_rp_keyspec(order, dims, sig_old, sig_new, &m_top, &m_low, &nr)) != ORC_OK)
        return rc;
    if (nnz == 0) return ORC_OK;
    newliv = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    ki = (keyidx_t *)malloc(sizeof(keyidx_t) * (size_t)nnz);
    if (!newliv || !ki) { free(newliv); free(ki); return ORC_ERR_OOM; }
    rc = lco_oracle_relinearise(order, dims, sig_old, sig_new, nnz, liv_in, newliv);
    if (rc != ORC_OK) { free(newliv); free(ki); return rc; }
    if (nr == 0) {
        for (int64_t e = 0; e < nnz; ++e) { liv_out[e] = newliv[e]; val_out[e] = val_in[e]; }
        free(newliv); free(ki);
        return ORC_OK;
    }
    {
        int64_t start = 0;
        while (start < nnz) {
            /* region of constant leading resting indices: the region value is
             * newLIV div m_top; its largest possible LIV bounds the scan. */
            int64_t region = newliv[start] / m_top;
            int64_t max_liv = region * m_top + (m_top - 1);
            int64_t end = start;
            while (end < nnz && newliv[end] <= max_liv && newliv[end] >= region * m_top) ++end;
            for (int64_t e = start; e < end; ++e) {
                ki[e - start].key = (newliv[e] % m_top) / m_low;
                ki[e - start].idx = e;
            }
            /* qsort with the input position as a tie-break is a stable sort */
            qsort(ki, (size_t)(end - start), sizeof(keyidx_t), cmp_keyidx);
            for (int64_t e = start; e < end; ++e) {
                int64_t src = ki[e - start].idx;
                liv_out[e] = newliv[src];
                val_out[e] = val_in[src];
            }
            start = end;
        }
    }
    free(newliv);
    free(ki);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Contraction by definition (Sec. 2 Einstein notation; Sec. 5).        */
/*                                                                     */
/*   C[f_A, f_B] = sum over matched contracted coordinates of a * b    */
/*                                                                     */
/* C's modes are A's free modes in increasing mode number followed by  */
/* B's free modes in increasing mode number; C is returned row-major    */
/* (its last mode least significant).  Every (f_A, f_B) that receives   */
/* at least one product is an entry of C, even when its sum is zero.    */
/* abs_c[e] is the sum of |a||b| over the products of entry e.          */
/* ------------------------------------------------------------------ */

typedef struct { int64_t key; int64_t liv; int64_t idx; } bent_t;   /* B entry, sortable */
typedef struct { int64_t out; int64_t seq; double v; double a; } prod_t;

static int cmp_bent(const void *pa, const void *pb)
{
    const bent_t *a = (const bent_t *)pa, *b = (const bent_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->liv != b->liv) return a->liv < b->liv ? -1 : 1;
    return 0;
}

static int cmp_prod(const void *pa, const void *pb)
{
    const prod_t *a = (const prod_t *)pa, *b = (const prod_t *)pb;
    if (a->out != b->out) return a->out < b->out ? -1 : 1;
    if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
    return 0;
}

static int cmp_i64(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* The contraction with entrywise mode pairs (emodes_a[t], emodes_b[t]):
 * shared indices that are neither summed nor dropped (Sec. 5: entrywise
 * products map the tensor product to repeated matrix products, one per
 * value of the shared indices).  By definition:
 *   C[h, free_a, free_b] = sum_k A[h, free_a, k] B[h, k, free_b]
 * with C's modes ordered entrywise pairs (pairing order), then A's free
 * modes, then B's free modes, row-major.  nentry = 0 is the plain
 * contraction. */
int lco_oracle_contract_ew(int32_t order_a, const int64_t *dims_a, const int32_t *sig_a,
                           int64_t nnz_a, const int64_t *liv_a, const double *val_a,
                           int32_t order_b, const int64_t *dims_b, const int32_t *sig_b,
                           int64_t nnz_b, const int64_t *liv_b, const double *val_b,
                           int32_t ncontract, const int32_t *modes_a, const int32_t *modes_b,
                           int32_t nentry, const int32_t *emodes_a, const int32_t *emodes_b,
                           int64_t *nnz_c, int64_t **liv_c, double **val_c, double **abs_c)
{
    int is_con_a[ORC_MAX_ORDER] = {0}, is_con_b[ORC_MAX_ORDER] = {0};
    int64_t tot_a, tot_b, m = 1, n = 1, hsz = 1;
    int64_t coord[ORC_MAX_ORDER];
    int rc;
    bent_t *bs = NULL;
    int64_t *order_idx_a = NULL;
    prod_t *prods = NULL;
    int64_t nprod = 0, cap = 0;

    *nnz_c = 0; *liv_c = NULL; *val_c = NULL; *abs_c = NULL;
    if (!valid_sig(order_a, sig_a) || !valid_sig(order_b, sig_b)) return ORC_ERR_INVALID;
    if ((rc = checked_product(order_a, dims_a, &tot_a)) != ORC_OK) return rc;
    if ((rc = checked_product(order_b, dims_b, &tot_b)) != ORC_OK) return rc;
    if (ncontract < 0 || ncontract > order_a || ncontract > order_b) return ORC_ERR_INVALID;
    for (int c = 0; c < ncontract; ++c) {
        int ma = modes_a[c], mb = modes_b[c];
        if (ma < 0 || ma >= order_a || mb < 0 || mb >= order_b) return ORC_ERR_INVALID;
        if (is_con_a[ma] || is_con_b[mb]) return ORC_ERR_INVALID;
        if (dims_a[ma] != dims_b[mb]) return ORC_ERR_INVALID;
        is_con_a[ma] = 1; is_con_b[mb] = 1;
    }
    if (nentry < 0 || ncontract + nentry > order_a || ncontract + nentry > order_b) return ORC_ERR_INVALID;
    for (int c = 0; c < nentry; ++c) {
        int ma = emodes_a[c], mb = emodes_b[c];
        if (ma < 0 || ma >= order_a || mb < 0 || mb >= order_b) return ORC_ERR_INVALID;
        if (is_con_a[ma] || is_con_b[mb]) return ORC_ERR_INVALID;
        if (dims_a[ma] != dims_b[mb]) return ORC_ERR_INVALID;
        is_con_a[ma] = 2; is_con_b[mb] = 2;   /* 2: entrywise */
        if (hsz > INT64_MAX / dims_a[ma]) return ORC_ERR_OVERFLOW;
        hsz *= dims_a[ma];
    }
    if (nentry + (order_a - ncontract - nentry) + (order_b - ncontract - nentry) > ORC_MAX_ORDER)
        return ORC_ERR_INVALID;
    for (int t = 0; t < order_a; ++t) if (!is_con_a[t]) {
        if (m > INT64_MAX / dims_a[t]) return ORC_ERR_OVERFLOW;
        m *= dims_a[t];
    }
    for (int t = 0; t < order_b; ++t) if (!is_con_b[t]) {
        if (n > INT64_MAX / dims_b[t]) return ORC_ERR_OVERFLOW;
        n *= dims_b[t];
    }
    if (m > INT64_MAX / n || hsz > INT64_MAX / (m * n)) return ORC_ERR_OVERFLOW;
    if (nnz_a == 0 || nnz_b == 0) return ORC_OK;

    /* B entries keyed by their entrywise, then contracted coordinates
     * (pairing order, the first pair most significant), then by B's own
     * LIV. */
    bs = (bent_t *)malloc(sizeof(bent_t) * (size_t)nnz_b);
    order_idx_a = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)nnz_a);
    if (!bs || !order_idx_a) { rc = ORC_ERR_OOM; goto done; }
    for (int64_t e = 0; e < nnz_b; ++e) {
        int64_t key = 0;
        if (liv_b[e] < 0 || liv_b[e] >= tot_b) { rc = ORC_ERR_INVALID; goto done; }
        delinearise_one(order_b, dims_b, sig_b, liv_b[e], coord);
        for (int c = 0; c < nentry; ++c) key = key * dims_b[emodes_b[c]] + coord[emodes_b[c]];
        for (int c = 0; c < ncontract; ++c) key = key * dims_b[modes_b[c]] + coord[modes_b[c]];
        bs[e].key = key; bs[e].liv = liv_b[e]; bs[e].idx = e;
    }
    qsort(bs, (size_t)nnz_b, sizeof(bent_t), cmp_bent);

    /* A entries visited in ascending A-LIV order */
    for (int64_t e = 0; e < nnz_a; ++e) {
        if (liv_a[e] < 0 || liv_a[e] >= tot_a) { rc = ORC_ERR_INVALID; goto done; }
        order_idx_a[2 * e] = liv_a[e];
        order_idx_a[2 * e + 1] = e;
    }
    qsort(order_idx_a, (size_t)nnz_a, 2 * sizeof(int64_t), cmp_i64);

    for (int64_t q = 0; q < nnz_a; ++q) {
        int64_t e = order_idx_a[2 * q + 1];
        int64_t key = 0, row = 0, h = 0;
        int64_t lo, hi;
        delinearise_one(order_a, dims_a, sig_a, liv_a[e], coord);
        for (int c = 0; c < nentry; ++c) h = h * dims_a[emodes_a[c]] + coord[emodes_a[c]];
        key = h;
        for (int c = 0; c < ncontract; ++c) key = key * dims_a[modes_a[c]] + coord[modes_a[c]];
        for (int t = 0; t < order_a; ++t) if (!is_con_a[t]) row = row * dims_a[t] + coord[t];
        row += h * m;
        /* first B entry with this key (binary search) */
        lo = 0; hi = nnz_b;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (bs[mid].key < key) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < nnz_b && bs[j].key == key; ++j) {
            int64_t cb[ORC_MAX_ORDER];
            int64_t col = 0;
            double av = val_a[e], bv = val_b[bs[j].idx];
            delinearise_one(order_b, dims_b, sig_b, bs[j].liv, cb);
            for (int t = 0; t < order_b; ++t) if (!is_con_b[t]) col = col * dims_b[t] + cb[t];
            if (nprod == cap) {
                int64_t ncap = cap ? cap * 2 : 1024;
                prod_t *np = (prod_t *)realloc(prods, sizeof(prod_t) * (size_t)ncap);
                if (!np) { rc = ORC_ERR_OOM; goto done; }
                prods = np; cap = ncap;
            }
            prods[nprod].out = row * n + col;
            prods[nprod].seq = nprod;
            prods[nprod].v = av * bv;
            prods[nprod].a = fabs(av) * fabs(bv);
            ++nprod;
        }
    }

    /* sum equal output LIVs in generation order */
    qsort(prods, (size_t)nprod, sizeof(prod_t), cmp_prod);
    {
        int64_t nc = 0;
        for (int64_t i = 0; i < nprod; ++i)
            if (i == 0 || prods[i].out != prods[i - 1].out) ++nc;
        *liv_c = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc ? nc : 1));
        *val_c = (double *)malloc(sizeof(double) * (size_t)(nc ? nc : 1));
        *abs_c = (double *)malloc(sizeof(double) * (size_t)(nc ? nc : 1));
        if (!*liv_c || !*val_c || !*abs_c) { rc = ORC_ERR_OOM; goto done; }
        nc = -1;
        for (int64_t i = 0; i < nprod; ++i) {
            if (i == 0 || prods[i].out != prods[i - 1].out) {
                ++nc;
                (*liv_c)[nc] = prods[i].out;
                (*val_c)[nc] = 0.0;
                (*abs_c)[nc] = 0.0;
            }
            (*val_c)[nc] += prods[i].v;
            (*abs_c)[nc] += prods[i].a;
        }
        *nnz_c = nc + 1;
    }
    rc = ORC_OK;
done:
    if (rc != ORC_OK) {
        free(*liv_c); free(*val_c); free(*abs_c);
        *liv_c = NULL; *val_c = NULL; *abs_c = NULL; *nnz_c = 0;
    }
    free(bs);
    free(order_idx_a);
    free(prods);
    return rc;
}

int lco_oracle_contract(int32_t order_a, const int64_t *dims_a, const int32_t *sig_a,
                        int64_t nnz_a, const int64_t *liv_a, const double *val_a,
                        int32_t order_b, const int64_t *dims_b, const int32_t *sig_b,
                        int64_t nnz_b, const int64_t *liv_b, const double *val_b,
                        int32_t ncontract, const int32_t *modes_a, const int32_t *modes_b,
                        int64_t *nnz_c, int64_t **liv_c, double **val_c, double **abs_c)
{
    return lco_oracle_contract_ew(order_a, dims_a, sig_a, nnz_a, liv_a, val_a, order_b, dims_b, sig_b, nnz_b,
                                  liv_b, val_b, ncontract, modes_a, modes_b, 0, NULL, NULL, nnz_c, liv_c, val_c,
                                  abs_c);
}

/* Number of products f = sum over A entries of the matching B entries
 * (Sec. 5.2, the flop count f), by the same bucketing as the contraction. */
int lco_oracle_flops(int32_t order_a, const int64_t *dims_a, const int32_t *sig_a,
                     int64_t nnz_a, const int64_t *liv_a,
                     int32_t order_b, const int64_t *dims_b, const int32_t *sig_b,
                     int64_t nnz_b, const int64_t *liv_b,
                     int32_t ncontract, const int32_t *modes_a, const int32_t *modes_b,
                     int64_t *f)
{
    int64_t coord[ORC_MAX_ORDER];
    int64_t *kb;
    int64_t total = 0;
    if (!valid_sig(order_a, sig_a) || !valid_sig(order_b, sig_b)) return ORC_ERR_INVALID;
    *f = 0;
    if (nnz_a == 0 || nnz_b == 0) return ORC_OK;
    kb = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz_b);
    if (!kb) return ORC_ERR_OOM;
    for (int64_t e = 0; e < nnz_b; ++e) {
        int64_t key = 0;
        delinearise_one(order_b, dims_b, sig_b, liv_b[e], coord);
        for (int c = 0; c < ncontract; ++c) key = key * dims_b[modes_b[c]] + coord[modes_b[c]];
        kb[e] = key;
    }
    qsort(kb, (size_t)nnz_b, sizeof(int64_t), cmp_i64);
    for (int64_t e = 0; e < nnz_a; ++e) {
        int64_t key = 0, lo = 0, hi = nnz_b, lo2;
        delinearise_one(order_a, dims_a, sig_a, liv_a[e], coord);
        for (int c = 0; c < ncontract; ++c) key = key * dims_a[modes_a[c]] + coord[modes_a[c]];
        while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (kb[mid] < key) lo = mid + 1; else hi = mid; }
        lo2 = lo; hi = nnz_b;
        while (lo2 < hi) { int64_t mid = lo2 + (hi - lo2) / 2; if (kb[mid] <= key) lo2 = mid + 1; else hi = mid; }
        total += lo2 - lo;
    }
    free(kb);
    *f = total;
    return ORC_OK;
}

void lco_oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* Sorting and addition (Sec. 3.2; Fig. 3c and the sum of Eq. 4).      */
/* ------------------------------------------------------------------ */

/* Sorting by definition: the entries in ascending LIV order; equal LIVs
 * keep their input order (a stable sort on (LIV, input position)).  The
 * order is unchanged; only the entries move. */
int lco_oracle_sort(int64_t nnz, const int64_t *liv, const double *val, int64_t *liv_out, double *val_out)
{
    if (nnz < 0) return ORC_ERR_INVALID;
    if (nnz == 0) return ORC_OK;
    int64_t (*ki)[2] = malloc((size_t)nnz * sizeof *ki);
    if (!ki) return ORC_ERR_OOM;
    for (int64_t e = 0; e < nnz; ++e) {
        ki[e][0] = liv[e];
        ki[e][1] = e;
    }
    qsort(ki, (size_t)nnz, sizeof *ki, cmp_keyidx);
    for (int64_t e = 0; e < nnz; ++e) {
        liv_out[e] = ki[e][0];
        val_out[e] = val[ki[e][1]];
    }
    free(ki);
    return ORC_OK;
}

/* C = alpha A + beta B by definition, for two sorted LCO tensors in the
 * same order: every LIV of A or B is an entry of C (structural entries are
 * kept even when the sum is zero); an LIV present in both gets
 * alpha a + beta b, one present in one only gets its scaled value.  Output
 * ascending; returns the entry count in *nnz_c (c arrays must hold
 * nnz_a + nnz_b). */
int lco_oracle_add(double alpha, int64_t nnz_a, const int64_t *a_liv, const double *a_val,
                   double beta, int64_t nnz_b, const int64_t *b_liv, const double *b_val,
                   int64_t *c_liv, double *c_val, int64_t *nnz_c)
{
    if (nnz_a < 0 || nnz_b < 0 || !nnz_c) return ORC_ERR_INVALID;
    int64_t i = 0, j = 0, o = 0;
    while (i < nnz_a || j < nnz_b) {
        if (j >= nnz_b || (i < nnz_a && a_liv[i] < b_liv[j])) {
            c_liv[o] = a_liv[i];
            c_val[o] = alpha * a_val[i];
            ++i;
        } else if (i >= nnz_a || b_liv[j] < a_liv[i]) {
            c_liv[o] = b_liv[j];
            c_val[o] = beta * b_val[j];
            ++j;
        } else {
            const double pa = alpha * a_val[i];
            const double pb = beta * b_val[j];
            c_liv[o] = a_liv[i];
            c_val[o] = pa + pb;
            ++i;
            ++j;
        }
        ++o;
    }
    *nnz_c = o;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 5.2, Table 4: the poly-algorithm's choice.                     */
/*                                                                     */
/* Hyper-sparsity test (Sec. 5.2, "measuring the ratio"): a dimension   */
/* is hyper-sparse when dim / nnz > 3 (the switch-over used in Secs.    */
/* 5.2.3-5.2.5).  A is row-sparse when m/nnz_A > 3 and column-sparse     */
/* when k/nnz_A > 3; B is row-sparse when k/nnz_B > 3 and column-sparse */
/* when n/nnz_B > 3.  Class: 0 sparse, 1 row-sparse, 2 column-sparse,    */
/* 3 index-sparse (both).                                               */
/*                                                                     */
/* Algorithms: 0 CSR, 1 CSC, 2 DCSR, 3 DCSC, 4 CSRNA, 5 CSCNA, 6 SOP.  */
/*                                                                     */
/* Where a cell names a pair ("CSC/CSR"), the variant needing fewer     */
/* operand rearrangements wins; with a tie the column variant is chosen */
/* when n > m and the row variant otherwise (Sec. 5.2.2).               */
/* perm_row / perm_col: number of operands (0..2) that would need a     */
/* permutation for the row / column variant.                            */
/* ------------------------------------------------------------------ */

enum { ALG_CSR = 0, ALG_CSC = 1, ALG_DCSR = 2, ALG_DCSC = 3, ALG_CSRNA = 4, ALG_CSCNA = 5, ALG_SOP = 6,
       CELL_CSC_CSR = 10, CELL_DCSC_DCSR = 11, CELL_CSCNA_CSRNA = 12 };

/* rows: class of A; columns: class of B; order S, R, C, I */
static const int table4[4][4] = {
    /* A sparse        */ { CELL_CSC_CSR, ALG_CSC,        ALG_CSC,          ALG_CSC   },
    /* A row-sparse    */ { ALG_CSR,      ALG_DCSR,       CELL_CSCNA_CSRNA, ALG_CSCNA },
    /* A column-sparse */ { ALG_CSR,      CELL_DCSC_DCSR, ALG_DCSC,         ALG_DCSC  },
    /* A index-sparse  */ { ALG_CSR,      ALG_DCSR,       ALG_CSRNA,        ALG_SOP   },
};

static int sparsity_class(int64_t rows, int64_t cols, int64_t nnz)
{
    int rs, cs;
    if (nnz <= 0) return 3;
    rs = ((double)rows / (double)nnz) > 3.0;
    cs = ((double)cols / (double)nnz) > 3.0;
    return rs && cs ? 3 : (rs ? 1 : (cs ? 2 : 0));
}

int lco_oracle_sparsity_class(int64_t rows, int64_t cols, int64_t nnz)
{
    return sparsity_class(rows, cols, nnz);
}

int lco_oracle_dispatch(int64_t m, int64_t k, int64_t n, int64_t nnz_a, int64_t nnz_b,
                        int32_t perm_row, int32_t perm_col)
{
    int ca = sparsity_class(m, k, nnz_a);
    int cb = sparsity_class(k, n, nnz_b);
    int cell = table4[ca][cb];
    int col;
    if (cell < 10) return cell;
    if (perm_col < perm_row) col = 1;
    else if (perm_row < perm_col) col = 0;
    else col = n > m;
    switch (cell) {
    case CELL_CSC_CSR: return col ? ALG_CSC : ALG_CSR;
    case CELL_DCSC_DCSR: return col ? ALG_DCSC : ALG_DCSR;
    default: return col ? ALG_CSCNA : ALG_CSRNA;
    }
}

/* ------------------------------------------------------------------ */
/* Wide LIVs (Sec. 3.1 leaves LIVs past 2^63 - 1 to future work;        */
/* Sec. 7).  Same formula and same permutation definition as above in   */
/* unsigned 128-bit arithmetic; the dims multiply to at most 2^127 - 1. */
/* ------------------------------------------------------------------ */

typedef unsigned __int128 u128_t;

static int checked_product_wide(int order, const int64_t *dims, u128_t *out)
{
    const u128_t lim = ((u128_t)1 << 127) - 1;
    u128_t p = 1;
    if (order < 1 || order > ORC_MAX_ORDER) return ORC_ERR_INVALID;
    for (int i = 0; i < order; ++i) {
        if (dims[i] < 1) return ORC_ERR_INVALID;
        if (p > lim / (u128_t)dims[i]) return ORC_ERR_OVERFLOW;
        p *= (u128_t)dims[i];
    }
    *out = p;
    return ORC_OK;
}

int lco_oracle_relinearise_wide(int32_t order, const int64_t *dims, const int32_t *sig_old,
                                const int32_t *sig_new, int64_t nnz, const uint64_t *liv_in,
                                uint64_t *liv_out)
{
    u128_t total;
    int rc;
    u128_t coord[ORC_MAX_ORDER];
    if (!valid_sig(order, sig_old) || !valid_sig(order, sig_new)) return ORC_ERR_INVALID;
    if ((rc = checked_product_wide(order, dims, &total)) != ORC_OK) return rc;
    for (int64_t e = 0; e < nnz; ++e) {
        u128_t r = ((u128_t)liv_in[2 * e + 1] << 64) | liv_in[2 * e];
        u128_t out = 0;
        if (r >= total) return ORC_ERR_INVALID;
        /* coordinates: least significant mode of the old order first */
        for (int t = 0; t < order; ++t) {
            const u128_t n = (u128_t)dims[sig_old[t]];
            coord[sig_old[t]] = r % n;
            r /= n;
        }
        /* Horner from the most significant mode of the new order */
        for (int t = order - 1; t >= 0; --t) out = out * (u128_t)dims[sig_new[t]] + coord[sig_new[t]];
        liv_out[2 * e] = (uint64_t)out;
        liv_out[2 * e + 1] = (uint64_t)(out >> 64);
    }
    return ORC_OK;
}

typedef struct { u128_t key; int64_t idx; } wideidx_t;

static int cmp_wideidx(const void *pa, const void *pb)
{
    const wideidx_t *a = (const wideidx_t *)pa, *b = (const wideidx_t *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

int lco_oracle_permute_wide(int32_t order, const int64_t *dims, const int32_t *sig_old,
                            const int32_t *sig_new, int64_t nnz, const uint64_t *liv_in,
                            const double *val_in, uint64_t *liv_out, double *val_out)
{
    int rc;
    uint64_t *newliv;
    wideidx_t *ki;
    if (nnz == 0) {
        u128_t total;
        if (!valid_sig(order, sig_old) || !valid_sig(order, sig_new)) return ORC_ERR_INVALID;
        return checked_product_wide(order, dims, &total);
    }
    newliv = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)nnz);
    ki = (wideidx_t *)malloc(sizeof(wideidx_t) * (size_t)nnz);
    if (!newliv || !ki) { free(newliv); free(ki); return ORC_ERR_OOM; }
    rc = lco_oracle_relinearise_wide(order, dims, sig_old, sig_new, nnz, liv_in, newliv);
    if (rc != ORC_OK) { free(newliv); free(ki); return rc; }
    for (int64_t e = 0; e < nnz; ++e) {
        ki[e].key = ((u128_t)newliv[2 * e + 1] << 64) | newliv[2 * e];
        ki[e].idx = e;
    }
    qsort(ki, (size_t)nnz, sizeof(wideidx_t), cmp_wideidx);
    for (int64_t e = 0; e < nnz; ++e) {
        liv_out[2 * e] = (uint64_t)ki[e].key;
        liv_out[2 * e + 1] = (uint64_t)(ki[e].key >> 64);
        val_out[e] = val_in[ki[e].idx];
    }
    free(newliv);
    free(ki);
    return ORC_OK;
}

/* Contraction by definition with wide LIVs (no entrywise modes): C's modes
 * are A's free modes then B's free modes, row-major, and C's LIV range
 * (the product of those dims) must stay within 2^127 - 1.  Products are
 * summed per output LIV in generation order (A entries in ascending LIV
 * order, then B entries of the matching key in ascending LIV order).
 * liv_c receives 2 * nnz_c words. */
typedef struct { u128_t key; u128_t liv; int64_t idx; } wbent_t;
typedef struct { u128_t out; int64_t seq; double v; double a; } wprod_t;
typedef struct { u128_t liv; int64_t idx; } wa_t;

static int cmp_wbent(const void *pa, const void *pb)
{
    const wbent_t *a = (const wbent_t *)pa, *b = (const wbent_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->liv != b->liv) return a->liv < b->liv ? -1 : 1;
    return 0;
}

static int cmp_wprod(const void *pa, const void *pb)
{
    const wprod_t *a = (const wprod_t *)pa, *b = (const wprod_t *)pb;
    if (a->out != b->out) return a->out < b->out ? -1 : 1;
    if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
    return 0;
}

static int cmp_wa(const void *pa, const void *pb)
{
    const wa_t *a = (const wa_t *)pa, *b = (const wa_t *)pb;
    if (a->liv != b->liv) return a->liv < b->liv ? -1 : 1;
    return 0;
}

static void wide_coords(int order, const int64_t *dims, const int32_t *sig, u128_t liv, u128_t *coord)
{
    for (int t = 0; t < order; ++t) {
        const u128_t d = (u128_t)dims[sig[t]];
        coord[sig[t]] = liv % d;
        liv /= d;
    }
}

int lco_oracle_contract_wide(int32_t order_a, const int64_t *dims_a, const int32_t *sig_a,
                             int64_t nnz_a, const uint64_t *liv_a, const double *val_a,
                             int32_t order_b, const int64_t *dims_b, const int32_t *sig_b,
                             int64_t nnz_b, const uint64_t *liv_b, const double *val_b,
                             int32_t ncontract, const int32_t *modes_a, const int32_t *modes_b,
                             int64_t *nnz_c, uint64_t **liv_c, double **val_c, double **abs_c)
{
    const u128_t lim = ((u128_t)1 << 127) - 1;
    int is_con_a[ORC_MAX_ORDER] = {0}, is_con_b[ORC_MAX_ORDER] = {0};
    u128_t tot_a, tot_b, m = 1, n = 1;
    u128_t coord[ORC_MAX_ORDER];
    int rc;
    wbent_t *bs = NULL;
    wa_t *as = NULL;
    wprod_t *prods = NULL;
    int64_t nprod = 0, cap = 0;

    *nnz_c = 0; *liv_c = NULL; *val_c = NULL; *abs_c = NULL;
    if (!valid_sig(order_a, sig_a) || !valid_sig(order_b, sig_b)) return ORC_ERR_INVALID;
    if ((rc = checked_product_wide(order_a, dims_a, &tot_a)) != ORC_OK) return rc;
    if ((rc = checked_product_wide(order_b, dims_b, &tot_b)) != ORC_OK) return rc;
    if (ncontract < 0 || ncontract > order_a || ncontract > order_b) return ORC_ERR_INVALID;
    for (int c = 0; c < ncontract; ++c) {
        int ma = modes_a[c], mb = modes_b[c];
        if (ma < 0 || ma >= order_a || mb < 0 || mb >= order_b) return ORC_ERR_INVALID;
        if (is_con_a[ma] || is_con_b[mb]) return ORC_ERR_INVALID;
        if (dims_a[ma] != dims_b[mb]) return ORC_ERR_INVALID;
        is_con_a[ma] = 1; is_con_b[mb] = 1;
    }
    if ((order_a - ncontract) + (order_b - ncontract) > ORC_MAX_ORDER) return ORC_ERR_INVALID;
    for (int t = 0; t < order_a; ++t) if (!is_con_a[t]) m *= (u128_t)dims_a[t];
    for (int t = 0; t < order_b; ++t) if (!is_con_b[t]) n *= (u128_t)dims_b[t];
    if (m > lim / n) return ORC_ERR_OVERFLOW;
    if (nnz_a == 0 || nnz_b == 0) return ORC_OK;

    bs = (wbent_t *)malloc(sizeof(wbent_t) * (size_t)nnz_b);
    as = (wa_t *)malloc(sizeof(wa_t) * (size_t)nnz_a);
    if (!bs || !as) { rc = ORC_ERR_OOM; goto done; }
    /* B entries keyed by their contracted coordinates (pairing order, the
     * first pair most significant), then by B's own LIV */
    for (int64_t e = 0; e < nnz_b; ++e) {
        const u128_t lv = ((u128_t)liv_b[2 * e + 1] << 64) | liv_b[2 * e];
        u128_t key = 0;
        if (lv >= tot_b) { rc = ORC_ERR_INVALID; goto done; }
        wide_coords(order_b, dims_b, sig_b, lv, coord);
        for (int c = 0; c < ncontract; ++c) key = key * (u128_t)dims_b[modes_b[c]] + coord[modes_b[c]];
        bs[e].key = key; bs[e].liv = lv; bs[e].idx = e;
    }
    qsort(bs, (size_t)nnz_b, sizeof(wbent_t), cmp_wbent);
    for (int64_t e = 0; e < nnz_a; ++e) {
        as[e].liv = ((u128_t)liv_a[2 * e + 1] << 64) | liv_a[2 * e];
        as[e].idx = e;
        if (as[e].liv >= tot_a) { rc = ORC_ERR_INVALID; goto done; }
    }
    qsort(as, (size_t)nnz_a, sizeof(wa_t), cmp_wa);

    for (int64_t q = 0; q < nnz_a; ++q) {
        const int64_t e = as[q].idx;
        u128_t key = 0, row = 0;
        int64_t lo, hi;
        wide_coords(order_a, dims_a, sig_a, as[q].liv, coord);
        for (int c = 0; c < ncontract; ++c) key = key * (u128_t)dims_a[modes_a[c]] + coord[modes_a[c]];
        for (int t = 0; t < order_a; ++t) if (!is_con_a[t]) row = row * (u128_t)dims_a[t] + coord[t];
        lo = 0; hi = nnz_b;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (bs[mid].key < key) lo = mid + 1; else hi = mid;
        }
        for (int64_t j = lo; j < nnz_b && bs[j].key == key; ++j) {
            u128_t cb[ORC_MAX_ORDER];
            u128_t col = 0;
            const double av = val_a[e], bv = val_b[bs[j].idx];
            wide_coords(order_b, dims_b, sig_b, bs[j].liv, cb);
            for (int t = 0; t < order_b; ++t) if (!is_con_b[t]) col = col * (u128_t)dims_b[t] + cb[t];
            if (nprod == cap) {
                int64_t ncap = cap ? cap * 2 : 1024;
                wprod_t *np = (wprod_t *)realloc(prods, sizeof(wprod_t) * (size_t)ncap);
                if (!np) { rc = ORC_ERR_OOM; goto done; }
                prods = np; cap = ncap;
            }
            prods[nprod].out = row * n + col;
            prods[nprod].seq = nprod;
            prods[nprod].v = av * bv;
            prods[nprod].a = fabs(av) * fabs(bv);
            ++nprod;
        }
    }
    qsort(prods, (size_t)nprod, sizeof(wprod_t), cmp_wprod);
    {
        int64_t nc = 0;
        for (int64_t i = 0; i < nprod; ++i)
            if (i == 0 || prods[i].out != prods[i - 1].out) ++nc;
        *liv_c = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)(nc ? nc : 1));
        *val_c = (double *)malloc(sizeof(double) * (size_t)(nc ? nc : 1));
        *abs_c = (double *)malloc(sizeof(double) * (size_t)(nc ? nc : 1));
        if (!*liv_c || !*val_c || !*abs_c) { rc = ORC_ERR_OOM; goto done; }
        nc = -1;
        for (int64_t i = 0; i < nprod; ++i) {
            if (i == 0 || prods[i].out != prods[i - 1].out) {
                ++nc;
                (*liv_c)[2 * nc] = (uint64_t)prods[i].out;
                (*liv_c)[2 * nc + 1] = (uint64_t)(prods[i].out >> 64);
                (*val_c)[nc] = 0.0;
                (*abs_c)[nc] = 0.0;
            }
            (*val_c)[nc] += prods[i].v;
            (*abs_c)[nc] += prods[i].a;
        }
        *nnz_c = nc + 1;
    }
    rc = ORC_OK;
done:
    if (rc != ORC_OK) {
        free(*liv_c); free(*val_c); free(*abs_c);
        *liv_c = NULL; *val_c = NULL; *abs_c = NULL; *nnz_c = 0;
    }
    free(bs);
    free(as);
    free(prods);
    return rc;
}
