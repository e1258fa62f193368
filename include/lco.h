/*
 * lco.h -- C ABI of the GB300 (sm_103a) library for sparse-tensor
 * rearrangement and multiplication over the linearised-coordinate (LCO)
 * format (Harrison & Joseph, "High Performance Rearrangement and
 * Multiplication Routines for Sparse Tensor Arithmetic").
 *
 * Data model (Sec. 3.1, Table 1).  An LCO tensor of order N holds nnz
 * non-zeros as two parallel arrays: signed 64-bit linearised index values
 * (LIVs) and IEEE double values.  The LIV of coordinate (c_0 .. c_{N-1})
 * under lexicographic order `sig` (sig[0] = least significant mode) is
 *     LIV = c_{sig[0]} + n_{sig[0]} (c_{sig[1]} + n_{sig[1]} (c_{sig[2]} + ...)),
 * e.g. LIV = i + n_i (j + n_j k) for sig {0,1,2}.  The product of the dims
 * must not exceed 2^63 - 1 (Sec. 3.1).  A valid tensor has strictly
 * ascending LIVs (sorted, no duplicates).
 *
 * Conventions for every entry point:
 *   - Array arguments named *_liv, *_val, ws are DEVICE pointers owned by
 *     the caller; lco_shape / lco_plan_info / lco_rp_info are HOST structs.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work is enqueued asynchronously on it; nothing synchronises the stream
 *     unless the entry point says so.
 *   - The return value is a status (lco_status) of the host-side checks and
 *     launches.  Errors found on the device (a wait that ran out, a capacity
 *     that was too small) are written to the workspace header and read with
 *     lco_workspace_status() once the stream has finished.
 *   - Workspaces are device buffers of the size the matching *_workspace()
 *     call reports; they must be 256-byte aligned, zero-filled before their
 *     first use, and not touched by the caller between calls.  A workspace
 *     serves one call at a time.
 *   - Outputs must not alias inputs.
 *   - No entry point allocates device memory except lco_serve_create.
 *   - Within a call, a kernel that follows another kernel is enqueued as a
 *     programmatic dependent launch (scheduled while its predecessor
 *     drains; it waits for the predecessor's writes before touching
 *     memory).  LCO_PDL=0 in the environment, read once per process, makes
 *     these ordinary launches.  Results are identical either way, and both
 *     forms can be captured in a CUDA graph.
 */
#ifndef LCO_H
#define LCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LCO_MAX_ORDER 16

typedef enum {
    LCO_OK = 0,
    LCO_ERR_INVALID = 1,    /* malformed arguments (sig, dims, modes, sizes, pointers) */
    LCO_ERR_OVERFLOW = 2,   /* product of dims (or m*n of a contraction) > 2^63 - 1 (2^127 - 1 for wide LIVs) */
    LCO_ERR_UNSORTED = 3,   /* input LIVs not strictly ascending (checking entry points) */
    LCO_ERR_OOM = 4,        /* workspace smaller than reported, or host allocation failed */
    LCO_ERR_TIMEOUT = 5,    /* a device-side wait ran out (device status only) */
    LCO_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    LCO_ERR_ADMISSION = 7,  /* serve: request does not fit the memory budget */
    LCO_ERR_CAPACITY = 8,   /* output capacity smaller than the product count f */
    LCO_ERR_TOO_LARGE = 9   /* input larger than lco_radix_permute_static's fixed scratch */
} lco_status;

/* Shape of an LCO tensor (host struct).  sig[t] is the mode of significance
 * rank t, t = 0 least significant; dims[mode] is the range of that mode. */
typedef struct {
    int32_t order;
    int32_t sig[LCO_MAX_ORDER];
    int64_t dims[LCO_MAX_ORDER];
    int64_t nnz;
} lco_shape;

/* Human-readable name of a status code (static string). */
const char *lco_status_str(int32_t status);

/* Library build identification: returns the CUDA architecture the device
 * code was compiled for (e.g. 1030 for sm_103a). */
int32_t lco_build_arch(void);

/* Reads the device status word of a workspace (the first 4 bytes) after
 * synchronising `stream`.  *status receives LCO_OK or the device error. */
int32_t lco_workspace_status(const void *ws, int32_t *status, void *stream);

/* ------------------------------------------------------------------ */
/* Kernel timing and launch counting (tracing support; no paper        */
/* counterpart).  When timing is enabled, every kernel the library     */
/* launches on a stream that is not being captured into a CUDA graph   */
/* is bracketed by two CUDA events on that stream.                     */
/* ------------------------------------------------------------------ */

typedef struct {
    char name[40];   /* kernel name */
    float ms;        /* elapsed time between the bracketing events */
} lco_timing_record;

/* Enables (1) or disables (0) kernel timing and clears recorded launches. */
int32_t lco_timing_enable(int32_t enable);
/* Waits for the recorded launches to finish and copies up to `max` records
 * (oldest first) to `out`; *count receives the number copied.  The record
 * buffer (4096 launches) is then cleared. */
int32_t lco_timing_read(lco_timing_record *out, int32_t max, int32_t *count);
/* Number of kernels this library has launched from the host since it was
 * loaded (graph replays are not counted). */
int64_t lco_launch_count(void);

/* ------------------------------------------------------------------ */
/* Re-linearisation ("LIV shuffle", Sec. 3.1 and Sec. 4.1 first step)  */
/* ------------------------------------------------------------------ */

/* Recomputes every LIV of `t` (order t->sig) for the order `new_sig`:
 * liv_out[e] = LIV of the coordinates of liv_in[e] under new_sig.  The
 * element order is unchanged.  liv_in / liv_out: device, t->nnz int64 each.
 * Errors: LCO_ERR_INVALID (sig not a permutation, order outside 1..16,
 * dims < 1), LCO_ERR_OVERFLOW (product of dims > 2^63 - 1).  LIVs outside
 * [0, prod dims) give unspecified output values but never out-of-bounds
 * accesses. */
int32_t lco_relinearise(const lco_shape *t, const int32_t *new_sig,
                        const int64_t *liv_in, int64_t *liv_out, void *stream);

/* ------------------------------------------------------------------ */
/* Radix permutation (Sec. 4, "permutation": rearranging sorted data   */
/* into a new lexicographic order; Sec. 4.1 the RP algorithm)           */
/* ------------------------------------------------------------------ */

/* Host-side description of how a permutation is carried out (Sec. 4.1):
 * which modes are rearrangement indices, the region size m_top and the
 * resting-suffix divisor m_low, the sort key width and the radix passes. */
typedef struct {
    int32_t n_rearr;                 /* number of rearrangement indices; 0 = identity */
    int32_t is_rearr[LCO_MAX_ORDER]; /* per mode: 1 rearrangement, 0 resting */
    int64_t m_top;                   /* index values per region of constant leading resting indices */
    int64_t m_low;                   /* product of dims of the resting suffix */
    int32_t key_bits;                /* bits of the sort key newLIV / m_low */
    int32_t digit_bits;              /* radix digit width */
    int32_t passes;                  /* radix passes of the digit plan (before passes whose digit
                                        is constant are skipped on the device) */
    int32_t segments;                /* 1 = flat sort */
} lco_rp_info;

/* Fills *info for permuting a tensor of shape `t` to `new_sig`.  Host only,
 * no device work.  Errors: LCO_ERR_INVALID, LCO_ERR_OVERFLOW. */
int32_t lco_radix_permute_info(const lco_shape *t, const int32_t *new_sig, lco_rp_info *info);

/* Workspace bytes for lco_radix_permute on shape `t` (nnz = t->nnz). */
int32_t lco_radix_permute_workspace(const lco_shape *t, const int32_t *new_sig, size_t *ws_bytes);

/* Rearranges (liv_in, val_in), strictly ascending in order t->sig, into
 * (liv_out, val_out), strictly ascending in order new_sig, with liv_out
 * holding the new LIVs.  Values are moved bit-exactly.  Implementation:
 * one read of the re-linearised keys counts every pass's digits, then one
 * stable scatter pass per radix digit of the key newLIV div m_low (the
 * resting suffix is supplied by stability), least significant first, each
 * tile finding its digits' offsets by decoupled look-back; passes whose
 * digit is constant over the data are skipped on the device.  When two
 * passes remain and every bucket of the high digit holds at most 8,192
 * entries (decided on the device), the high digit is scattered first and
 * each bucket is then sorted by the low digit inside one CTA.
 * liv_in/val_in/liv_out/val_out: device, t->nnz elements each, no aliasing.
 * ws: device workspace of lco_radix_permute_workspace() bytes.
 * Errors: LCO_ERR_INVALID, LCO_ERR_OVERFLOW, LCO_ERR_OOM (ws too small),
 * LCO_ERR_CUDA; device status LCO_ERR_TIMEOUT. */
int32_t lco_radix_permute(const lco_shape *t, const int32_t *new_sig,
                          const int64_t *liv_in, const double *val_in,
                          int64_t *liv_out, double *val_out,
                          void *ws, size_t ws_bytes, void *stream);

/* Same permutation as lco_radix_permute, for callers that cannot
 * allocate device memory: a plug-in inside a host application that owns
 * every device allocation (its own caching allocator, or all memory
 * reserved at start-up with no allocation allowed afterwards) can neither
 * call cudaMalloc nor obtain a workspace of a size it does not know in
 * advance.  This entry point takes no workspace and allocates nothing:
 * its scratch is one fixed 3 MiB array in device memory, defined by this
 * library and held by every GPU that loads it until the process exits.
 * The paper has no counterpart; it is a deployment convenience.
 *   - t->nnz must not exceed 65536; larger inputs return
 *     LCO_ERR_TOO_LARGE without doing any device work.
 *   - The first call on each device looks up the device address of the
 *     array (with that device current); make that first call before any
 *     stream capture on the device.
 *   - Every call on a device shares the one array: calls whose device
 *     work overlaps (different streams, or different host threads) race
 *     and corrupt each other's results.  Serialise them.
 *   - The device address is cached per device ordinal for the life of
 *     the process: after cudaDeviceReset (or a release and re-creation of
 *     the device's primary context) the cached address is stale, so do not
 *     call this entry point on that device again in the same process.
 *   - Inputs and outputs are device arrays as for lco_radix_permute.  The
 *     return value covers the host-side checks and launches only; the
 *     device status of the last call on a device is read with
 *     lco_radix_permute_static_status.  When it is not LCO_OK the output
 *     of that call is undefined.
 * Errors: LCO_ERR_INVALID, LCO_ERR_OVERFLOW, LCO_ERR_TOO_LARGE,
 * LCO_ERR_CUDA. */
int32_t lco_radix_permute_static(const lco_shape *t, const int32_t *new_sig,
                                 const int64_t *liv_in, const double *val_in,
                                 int64_t *liv_out, double *val_out, void *stream);

/* Device status of the last lco_radix_permute_static call on the current
 * device: synchronises `stream` (the stream that call used), then copies the
 * status word of the fixed scratch array's header to *status (LCO_OK, or a
 * device error such as LCO_ERR_TIMEOUT; each call clears it first).  It
 * allocates nothing.  No paper counterpart.
 * Errors: LCO_ERR_INVALID (null status), LCO_ERR_CUDA. */
int32_t lco_radix_permute_static_status(int32_t *status, void *stream);

/* ------------------------------------------------------------------ */
/* Wide LIVs.  Sec. 3.1 limits LIVs to signed 64 bits (dims multiplying */
/* to at most 2^63 - 1) and leaves larger LIVs to future work, as does  */
/* Sec. 7.  A wide LIV is an unsigned 128-bit integer with the same     */
/* formula, stored as two uint64 words, low word first (16 bytes per    */
/* non-zero); the dims of a wide tensor multiply to at most 2^127 - 1.  */
/* lco_shape is used unchanged (each dim still fits int64).             */
/* ------------------------------------------------------------------ */

/* Wide counterpart of lco_relinearise: liv_in / liv_out are device arrays
 * of 2 * t->nnz uint64 (low, high word per non-zero).  Errors:
 * LCO_ERR_INVALID (sig, order, dims, pointers), LCO_ERR_OVERFLOW (product
 * of dims > 2^127 - 1).  LIVs outside [0, prod dims) give unspecified
 * output values but never out-of-bounds accesses. */
int32_t lco_relinearise_wide(const lco_shape *t, const int32_t *new_sig,
                             const uint64_t *liv_in, uint64_t *liv_out, void *stream);

/* How a wide permutation is carried out: rearrangement indices (Sec. 4.1),
 * the width of the sort key (the new LIV without its resting suffix), the
 * 54-bit chunks it is sorted in (least significant first) and the radix
 * passes before device-side skipping of constant digits. */
typedef struct {
    int32_t n_rearr;
    int32_t key_bits;
    int32_t chunks;
    int32_t passes;
} lco_rp_wide_info;

int32_t lco_radix_permute_wide_info(const lco_shape *t, const int32_t *new_sig, lco_rp_wide_info *info);

/* Workspace bytes for lco_radix_permute_wide (about 100 bytes per non-zero
 * plus the radix engine's tables). */
int32_t lco_radix_permute_wide_workspace(const lco_shape *t, const int32_t *new_sig, size_t *ws_bytes);

/* Wide counterpart of lco_radix_permute (Sec. 4.1 with 128-bit LIVs):
 * rearranges (liv_in, val_in), strictly ascending in order t->sig, into
 * (liv_out, val_out), strictly ascending in order new_sig.  liv arrays hold
 * 2 * t->nnz uint64 (low, high word per non-zero), val arrays t->nnz
 * doubles, all on the device, no aliasing.  The key (new LIV without its
 * resting suffix) is sorted in 54-bit chunks by the stable radix engine,
 * least significant chunk first, carrying input positions; the new LIVs and
 * values are then gathered.  ws: lco_radix_permute_wide_workspace() bytes,
 * 256-byte aligned, zero-filled before its first use.  Errors as
 * lco_radix_permute (LCO_ERR_OVERFLOW past 2^127 - 1). */
int32_t lco_radix_permute_wide(const lco_shape *t, const int32_t *new_sig,
                               const uint64_t *liv_in, const double *val_in,
                               uint64_t *liv_out, double *val_out,
                               void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* Contraction C = A x_modes B (Sec. 5: map to matrices, convert to a   */
/* multiplication datatype and multiply, map back; Table 4 dispatch)    */
/* ------------------------------------------------------------------ */

typedef enum {
    LCO_ALG_AUTO = -1,
    LCO_ALG_CSR = 0,    /* Sec. 5.2.2, row-by-row with an accumulator, B singly compressed */
    LCO_ALG_CSC = 1,    /* column-by-column counterpart (run as CSR on the transposed product) */
    LCO_ALG_DCSR = 2,   /* Sec. 5.2.3, B doubly compressed (row-sparse B) */
    LCO_ALG_DCSC = 3,
    LCO_ALG_CSRNA = 4,  /* Sec. 5.2.4, no accumulator: expand f(i), sort, sum duplicates */
    LCO_ALG_CSCNA = 5,
    LCO_ALG_SOP = 6     /* Sec. 5.2.5, simple outer product: expand all f, sort, sum */
} lco_alg;

typedef struct lco_plan lco_plan;   /* opaque host object */

typedef struct {
    int32_t alg;             /* lco_alg chosen (Table 4, or forced) */
    int32_t transposed;      /* 1: column variant, run on B^T A^T; C is column-major */
    int32_t class_a;         /* 0 sparse, 1 row-sparse, 2 column-sparse, 3 index-sparse */
    int32_t class_b;
    int32_t permute_a;       /* 1 if A must be rearranged into its matrix order */
    int32_t permute_b;
    int64_t m, k, n;         /* matrix sizes: A is m x k, B is k x n */
    lco_shape c_shape;       /* modes, dims and order of C; c_shape.nnz is 0 */
} lco_plan_info;

/* Plans C = A x B contracting modes_a[i] of A with modes_b[i] of B
 * (i < ncontract; pairs listed most significant first in the matrix
 * column/row index).  C's modes are A's free modes in increasing mode
 * number followed by B's free modes in increasing mode number.  C is
 * row-major (its last mode least significant) for the row variants and
 * column-major (B's free modes most significant) for the column variants;
 * the chosen order is reported in lco_plan_info.c_shape.sig.
 * force_alg = LCO_ALG_AUTO applies Table 4 with the hyper-sparsity test
 * dim / nnz > 3; any other lco_alg value forces that algorithm.
 * Host only.  Errors: LCO_ERR_INVALID (modes, dims mismatch, order),
 * LCO_ERR_OVERFLOW (m*n > 2^63 - 1). */
int32_t lco_contract_plan(const lco_shape *a, const lco_shape *b, int32_t ncontract,
                          const int32_t *modes_a, const int32_t *modes_b,
                          int32_t force_alg, lco_plan **plan);
int32_t lco_plan_get_info(const lco_plan *plan, lco_plan_info *info);
int32_t lco_plan_destroy(lco_plan *plan);

/* Workspace bytes for a contraction whose output capacity is `cap` entries
 * (cap must be >= f, the number of scalar products). */
int32_t lco_contract_workspace(const lco_plan *plan, int64_t cap, size_t *ws_bytes);

/* Results of a contraction, written by the device into the workspace
 * header and read with lco_contract_result(). */
typedef struct {
    int32_t status;   /* LCO_OK, LCO_ERR_CAPACITY (f > cap), LCO_ERR_TIMEOUT */
    int32_t alg;      /* algorithm that ran */
    int64_t nnz_c;    /* number of entries written to C */
    int64_t f;        /* number of scalar products (Sec. 5.2 notation f) */
    int64_t nzr_b;    /* non-empty rows of the (matricised) B */
} lco_contract_result;

/* Phase 1 ("symbolic"): rearranges A and B into their matrix orders when
 * needed, builds B's multiplication datatype (CSR row pointers or DCSR
 * rows with an auxiliary index) and counts the products f.  Leaves its
 * results in `ws`.  a_liv/a_val/b_liv/b_val: device, nnz of each shape. */
int32_t lco_contract_symbolic(const lco_plan *plan,
                              const int64_t *a_liv, const double *a_val,
                              const int64_t *b_liv, const double *b_val,
                              void *ws, size_t ws_bytes, void *stream);

/* Phase 2 ("numeric"): multiplies and writes C (c_liv/c_val, device, room
 * for `cap` entries) sorted in C's order, using the phase-1 results in
 * `ws`.  If f > cap nothing is written and the device status is
 * LCO_ERR_CAPACITY.  The number of entries written is in the result. */
int32_t lco_contract_numeric(const lco_plan *plan,
                             const int64_t *a_liv, const double *a_val,
                             const int64_t *b_liv, const double *b_val,
                             int64_t *c_liv, double *c_val, int64_t cap,
                             void *ws, size_t ws_bytes, void *stream);

/* Phase 1 followed by phase 2 on the same stream, no host synchronisation. */
int32_t lco_contract(const lco_plan *plan,
                     const int64_t *a_liv, const double *a_val,
                     const int64_t *b_liv, const double *b_val,
                     int64_t *c_liv, double *c_val, int64_t cap,
                     void *ws, size_t ws_bytes, void *stream);

/* Synchronises `stream` and copies the result header of `ws` to *out. */
int32_t lco_contract_result_get(const void *ws, lco_contract_result *out, void *stream);

/* Contraction of wide tensors (Sec. 5's product with the LIVs of Sec. 3.1
 * evaluated as unsigned 128-bit integers; Sec. 3.1 and Sec. 7 leave such
 * index spaces to future work).  C[i, j] = sum_k A[i, k] B[k, j] over the
 * matricised operands, C's modes being A's free modes then B's (increasing
 * mode numbers), row-major, every index (row, contracted, column) up to 127
 * bits; A's and B's dims, and C's, multiply to at most 2^127 - 1.
 * Implementation: A and B are permuted (lco_radix_permute_wide) into their
 * matrix orders; every row, contracted and column key is replaced by its
 * rank among the keys that occur (ranks keep the order); the 64-bit
 * contraction (lco_contract, Table 4 on the rank matrices) multiplies the
 * rank matrices, whose shapes (2 nnz_A x (nnz_B + 1), (nnz_B + 1) x nnz_B)
 * are fixed at planning; each entry of the rank product is mapped back to
 * row key * n + column key.  Sums run in the same order as every 64-bit
 * branch (entries of A in order, each B row in order).
 * Liv arrays are device arrays of 2 * nnz uint64 (low, high word per
 * entry), values device doubles; ws: lco_contract_wide_workspace bytes,
 * 256-byte aligned, any content (each call resets what it uses).  The same
 * ws must carry phase 1's results into phase 2 (a workspace sized for a
 * larger capacity keeps phase 1's layout).  Phase 1 reports f (the
 * product count) through lco_contract_wide_result_get; C needs room for f
 * entries.  Errors: LCO_ERR_INVALID (modes, dims, order, pointers),
 * LCO_ERR_OVERFLOW (a product of dims past 2^127 - 1, or nnz too large for
 * the rank matrices' 63-bit LIVs), LCO_ERR_OOM (ws too small), LCO_ERR_CUDA;
 * device status LCO_ERR_CAPACITY (f > cap), LCO_ERR_TIMEOUT. */
typedef struct lco_wide_plan lco_wide_plan;   /* opaque host object */

int32_t lco_contract_wide_plan(const lco_shape *a, const lco_shape *b, int32_t ncontract,
                               const int32_t *modes_a, const int32_t *modes_b, lco_wide_plan **plan);
int32_t lco_contract_wide_plan_destroy(lco_wide_plan *plan);
/* C's shape (nnz 0) and the Table-4 branch the rank product takes (may be NULL). */
int32_t lco_contract_wide_info(const lco_wide_plan *plan, lco_shape *c_shape, int32_t *inner_alg);
/* Workspace bytes for output capacity cap (0 suffices for phase 1). */
int32_t lco_contract_wide_workspace(const lco_wide_plan *plan, int64_t cap, size_t *ws_bytes);
/* Phase 1: permutations, ranks, rank matrices, phase 1 of their product. */
int32_t lco_contract_wide_symbolic(const lco_wide_plan *plan, const uint64_t *a_liv, const double *a_val,
                                   const uint64_t *b_liv, const double *b_val, void *ws, size_t ws_bytes,
                                   void *stream);
/* Phase 2: the rank product and C (c_liv: 2 * cap uint64, c_val: cap doubles). */
int32_t lco_contract_wide_numeric(const lco_wide_plan *plan, uint64_t *c_liv, double *c_val, int64_t cap,
                                  void *ws, size_t ws_bytes, void *stream);
/* Synchronises `stream`; status, f and the number of entries of C. */
int32_t lco_contract_wide_result_get(const lco_wide_plan *plan, const void *ws, lco_contract_result *out,
                                     void *stream);

/* ------------------------------------------------------------------ */
/* Tuning hints (planner inputs chosen by an autotuner; no paper        */
/* counterpart beyond Table 4's choice, which they may override)        */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t alg;             /* LCO_ALG_AUTO (Table 4) or a forced lco_alg */
    int32_t max_digit_bits;  /* radix digit width cap for operand permutations, 1..11; 0 = the
                                default of 9 bits (wider digits coalesce worse on random keys) */
    int32_t radix_order;     /* operand permutations: 0 = decided on the device (high digit
                                first, each high-digit bucket then sorted inside one CTA, when
                                two passes remain and every bucket holds at most 8,192 entries;
                                LSD passes otherwise), 1 = LSD passes only */
} lco_tune;

/* lco_contract_plan with tuning hints (tune may be NULL = defaults). */
int32_t lco_contract_plan_ex(const lco_shape *a, const lco_shape *b, int32_t ncontract,
                             const int32_t *modes_a, const int32_t *modes_b,
                             const lco_tune *tune, lco_plan **plan);

/* Contraction with entrywise mode pairs (Sec. 5: a product whose operands
 * share indices that are neither summed nor dropped maps to one matrix
 * product per value of the shared indices):
 *     C[h, free_a, free_b] = sum_k A[h, free_a, k] B[h, k, free_b]
 * (emodes_a[t], emodes_b[t]) are the shared pairs (equal dims, distinct from
 * the contracted modes).  C's modes are the shared pairs (pairing order,
 * dims from A), then A's free modes, then B's free modes; the shared modes
 * are the most significant in C's order (lco_plan_info.c_shape gives the
 * sig).  All of it is one product: the shared indices lead the rows of both
 * matrix views, and an entry of row (h, i) meets R's row (h, k).  Table 4 is
 * applied to the flattened views, whose dim/nnz ratios are the per-batch
 * ones.  nentry = 0 is lco_contract_plan_ex.  The rest of the contraction
 * API (workspace, phases, results) is unchanged. */
int32_t lco_contract_plan_entrywise(const lco_shape *a, const lco_shape *b, int32_t ncontract,
                                    const int32_t *modes_a, const int32_t *modes_b, int32_t nentry,
                                    const int32_t *emodes_a, const int32_t *emodes_b, const lco_tune *tune,
                                    lco_plan **plan);

/* ------------------------------------------------------------------ */
/* Batched contractions (many independent, uneven problems per call)    */
/* ------------------------------------------------------------------ */

/* One problem of a batch: operand shapes, the contracted mode pairs and
 * the algorithm (LCO_ALG_AUTO or a tuner's choice). */
typedef struct {
    lco_shape a;
    lco_shape b;
    int32_t ncontract;
    int32_t modes_a[LCO_MAX_ORDER];
    int32_t modes_b[LCO_MAX_ORDER];
    int32_t alg;             /* LCO_ALG_AUTO or a forced algorithm */
    int32_t max_digit_bits;  /* radix digit width cap (0 = default), see lco_tune */
    int32_t radix_order;     /* 0 = decided on the device, 1 = LSD passes only; see lco_tune */
} lco_problem;

/* Device pointers of one problem's operands and output (C with room for
 * caps[i] entries). */
typedef struct {
    const int64_t *a_liv;
    const double *a_val;
    const int64_t *b_liv;
    const double *b_val;
    int64_t *c_liv;
    double *c_val;
} lco_operands;

typedef struct lco_batch lco_batch;   /* opaque host object */

/* Plans nprob problems and creates `nstreams` (1..64) worker streams.  Each
 * problem is planned exactly as lco_contract_plan does (host only). */
int32_t lco_batch_plan(int32_t nprob, const lco_problem *probs, int32_t nstreams, lco_batch **batch);
int32_t lco_batch_destroy(lco_batch *batch);
int32_t lco_batch_info(const lco_batch *batch, int32_t i, lco_plan_info *info);

/* Bytes of the single batch workspace for output capacities caps[nprob]
 * (caps = NULL: enough for lco_batch_symbolic only). */
int32_t lco_batch_workspace(const lco_batch *batch, const int64_t *caps, size_t *ws_bytes);

/* Phase 1 / phase 2 / both for every problem, as lco_contract_symbolic /
 * _numeric / lco_contract do for one.  Work is forked from `stream` onto
 * the batch's worker streams (events) and joined back into `stream`, so a
 * whole call can be captured into one CUDA graph.  ops[nprob]: device
 * pointers; caps must be the same array (values) the workspace was sized
 * with.  No host synchronisation.
 * lco_batch_symbolic / _numeric run each problem's phases on its own.
 * lco_batch_contract runs the problems whose operands are already in their
 * matrix orders as a few stacked products (Sec. 5's entrywise modes read
 * the other way: independent products are one product over a shared
 * problem index; grouped by row-kernel family), each problem's results
 * bit-identical to a single call; the other problems run on their own.  It
 * copies a table of the problems' pointers into the workspace from a host
 * buffer the batch owns: a CUDA graph captured from it replays with the
 * pointers of the latest lco_batch_contract call on this batch, and calls
 * with different ops must not overlap in time. */
int32_t lco_batch_symbolic(lco_batch *batch, const lco_operands *ops, const int64_t *caps,
                           void *ws, size_t ws_bytes, void *stream);
int32_t lco_batch_numeric(lco_batch *batch, const lco_operands *ops, const int64_t *caps,
                          void *ws, size_t ws_bytes, void *stream);
int32_t lco_batch_contract(lco_batch *batch, const lco_operands *ops, const int64_t *caps,
                           void *ws, size_t ws_bytes, void *stream);

/* Synchronises `stream` and reads every problem's result (out[nprob]). */
int32_t lco_batch_results(const lco_batch *batch, const int64_t *caps, const void *ws,
                          lco_contract_result *out, void *stream);

/* ------------------------------------------------------------------ */
/* Failure detection self-test (no paper counterpart)                   */
/* ------------------------------------------------------------------ */

/* Every device-side wait in the library (decoupled look-back over tiles,
 * and the mbarrier phase wait of its bulk-copy helper) gives up after a
 * budget of SM clock cycles (about one second), records LCO_ERR_TIMEOUT in
 * the status word and lets its kernel finish, so a lost producer never
 * hangs the GPU.  This call
 * makes both kinds of wait run out on purpose: with the budget lowered to
 * budget_cycles (an argument of this test kernel only: kernels running at
 * the same time on other streams keep the full budget), one warp looks back over tiles
 * that never publish and one thread waits on an mbarrier phase that never
 * completes.  scratch: device memory of at least 512 bytes (any content).
 * Synchronises `stream`; *lookback_status and *mbarrier_status receive the
 * two waits' status (LCO_ERR_TIMEOUT when they ran out as designed).
 * Errors: LCO_ERR_INVALID, LCO_ERR_CUDA. */
int32_t lco_selftest_wait(void *scratch, int64_t budget_cycles, int32_t *lookback_status,
                          int32_t *mbarrier_status, void *stream);

/* ------------------------------------------------------------------ */
/* Sorting and addition (Sec. 3.2; the sum of Eq. 4, Fig. 3c)           */
/* ------------------------------------------------------------------ */

/* Sorts nnz entries of a tensor of shape t (order, dims, sig) into
 * ascending LIV order: Sec. 3.2's sorting task (e.g. after construction or
 * unordered insertion), the general case of which a permutation is the
 * pre-sorted special case.  Every radix digit of the LIV is sorted (passes
 * whose digit is constant over the data are skipped); equal LIVs keep their
 * input order.  in_* and out_* are device arrays of t->nnz entries (not
 * aliased); ws is a device workspace of lco_sort_workspace bytes (256-byte
 * aligned, any content: the call resets what it uses).
 * Errors: LCO_ERR_INVALID, LCO_ERR_OVERFLOW, LCO_ERR_OOM (ws too small),
 * LCO_ERR_CUDA; device status (lco_workspace_status) LCO_ERR_TIMEOUT. */
int32_t lco_sort_workspace(const lco_shape *t, size_t *ws_bytes);
int32_t lco_sort(const lco_shape *t, const int64_t *in_liv, const double *in_val, int64_t *out_liv,
                 double *out_val, void *ws, size_t ws_bytes, void *stream);

/* C = alpha A + beta B for two sorted LCO tensors of the same shape and
 * order t (t->nnz is ignored): the addition of Eq. 4's two terms once one
 * is re-sorted into the other's order (Sec. 3.2, Fig. 3c).  Every LIV of A
 * or B is an entry of C -- a cancelled sum is kept as an explicit zero --
 * with alpha*a + beta*b where both have it (each product rounded, then
 * added) and the scaled value otherwise.  c_liv/c_val need room for
 * nnz_a + nnz_b entries; the entry count is read with lco_add_result.  ws
 * holds lco_add_workspace bytes (any content).  No host synchronisation.
 * Errors: LCO_ERR_INVALID, LCO_ERR_OOM, LCO_ERR_CUDA. */
int32_t lco_add_workspace(int64_t nnz_a, int64_t nnz_b, size_t *ws_bytes);
int32_t lco_add(const lco_shape *t, double alpha, const int64_t *a_liv, const double *a_val, int64_t nnz_a,
                double beta, const int64_t *b_liv, const double *b_val, int64_t nnz_b, int64_t *c_liv,
                double *c_val, void *ws, size_t ws_bytes, void *stream);
/* Synchronises `stream`; *nnz_c = entries of C, *status = device status. */
int32_t lco_add_result(const void *ws, int64_t *nnz_c, int32_t *status, void *stream);

/* ------------------------------------------------------------------ */
/* Device memory pool (bookkeeping over a caller-given address range;   */
/* no paper counterpart).  The served path keeps its operands, results  */
/* and workspaces in one such pool so that admission is a host-side    */
/* allocation that either fits or waits.                                */
/* ------------------------------------------------------------------ */

typedef struct lco_pool lco_pool;     /* opaque host object */

/* A first-fit pool over [base, base + bytes).  The pool never touches the
 * memory itself (any address range works, including one that is not
 * device memory); blocks are 256-byte aligned; freed neighbours merge.
 * Errors: LCO_ERR_INVALID (null base/out, bytes < 256), LCO_ERR_OOM. */
int32_t lco_pool_create(void *base, size_t bytes, lco_pool **pool);
int32_t lco_pool_destroy(lco_pool *pool);
/* *ptr = start of a free block of at least `bytes` bytes, or NULL with
 * LCO_ERR_OOM when no free block is large enough (nothing changes). */
int32_t lco_pool_alloc(lco_pool *pool, size_t bytes, void **ptr);
/* Returns a block from lco_pool_alloc; LCO_ERR_INVALID for any other
 * pointer (including a second free of the same block). */
int32_t lco_pool_free(lco_pool *pool, void *ptr);
/* Bytes in use, the peak of that, and the largest free block. */
int32_t lco_pool_stats(const lco_pool *pool, size_t *used, size_t *peak, size_t *largest_free);

/* ------------------------------------------------------------------ */
/* Served contractions (continuous batching; no paper counterpart).     */
/*                                                                      */
/* A server owns a device memory pool and a set of worker streams.      */
/* Operands are put once (copied into the pool) and referred to by      */
/* handle; requests name two handles and the contracted mode pairs and  */
/* are admitted, in arrival order, as soon as a stream slot is free and */
/* the pool holds their workspace.  A host worker thread runs each      */
/* request as Sec. 5.2's steps on its slot's stream -- phase 1 (f),     */
/* an asynchronous read of f, phase 2 into a pool buffer of f entries --  */
/* observing completion with CUDA events, so many requests are in       */
/* flight at once and none waits on another's host round trip.  The     */
/* arithmetic of a request is exactly that of lco_contract.             */
/* ------------------------------------------------------------------ */

typedef struct lco_server lco_server; /* opaque host object */

typedef struct {
    void *pool;            /* device memory for the pool, or NULL: the server cudaMallocs pool_bytes */
    size_t pool_bytes;     /* size of the pool */
    int32_t nslots;        /* requests in flight at once (1..256), one stream each */
    int32_t device;        /* CUDA device of the pool and streams (-1: current) */
    int32_t nworkers;      /* host worker threads sharing the slots (0: 4) */
} lco_serve_config;

/* Creates the server and starts its worker threads.  Errors: LCO_ERR_INVALID,
 * LCO_ERR_OOM (pool allocation), LCO_ERR_CUDA. */
int32_t lco_serve_create(const lco_serve_config *cfg, lco_server **srv);
/* Stops the worker (requests still queued fail with LCO_ERR_ADMISSION),
 * waits for work in flight, frees everything the server allocated. */
int32_t lco_serve_destroy(lco_server *srv);

/* Copies a sorted LCO tensor (liv/val on the host or the device) into the
 * pool and returns its handle (> 0).  Blocks until the copy is done.
 * Errors: LCO_ERR_INVALID, LCO_ERR_OVERFLOW, LCO_ERR_ADMISSION (pool full),
 * LCO_ERR_CUDA. */
int32_t lco_serve_put(lco_server *srv, const lco_shape *t, const int64_t *liv, const double *val,
                      int64_t *handle);
/* Releases an operand; requests already submitted keep it alive. */
int32_t lco_serve_drop(lco_server *srv, int64_t handle);

/* Queues C = A x_modes B (ncontract pairs, as lco_contract_plan) on operand
 * handles and returns its id at once.  The plan is made here, so shape
 * errors are returned synchronously (LCO_ERR_INVALID, LCO_ERR_OVERFLOW). */
int32_t lco_serve_submit(lco_server *srv, int64_t ha, int64_t hb, int32_t ncontract,
                         const int32_t *modes_a, const int32_t *modes_b, uint64_t *req);

typedef struct {
    int32_t done;          /* 0 queued or running, 1 finished */
    int32_t status;        /* LCO_OK or the request's error (device status, LCO_ERR_ADMISSION, ...) */
    int32_t alg;           /* algorithm that ran */
    lco_shape c;           /* shape of C (order, dims, sig; nnz = entries of C) */
    const int64_t *c_liv;  /* device, sorted; valid until lco_serve_release */
    const double *c_val;
    int64_t f;             /* scalar products */
    double submit_us;      /* host steady-clock times (microseconds, server epoch) */
    double done_us;
} lco_serve_result;

/* Non-blocking state of a request. Errors: LCO_ERR_INVALID (unknown id). */
int32_t lco_serve_poll(lco_server *srv, uint64_t req, lco_serve_result *out);
/* Blocks until the request finishes or timeout_us passes (out->done says
 * which); timeout_us < 0 waits without limit. */
int32_t lco_serve_wait(lco_server *srv, uint64_t req, int64_t timeout_us, lco_serve_result *out);
/* Frees a finished request's output; the pointers become invalid. */
int32_t lco_serve_release(lco_server *srv, uint64_t req);

typedef struct {
    uint64_t submitted, completed, failed;
    int64_t queued, in_flight;
    size_t pool_used, pool_peak, pool_bytes;
} lco_serve_stats;

int32_t lco_serve_get_stats(const lco_server *srv, lco_serve_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* LCO_H */
