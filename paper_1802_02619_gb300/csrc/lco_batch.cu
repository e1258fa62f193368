// lco_batch.cu -- many independent contractions in one enqueue.
//
// Every problem keeps its own plan (the Table-4 choice of Sec. 5.2, or the
// tuner's forced choice).  lco_batch_contract runs most problems as a few
// stacked products: Sec. 5 notes that a product whose operands share an
// index that is neither summed nor dropped (an entrywise mode) is one
// matrix product per value of that index -- so independent products are
// one product over a shared problem index h.  Problems whose operands are
// already in their matrix orders and whose plans take the same row kernel
// family (CSR, DCSR, CSRNA or SOP; a column variant is its row counterpart
// on the transposed product, as for a single call) form a group; each
// member's matrix view (L: mL x k, R: k x nR) is placed at h in stacked
// operands
//     L'[h, row, col]  (H x M x K),   R'[h, col, j]  (H x K x N),
// M, K, N the largest member sizes, which are then sorted as they stand;
// one entrywise contraction multiplies the group; each member's entries of
// C'[h, row, j] are mapped back into its own output.  A problem whose
// operand needs rearranging runs on its own (its own permutation keeps its
// own key width; a stacked sort would carry the problem index and the
// largest member's widths in every key -- measured slower).  A row (h, row) of L' holds exactly the member's
// row entries and meets exactly its R rows, in the same order, so every
// output sums the same products in the same order as a single call: results
// are bit-identical.  A group has a fixed number of launches however many
// problems it holds; the groups run concurrently on a pool of streams forked
// from the caller's stream and joined back into it, so a whole batch is
// captured as one CUDA graph.
//
// lco_batch_symbolic / lco_batch_numeric run each problem's phases on its
// own (they size the outputs).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lco_host.h"

namespace lco {
namespace {

// One member's side of a stacked operand (device table entry).
struct StackDesc {
    const int64_t *src_liv;
    const double *src_val;
    int64_t n;            // entries
    int64_t off;          // first stacked entry
    RelinParams relin;    // source LIV -> matrix-order LIV
    DivU64 div;           // k (L side: row = x div k) or nR (R side: col = x div nR)
};

// One member's output and results (device table entry).
struct OutDesc {
    int64_t *c_liv;
    double *c_val;
    int64_t cap;
    int64_t nR;           // the member's C row length
    int32_t alg;          // the member's own plan's algorithm
    int32_t pad;
};

constexpr int kST = 256;

// Member of stacked entry e: offs[m] <= e < offs[m + 1] (offs has H + 1
// entries, non-decreasing).
__device__ __forceinline__ int member_of(const int64_t *offs, int H, int64_t e) {
    int lo = 0, hi = H;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (offs[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Stacked LIVs of one side: L' = (h M + row) K + col, R' = (h K + col) N + j,
// from each member's matrix-order LIV.
__global__ void __launch_bounds__(kST) k_stack(const StackDesc *d, const int64_t *offs, int H, int64_t total,
                                               int side_r, int64_t M, int64_t K, int64_t N, int64_t *out_liv,
                                               double *out_val) {
    __shared__ int s_m0;
    const int64_t base = (int64_t)blockIdx.x * kST;
    if (base >= total) return;
    if (threadIdx.x == 0) s_m0 = member_of(offs, H, base);
    __syncthreads();
    const int64_t e = base + threadIdx.x;
    if (e >= total) return;
    int m = s_m0;
    while (m + 1 < H && offs[m + 1] <= e) ++m;
    const StackDesc &sd = d[m];
    const int64_t i = e - sd.off;
    if (i < 0 || i >= sd.n) return;     // entries of member m only
    const uint64_t x = (uint64_t)relin(sd.relin, sd.src_liv[i]);
    const uint64_t q = divu(sd.div, x);
    const int64_t r = (int64_t)(x - q * sd.div.d);
    out_liv[e] = side_r ? ((int64_t)m * K + (int64_t)q) * N + r : ((int64_t)m * M + (int64_t)q) * K + r;
    out_val[e] = sd.src_val[i];
}

// Per member: its entries of the stacked product (first, last), its product
// count f (from the stacked L row table: the work of the member's rows less
// their entries) and its result record; members whose f exceeds their
// capacity are marked (nothing of theirs is written).
struct ResultArgs {
    const WsHeader *hdr;        // the stacked contraction's header
    const int64_t *c_liv;       // stacked product
    const double *c_val;
    DivU64 div_mn;              // M N
    const int64_t *row_start, *row_id, *row_work;
    int64_t M;
    int H;
    const OutDesc *out;
    int64_t *first;             // [H]
    int64_t *last;              // [H]
    lco_contract_result *res;   // [H]
};

__device__ __forceinline__ int64_t lower_row(const int64_t *row_id, int64_t nrows, int64_t v) {
    int64_t lo = 0, hi = nrows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (row_id[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kST) k_unstack_bounds(const __grid_constant__ ResultArgs a) {
    const int64_t nc = a.hdr->status == 0 ? a.hdr->nnz_c : 0;
    for (int64_t i = (int64_t)blockIdx.x * kST + threadIdx.x; i < nc; i += (int64_t)gridDim.x * kST) {
        const int64_t h = (int64_t)divu(a.div_mn, (uint64_t)a.c_liv[i]);
        if (h >= a.H) continue;          // not a member's entry
        if (i == 0 || (int64_t)divu(a.div_mn, (uint64_t)a.c_liv[i - 1]) != h) a.first[h] = i;
        if (i == nc - 1 || (int64_t)divu(a.div_mn, (uint64_t)a.c_liv[i + 1]) != h) a.last[h] = i + 1;
    }
}

__global__ void __launch_bounds__(kST) k_unstack_results(const __grid_constant__ ResultArgs a) {
    const int h = blockIdx.x * kST + threadIdx.x;
    if (h >= a.H) return;
    const int64_t nrows = a.hdr->nrows_l;
    const int64_t ra = lower_row(a.row_id, nrows, (int64_t)h * a.M);
    const int64_t rb = lower_row(a.row_id, nrows, (int64_t)(h + 1) * a.M);
    const int64_t f = (a.row_work[rb] - a.row_work[ra]) - (a.row_start[rb] - a.row_start[ra]);
    lco_contract_result r{};
    r.status = a.hdr->status;
    r.alg = a.out[h].alg;
    r.f = f;
    r.nnz_c = r.status == 0 ? a.last[h] - a.first[h] : 0;
    r.nzr_b = 0;
    if (r.status == 0 && f > a.out[h].cap) {
        r.status = LCO_ERR_CAPACITY;
        r.nnz_c = 0;
    }
    a.res[h] = r;
}

// Each entry of the stacked product into its member's output (row-major in
// the member's own C: row * nR + j).
__global__ void __launch_bounds__(kST) k_unstack(const __grid_constant__ ResultArgs a, DivU64 div_n) {
    const int64_t nc = a.hdr->status == 0 ? a.hdr->nnz_c : 0;
    const uint64_t MN = a.div_mn.d;
    for (int64_t i = (int64_t)blockIdx.x * kST + threadIdx.x; i < nc; i += (int64_t)gridDim.x * kST) {
        const uint64_t l = (uint64_t)a.c_liv[i];
        const uint64_t h = divu(a.div_mn, l);
        if (h >= (uint64_t)a.H || a.res[h].status != 0) continue;
        const uint64_t rem = l - h * MN;
        const uint64_t row = divu(div_n, rem);
        const uint64_t j = rem - row * div_n.d;
        const OutDesc &o = a.out[h];
        const int64_t pos = i - a.first[h];
        if (pos < 0 || pos >= o.cap) continue;   // within the member's output only
        o.c_liv[pos] = (int64_t)row * o.nR + (int64_t)j;
        o.c_val[pos] = a.c_val[i];
    }
}

}  // namespace

// A group of problems multiplied as one stacked product.
struct Group {
    int32_t family = 0;              // row algorithm forced on the stacked product
    std::vector<int32_t> members;    // problem index of each h
    int64_t M = 1, K = 1, N = 1;     // largest member sizes
    int64_t nl = 0, nr = 0;          // stacked entries
    lco_plan *plan = nullptr;        // the stacked entrywise product
    lco_shape sl{}, sr{};            // stacked operand shapes (sorted as built)
    void *table_host = nullptr;      // pinned: descriptors, offsets, outputs
    size_t table_bytes = 0;
};

// Byte layout of a group's problem table (descriptors of both sides, their
// entry offsets, the outputs): the same in the pinned host copy and at the
// start of the group's workspace region, so one copy moves it.
struct TableLayout {
    size_t desc_l, desc_r, offs_l, offs_r, out, bytes;
};

inline TableLayout table_layout(size_t H) {
    TableLayout t{};
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += align_up(bytes ? bytes : 1); return o; };
    t.desc_l = take(H * sizeof(StackDesc));
    t.desc_r = take(H * sizeof(StackDesc));
    t.offs_l = take((H + 1) * 8);
    t.offs_r = take((H + 1) * 8);
    t.out = take(H * sizeof(OutDesc));
    t.bytes = off;
    return t;
}

// Byte layout of one group's region of the workspace for capacity cap_g.
struct GroupLayout {
    size_t desc_l, desc_r, offs_l, offs_r, out, first, last, res;   // table (desc_l .. out) is one copy
    size_t l_liv, l_val, r_liv, r_val;
    size_t c_liv, c_val, ws;
    size_t ws_bytes, total;
    int64_t cap;
};

}  // namespace lco

struct lco_batch {
    int32_t nprob;
    int32_t nstreams;
    std::vector<lco_plan *> plans;
    std::vector<lco::PlanView> views;
    std::vector<lco::Group> groups;
    std::vector<int32_t> group_of;       // group of each problem (-1: runs on its own)
    std::vector<int32_t> solo;           // problems outside every group
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> fork_ev, join_ev;
    int device;
    bool stacked_last = false;           // the last enqueue ran the stacked path
};

namespace {

using lco::Group;
using lco::GroupLayout;

void destroy(lco_batch *b) {
    if (!b) return;
    for (lco_plan *p : b->plans) lco_plan_destroy(p);
    for (auto &g : b->groups) {
        if (g.plan) lco_plan_destroy(g.plan);
        if (g.table_host) cudaFreeHost(g.table_host);
    }
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->fork_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : b->join_ev) cudaEventDestroy(e);
    delete b;
}

// Offsets of every problem's workspace inside the batch workspace (the
// per-problem phases).
int32_t layout(const lco_batch *b, const int64_t *caps, std::vector<size_t> &offs, size_t *total) {
    offs.resize(b->nprob);
    size_t off = 0;
    for (int i = 0; i < b->nprob; ++i) {
        size_t nb = 0;
        const int64_t cap = caps ? caps[i] : 0;
        if (cap < 0) return LCO_ERR_INVALID;
        int32_t rc = lco_contract_workspace(b->plans[i], cap, &nb);
        if (rc != LCO_OK) return rc;
        offs[i] = off;
        off += lco::align_up(nb);
    }
    *total = off;
    return LCO_OK;
}

GroupLayout group_layout(const Group &g, int64_t cap) {
    GroupLayout L{};
    const size_t H = g.members.size();
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += lco::align_up(bytes ? bytes : 1); return o; };
    L.cap = cap > 0 ? cap : 1;
    const lco::TableLayout T = lco::table_layout(H);
    L.desc_l = take(T.bytes);        // the whole table, sub-arrays at T's offsets
    L.desc_r = L.desc_l + T.desc_r;
    L.offs_l = L.desc_l + T.offs_l;
    L.offs_r = L.desc_l + T.offs_r;
    L.out = L.desc_l + T.out;
    L.first = take(H * 8);
    L.last = take(H * 8);
    L.res = take(H * sizeof(lco_contract_result));
    const size_t nl = (size_t)(g.nl > 0 ? g.nl : 1), nr = (size_t)(g.nr > 0 ? g.nr : 1);
    L.l_liv = take(nl * 8);
    L.l_val = take(nl * 8);
    L.r_liv = take(nr * 8);
    L.r_val = take(nr * 8);
    L.c_liv = take((size_t)L.cap * 8);
    L.c_val = take((size_t)L.cap * 8);
    lco_contract_workspace(g.plan, L.cap, &L.ws_bytes);
    L.ws = take(L.ws_bytes);
    L.total = off;
    return L;
}

// The stacked path's layout: one region per group, then one per problem
// that runs on its own (solo_offs[i], for problems outside every group).
int32_t stacked_layout(const lco_batch *b, const int64_t *caps, std::vector<size_t> &goffs,
                       std::vector<GroupLayout> &gl, std::vector<size_t> &solo_offs, size_t *total) {
    goffs.resize(b->groups.size());
    gl.resize(b->groups.size());
    solo_offs.assign(b->nprob, 0);
    size_t off = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group &g = b->groups[gi];
        int64_t cap = 0;
        for (int32_t i : g.members) {
            if (caps[i] < 0) return LCO_ERR_INVALID;
            cap += caps[i];
        }
        gl[gi] = group_layout(g, cap);
        goffs[gi] = off;
        off += lco::align_up(gl[gi].total);
    }
    for (int32_t i : b->solo) {
        if (caps[i] < 0) return LCO_ERR_INVALID;
        size_t nb = 0;
        int32_t rc = lco_contract_workspace(b->plans[i], caps[i], &nb);
        if (rc != LCO_OK) return rc;
        solo_offs[i] = off;
        off += lco::align_up(nb);
    }
    *total = off;
    return LCO_OK;
}

// Forks the pool from `origin`, runs fn(item, stream) for `count` items,
// joins the pool back into `origin`.
template <typename Fn>
int32_t fan_out(lco_batch *b, int count, cudaStream_t origin, Fn fn) {
    if (cudaEventRecord(b->fork_ev[0], origin) != cudaSuccess) return LCO_ERR_CUDA;
    for (int s = 0; s < b->nstreams; ++s)
        if (cudaStreamWaitEvent(b->streams[s], b->fork_ev[0], 0) != cudaSuccess) return LCO_ERR_CUDA;
    int32_t rc = LCO_OK;
    for (int i = 0; i < count && rc == LCO_OK; ++i) rc = fn(i, b->streams[i % b->nstreams]);
    for (int s = 0; s < b->nstreams; ++s) {
        if (cudaEventRecord(b->join_ev[s], b->streams[s]) != cudaSuccess) return LCO_ERR_CUDA;
        if (cudaStreamWaitEvent(origin, b->join_ev[s], 0) != cudaSuccess) return LCO_ERR_CUDA;
    }
    return rc;
}

// Row kernel family of a plan's algorithm (column variants run as their row
// counterparts on the transposed product).
int32_t row_family(int32_t alg) {
    switch (alg) {
    case LCO_ALG_CSC: return LCO_ALG_CSR;
    case LCO_ALG_DCSC: return LCO_ALG_DCSR;
    case LCO_ALG_CSCNA: return LCO_ALG_CSRNA;
    default: return alg;
    }
}

// Stacked index spaces stay below 2^62; groups that look rows up through
// CSR row pointers (one per stacked R row) keep H K at most 2^27.
bool fits(const Group &g, const lco::PlanView &v) {
    typedef unsigned __int128 u128;
    const u128 H = (u128)g.members.size() + 1;
    const u128 M = (u128)std::max<int64_t>(g.M, v.mL), K = (u128)std::max<int64_t>(g.K, v.k),
               N = (u128)std::max<int64_t>(g.N, v.nR);
    const u128 lim = (u128)1 << 62;
    if (H * M * K > lim || H * K * N > lim || H * M * N > lim) return false;
    if (v.lookup == 0 && H * K > ((u128)1 << 27)) return false;
    return true;
}

int32_t build_groups(lco_batch *b) {
    const int n = b->nprob;
    b->views.resize(n);
    b->group_of.assign(n, -1);
    std::vector<int> open;    // index of the open group of each key, -1 none
    open.assign(16, -1);
    for (int i = 0; i < n; ++i) {
        lco::PlanView &v = b->views[i];
        lco::plan_view(b->plans[i], &v);
        if (v.need_l || v.need_r) {
            b->solo.push_back(i);
            continue;
        }
        const int key = row_family(v.alg);
        int gi = open[key];
        if (gi < 0 || !fits(b->groups[gi], v)) {
            Group g;
            g.family = row_family(v.alg);
            b->groups.push_back(std::move(g));
            gi = (int)b->groups.size() - 1;
            open[key] = gi;
        }
        Group &g = b->groups[gi];
        g.members.push_back(i);
        g.M = std::max<int64_t>(g.M, v.mL);
        g.K = std::max<int64_t>(g.K, v.k);
        g.N = std::max<int64_t>(g.N, v.nR);
        g.nl += v.nnz_l;
        g.nr += v.nnz_r;
        b->group_of[i] = gi;
    }
    for (Group &g : b->groups) {
        const int64_t H = (int64_t)g.members.size();
        g.sl = lco_shape{};
        g.sl.order = 3;
        g.sl.dims[0] = H;
        g.sl.dims[1] = g.M;
        g.sl.dims[2] = g.K;
        g.sl.sig[0] = 2;
        g.sl.sig[1] = 1;
        g.sl.sig[2] = 0;
        g.sl.nnz = g.nl;
        g.sr = g.sl;
        g.sr.dims[1] = g.K;
        g.sr.dims[2] = g.N;
        g.sr.nnz = g.nr;
        const int32_t ma = 2, mb = 1, ea = 0, eb = 0;
        lco_tune t;
        t.alg = g.family;
        t.max_digit_bits = 0;
        t.radix_order = 0;
        int32_t rc = lco_contract_plan_entrywise(&g.sl, &g.sr, 1, &ma, &mb, 1, &ea, &eb, &t, &g.plan);
        if (rc != LCO_OK) return rc;
        g.table_bytes = lco::table_layout((size_t)H).bytes;
        if (cudaMallocHost(&g.table_host, g.table_bytes) != cudaSuccess) return LCO_ERR_OOM;
    }
    return LCO_OK;
}

// The pinned table of group g (descriptors, offsets, outputs) for `ops`,
// laid out by table_layout, as the copy to the workspace lands it.
void fill_table(const lco_batch *b, const Group &g, const lco_operands *ops, const int64_t *caps) {
    const size_t H = g.members.size();
    const lco::TableLayout T = lco::table_layout(H);
    char *t = reinterpret_cast<char *>(g.table_host);
    auto *dl = reinterpret_cast<lco::StackDesc *>(t + T.desc_l);
    auto *dr = reinterpret_cast<lco::StackDesc *>(t + T.desc_r);
    auto *ol = reinterpret_cast<int64_t *>(t + T.offs_l);
    auto *orr = reinterpret_cast<int64_t *>(t + T.offs_r);
    auto *out = reinterpret_cast<lco::OutDesc *>(t + T.out);
    int64_t sl = 0, sr = 0;
    for (size_t h = 0; h < H; ++h) {
        const int i = g.members[h];
        const lco::PlanView &v = b->views[i];
        const lco_operands &o = ops[i];
        dl[h].src_liv = v.l_is_a ? o.a_liv : o.b_liv;
        dl[h].src_val = v.l_is_a ? o.a_val : o.b_val;
        dl[h].n = v.nnz_l;
        dl[h].off = sl;
        dl[h].relin = v.relin_l;
        dl[h].div = lco::make_div((uint64_t)v.k);
        dr[h].src_liv = v.l_is_a ? o.b_liv : o.a_liv;
        dr[h].src_val = v.l_is_a ? o.b_val : o.a_val;
        dr[h].n = v.nnz_r;
        dr[h].off = sr;
        dr[h].relin = v.relin_r;
        dr[h].div = lco::make_div((uint64_t)v.nR);
        ol[h] = sl;
        orr[h] = sr;
        sl += v.nnz_l;
        sr += v.nnz_r;
        out[h].c_liv = o.c_liv;
        out[h].c_val = o.c_val;
        out[h].cap = caps[i];
        out[h].nR = v.nR;
        out[h].alg = v.alg;
        out[h].pad = 0;
    }
    ol[H] = sl;
    orr[H] = sr;
}

unsigned grid_of(int64_t n) { return (unsigned)((n + lco::kST - 1) / lco::kST); }

// Enqueues group g's stacked product on stream s.
int32_t run_group(lco_batch *b, Group &g, const GroupLayout &L, char *base, const lco_operands *ops,
                  const int64_t *caps, cudaStream_t s) {
    using namespace lco;
    const int H = (int)g.members.size();
    fill_table(b, g, ops, caps);
    if (cudaMemcpyAsync(base + L.desc_l, g.table_host, g.table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return LCO_ERR_CUDA;
    if (cudaMemsetAsync(base + L.first, 0, (size_t)H * 8, s) != cudaSuccess ||
        cudaMemsetAsync(base + L.last, 0, (size_t)H * 8, s) != cudaSuccess)
        return LCO_ERR_CUDA;
    const StackDesc *dl = reinterpret_cast<const StackDesc *>(base + L.desc_l);
    const StackDesc *dr = reinterpret_cast<const StackDesc *>(base + L.desc_r);
    const int64_t *ol = reinterpret_cast<const int64_t *>(base + L.offs_l);
    const int64_t *orr = reinterpret_cast<const int64_t *>(base + L.offs_r);
    int64_t *l_liv = reinterpret_cast<int64_t *>(base + L.l_liv);
    double *l_val = reinterpret_cast<double *>(base + L.l_val);
    int64_t *r_liv = reinterpret_cast<int64_t *>(base + L.r_liv);
    double *r_val = reinterpret_cast<double *>(base + L.r_val);
    if (g.nl > 0)
        LCO_LAUNCH("k_stack", s, k_stack<<<grid_of(g.nl), kST, 0, s>>>(dl, ol, H, g.nl, 0, g.M, g.K, g.N, l_liv,
                                                                     l_val));
    if (g.nr > 0)
        LCO_LAUNCH("k_stack", s, k_stack<<<grid_of(g.nr), kST, 0, s>>>(dr, orr, H, g.nr, 1, g.M, g.K, g.N, r_liv,
                                                                     r_val));
    int32_t rc;
    int64_t *c_liv = reinterpret_cast<int64_t *>(base + L.c_liv);
    double *c_val = reinterpret_cast<double *>(base + L.c_val);
    char *ws = base + L.ws;
    if ((rc = lco_contract(g.plan, l_liv, l_val, r_liv, r_val, c_liv, c_val, L.cap, ws, L.ws_bytes, s)) != LCO_OK)
        return rc;
    ResultArgs ra{};
    ra.hdr = reinterpret_cast<const WsHeader *>(ws);
    ra.c_liv = c_liv;
    ra.c_val = c_val;
    ra.div_mn = make_div((uint64_t)(g.M * g.N));
    plan_row_table(g.plan, ws, &ra.row_start, &ra.row_id, &ra.row_work);
    ra.M = g.M;
    ra.H = H;
    ra.out = reinterpret_cast<const OutDesc *>(base + L.out);
    ra.first = reinterpret_cast<int64_t *>(base + L.first);
    ra.last = reinterpret_cast<int64_t *>(base + L.last);
    ra.res = reinterpret_cast<lco_contract_result *>(base + L.res);
    const unsigned gc = (unsigned)std::min<int64_t>((L.cap + kST - 1) / kST, (int64_t)radix_sm_count() * 8);
    LCO_LAUNCH("k_unstack_bounds", s, k_unstack_bounds<<<gc, kST, 0, s>>>(ra));
    LCO_LAUNCH("k_unstack_results", s, k_unstack_results<<<grid_of(H), kST, 0, s>>>(ra));
    LCO_LAUNCH("k_unstack", s, k_unstack<<<gc, kST, 0, s>>>(ra, make_div((uint64_t)g.N)));
    return cudaGetLastError() == cudaSuccess ? LCO_OK : LCO_ERR_CUDA;
}

}  // namespace

extern "C" {

int32_t lco_batch_plan(int32_t nprob, const lco_problem *probs, int32_t nstreams, lco_batch **out) {
    if (!out || nprob < 1 || !probs) return LCO_ERR_INVALID;
    *out = nullptr;
    if (nstreams < 1) nstreams = 1;
    if (nstreams > 64) nstreams = 64;
    lco_batch *b = new (std::nothrow) lco_batch();
    if (!b) return LCO_ERR_OOM;
    b->nprob = nprob;
    b->nstreams = nstreams;
    cudaGetDevice(&b->device);
    for (int i = 0; i < nprob; ++i) {
        lco_plan *p = nullptr;
        lco_tune t;
        t.alg = probs[i].alg;
        t.max_digit_bits = probs[i].max_digit_bits;
        t.radix_order = probs[i].radix_order;
        int32_t rc = lco_contract_plan_ex(&probs[i].a, &probs[i].b, probs[i].ncontract, probs[i].modes_a,
                                          probs[i].modes_b, &t, &p);
        if (rc != LCO_OK) {
            destroy(b);
            return rc;
        }
        b->plans.push_back(p);
    }
    b->streams.resize(nstreams);
    b->join_ev.resize(nstreams);
    b->fork_ev.resize(1);
    for (int s = 0; s < nstreams; ++s) {
        if (cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[s], cudaEventDisableTiming) != cudaSuccess) {
            destroy(b);
            return LCO_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&b->fork_ev[0], cudaEventDisableTiming) != cudaSuccess) {
        destroy(b);
        return LCO_ERR_CUDA;
    }
    int32_t rc = build_groups(b);
    if (rc != LCO_OK) {
        destroy(b);
        return rc;
    }
    *out = b;
    return LCO_OK;
}

int32_t lco_batch_destroy(lco_batch *b) {
    destroy(b);
    return LCO_OK;
}

int32_t lco_batch_info(const lco_batch *b, int32_t i, lco_plan_info *info) {
    if (!b || i < 0 || i >= b->nprob) return LCO_ERR_INVALID;
    return lco_plan_get_info(b->plans[i], info);
}

int32_t lco_batch_workspace(const lco_batch *b, const int64_t *caps, size_t *ws_bytes) {
    if (!b || !ws_bytes) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t per_problem = 0;
    int32_t rc = layout(b, caps, offs, &per_problem);
    if (rc != LCO_OK) return rc;
    size_t stacked = 0;
    if (caps) {
        std::vector<size_t> goffs, solo;
        std::vector<GroupLayout> gl;
        if ((rc = stacked_layout(b, caps, goffs, gl, solo, &stacked)) != LCO_OK) return rc;
    }
    // one region serves both views: the per-problem phases and the stacked path
    *ws_bytes = per_problem > stacked ? per_problem : stacked;
    return LCO_OK;
}

int32_t lco_batch_symbolic(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws,
                           size_t ws_bytes, void *stream) {
    if (!b || !ops || !ws) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    char *base = reinterpret_cast<char *>(ws);
    b->stacked_last = false;
    return fan_out(b, b->nprob, (cudaStream_t)stream, [&](int i, cudaStream_t s) {
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps ? caps[i] : 0, &nb);
        return lco_contract_symbolic(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val,
                                     base + offs[i], nb, s);
    });
}

int32_t lco_batch_numeric(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws, size_t ws_bytes,
                          void *stream) {
    if (!b || !ops || !ws || !caps) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    char *base = reinterpret_cast<char *>(ws);
    b->stacked_last = false;
    return fan_out(b, b->nprob, (cudaStream_t)stream, [&](int i, cudaStream_t s) {
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps[i], &nb);
        return lco_contract_numeric(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val,
                                    ops[i].c_liv, ops[i].c_val, caps[i], base + offs[i], nb, s);
    });
}

int32_t lco_batch_contract(lco_batch *b, const lco_operands *ops, const int64_t *caps, void *ws, size_t ws_bytes,
                           void *stream) {
    lco::NvtxRange nvtx("lco_batch_contract");
    if (!b || !ops || !ws || !caps) return LCO_ERR_INVALID;
    std::vector<size_t> goffs, solo;
    std::vector<GroupLayout> gl;
    size_t total = 0;
    int32_t rc = stacked_layout(b, caps, goffs, gl, solo, &total);
    if (rc != LCO_OK) return rc;
    if (ws_bytes < total) return LCO_ERR_OOM;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LCO_ERR_INVALID;
    char *base = reinterpret_cast<char *>(ws);
    b->stacked_last = true;
    const int ng = (int)b->groups.size();
    return fan_out(b, ng + (int)b->solo.size(), (cudaStream_t)stream, [&](int item, cudaStream_t s) {
        if (item < ng) return run_group(b, b->groups[item], gl[item], base + goffs[item], ops, caps, s);
        const int i = b->solo[item - ng];
        size_t nb = 0;
        lco_contract_workspace(b->plans[i], caps[i], &nb);
        return lco_contract(b->plans[i], ops[i].a_liv, ops[i].a_val, ops[i].b_liv, ops[i].b_val, ops[i].c_liv,
                            ops[i].c_val, caps[i], base + solo[i], nb, s);
    });
}

int32_t lco_batch_results(const lco_batch *b, const int64_t *caps, const void *ws, lco_contract_result *out,
                          void *stream) {
    if (!b || !ws || !out) return LCO_ERR_INVALID;
    std::vector<size_t> offs;
    size_t total = 0;
    int32_t rc = layout(b, caps, offs, &total);
    if (rc != LCO_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCO_ERR_CUDA;
    const char *base = reinterpret_cast<const char *>(ws);
    if (b->stacked_last && caps) {
        // the stacked path leaves one result record per member of each group
        std::vector<size_t> goffs, solo;
        std::vector<GroupLayout> gl;
        size_t st = 0;
        if ((rc = stacked_layout(b, caps, goffs, gl, solo, &st)) != LCO_OK) return rc;
        std::vector<lco_contract_result> tmp;
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            const Group &g = b->groups[gi];
            tmp.resize(g.members.size());
            if (cudaMemcpy(tmp.data(), base + goffs[gi] + gl[gi].res, tmp.size() * sizeof(lco_contract_result),
                           cudaMemcpyDeviceToHost) != cudaSuccess)
                return LCO_ERR_CUDA;
            for (size_t h = 0; h < g.members.size(); ++h) out[g.members[h]] = tmp[h];
        }
        for (int32_t i : b->solo) {
            if ((rc = lco_contract_result_get(base + solo[i], &out[i], stream)) != LCO_OK) return rc;
        }
        return LCO_OK;
    }
    for (int i = 0; i < b->nprob; ++i) {
        rc = lco_contract_result_get(base + offs[i], &out[i], stream);
        if (rc != LCO_OK) return rc;
    }
    return LCO_OK;
}

}  // extern "C"
