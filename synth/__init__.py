"""Seeded synthetic inputs for the LCO hot path.

This package is shared by the tests, the benchmark and the oracle checks.  It
holds none of the method's arithmetic: it only draws coordinates and values
and hands them over as sorted LCO tensors, using numpy's own row-major
``ravel_multi_index`` for the input LIVs.  Every generator is deterministic in
its seed.

Tensors are dicts: ``dims`` (int64 list), ``sig`` (least significant mode
first; row-major is ``[order-1, ..., 0]``), ``liv`` (int64, strictly
ascending) and ``val`` (float64).

Workloads (the paper's own workloads are synthetic too):

* finite-difference operators built from the FD matrix of Eq. 1 and the
  5-/7-point Laplacians of the differential-operator example (Sec. 2);
* order-3 R-MAT ("R-TENSOR", Sec. 5.2.1) tensors from recursive per-bit-level
  probabilities.
"""
from __future__ import annotations

import numpy as np


def row_major_sig(order):
    return list(range(order - 1, -1, -1))


def _pack(dims, coords, vals):
    """Sort entries row-major and return an LCO dict.  coords: (nnz, order)."""
    dims = [int(d) for d in dims]
    coords = np.asarray(coords, dtype=np.int64).reshape(-1, len(dims))
    vals = np.asarray(vals, dtype=np.float64).reshape(-1)
    if coords.shape[0]:
        liv = np.ravel_multi_index(tuple(coords.T), dims).astype(np.int64)
    else:
        liv = np.empty(0, np.int64)
    order = np.argsort(liv, kind="stable")
    liv, vals = liv[order], vals[order]
    if liv.size > 1 and np.any(liv[1:] == liv[:-1]):
        raise ValueError("duplicate coordinates")
    return {"dims": dims, "sig": row_major_sig(len(dims)), "liv": liv, "val": vals}


# ---------------------------------------------------------------------------
# Finite-difference operators
# ---------------------------------------------------------------------------

def fd_matrix_entries(N, coeffs="eq1", rng=None):
    """Entries (row, col, value) of the N x N FD matrix of Eq. 1.

    Interior rows use the O(h^2) central difference (-1/2, +1/2); row 0 the
    forward one-sided difference (-3, 4, -1)/2 and row N-1 the backward
    one-sided difference (1, -4, 3)/2 (the printed last row has its sign
    flipped; this is the O(h^2) backward difference the text names).
    ``coeffs="uniform"`` replaces every value by an independent U(-1,1) draw
    from ``rng`` (same pattern).
    """
    if N < 3:
        raise ValueError("Eq. 1 needs N >= 3")
    rows, cols, vals = [], [], []
    rows += [0, 0, 0]; cols += [0, 1, 2]; vals += [-1.5, 2.0, -0.5]
    for i in range(1, N - 1):
        rows += [i, i]; cols += [i - 1, i + 1]; vals += [-0.5, 0.5]
    rows += [N - 1] * 3; cols += [N - 3, N - 2, N - 1]; vals += [0.5, -2.0, 1.5]
    rows, cols, vals = np.array(rows, np.int64), np.array(cols, np.int64), np.array(vals)
    if coeffs == "uniform":
        vals = rng.uniform(-1.0, 1.0, size=vals.shape[0])
    elif coeffs != "eq1":
        raise ValueError(coeffs)
    return rows, cols, vals


def laplacian(shape, center=None, neighbor=1.0):
    """Dirichlet Laplacian on a grid of ``shape`` as a 2*d-order tensor.

    Entry [p, q] (output point p, input point q) is ``center`` (default -2d)
    on the diagonal and ``neighbor`` for every in-grid axis neighbour; points
    outside the grid are dropped.  2D gives the 5-point -4/1 operator, 3D the
    7-point -6/1 operator.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    if center is None:
        center = -2.0 * d
    pts = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, d)
    coords, vals = [np.concatenate([pts, pts], 1)], [np.full(pts.shape[0], center)]
    for ax in range(d):
        for step in (-1, 1):
            q = pts.copy()
            q[:, ax] += step
            ok = (q[:, ax] >= 0) & (q[:, ax] < shape[ax])
            coords.append(np.concatenate([pts[ok], q[ok]], 1))
            vals.append(np.full(int(ok.sum()), neighbor))
    return _pack(list(shape) * 2, np.concatenate(coords), np.concatenate(vals))


def stencil_operator(shape, offsets, coeffs):
    """Constant-coefficient stencil operator on a grid as a 2*d-order tensor:
    [p, p + o] = c for each offset o with p + o inside the grid."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    pts = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, d)
    coords, vals = [], []
    for off, c in zip(offsets, coeffs):
        q = pts + np.asarray(off, np.int64)[None, :]
        ok = np.all((q >= 0) & (q < np.asarray(shape)[None, :]), axis=1)
        coords.append(np.concatenate([pts[ok], q[ok]], 1))
        vals.append(np.full(int(ok.sum()), float(c)))
    return _pack(list(shape) * 2, np.concatenate(coords), np.concatenate(vals))


def derivative_x(shape, coeffs="eq1", seed=None):
    """FD first derivative along the first grid axis as a 2*d-order tensor:
    D[x, y.., x', y'..] = delta(y, y') * Eq.1[x, x'].  ``coeffs="uniform"``
    gives every non-zero an independent U(-1,1) value (seeded)."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed) if coeffs == "uniform" else None
    r, c, v = fd_matrix_entries(shape[0], "eq1")
    rest = np.stack(np.meshgrid(*[np.arange(s) for s in shape[1:]], indexing="ij"), -1)
    rest = rest.reshape(-1, len(shape) - 1)
    nrest = rest.shape[0]
    # entries ordered (rest point, Eq.1 entry) so that the uniform draws are reproducible
    R = np.repeat(rest, r.shape[0], axis=0)
    rr, cc, vv = np.tile(r, nrest), np.tile(c, nrest), np.tile(v, nrest)
    if rng is not None:
        vv = rng.uniform(-1.0, 1.0, size=vv.shape[0])
    coords = np.concatenate([rr[:, None], R, cc[:, None], R], 1)
    return _pack(list(shape) * 2, coords, vv)


# ---------------------------------------------------------------------------
# R-MAT order-3 tensors
# ---------------------------------------------------------------------------

RMAT_PROBS = (0.45, 0.15, 0.15, 0.25)


def rmat3(bits, nnz, seed, probs=RMAT_PROBS, jitter=False):
    """Order-3 R-MAT tensor with dims (2^bits[0], 2^bits[1], 2^bits[2]).

    Bits are drawn level by level from the most significant one.  At a level
    where modes 0 and 1 both still have bits, (b0, b1) is drawn from
    ``probs`` over (0,0), (0,1), (1,0), (1,1); where only one of them has a
    bit it is drawn from that mode's marginal.  Mode 2's bits are aligned to
    the top levels; its bit is drawn from the row of ``probs`` selected by b0
    (normalised), or from the marginal of mode 0 when mode 0 has no bit at
    that level.  ``jitter`` adds U(-0.1, 0.1) to each probability once per
    tensor and renormalises (the R-TENSOR variability of Sec. 5.2.1).
    Duplicate coordinates are dropped, keeping the first draw, until exactly
    ``nnz`` distinct entries remain.  Values are U(-1, 1).
    """
    rng = np.random.default_rng(seed)
    p = np.asarray(probs, dtype=np.float64)
    if jitter:
        p = np.clip(p + rng.uniform(-0.1, 0.1, size=4), 1e-6, None)
    p = p / p.sum()
    cum = np.cumsum(p)
    p0_zero = p[0] + p[1]
    p1_zero = p[0] + p[2]
    p2_given = (p[0] / (p[0] + p[1]), p[2] / (p[2] + p[3]))
    bits = [int(b) for b in bits]
    dims = [1 << b for b in bits]
    L = max(bits)

    def draw(count):
        co = np.zeros((count, 3), dtype=np.int64)
        for t in range(L):
            act = [t < b for b in bits]
            b0 = b1 = None
            if act[0] and act[1]:
                q = np.searchsorted(cum, rng.random(count), side="right")
                q = np.minimum(q, 3)
                b0, b1 = q >> 1, q & 1
            elif act[0]:
                b0 = (rng.random(count) >= p0_zero).astype(np.int64)
            elif act[1]:
                b1 = (rng.random(count) >= p1_zero).astype(np.int64)
            if act[2]:
                u = rng.random(count)
                if b0 is not None:
                    thr = np.where(b0 == 0, p2_given[0], p2_given[1])
                else:
                    thr = np.full(count, p0_zero)
                b2 = (u >= thr).astype(np.int64)
                co[:, 2] |= b2 << (bits[2] - 1 - t)
            if b0 is not None:
                co[:, 0] |= b0.astype(np.int64) << (bits[0] - 1 - t)
            if b1 is not None:
                co[:, 1] |= b1.astype(np.int64) << (bits[1] - 1 - t)
        vals = rng.uniform(-1.0, 1.0, size=count)
        return co, vals

    all_co, all_val = np.empty((0, 3), np.int64), np.empty(0)
    need = nnz
    while True:
        co, vals = draw(int(need * 1.05) + 64)
        all_co = np.concatenate([all_co, co])
        all_val = np.concatenate([all_val, vals])
        liv = np.ravel_multi_index(tuple(all_co.T), dims).astype(np.int64)
        _, first = np.unique(liv, return_index=True)
        if first.shape[0] >= nnz:
            keep = np.sort(first)[:nnz]
            return _pack(dims, all_co[keep], all_val[keep])
        need = nnz - first.shape[0]


def rotate_modes(T, shift):
    """Re-label the modes of a row-major tensor: new mode t = old mode (t + shift) % order."""
    order = len(T["dims"])
    co = np.stack(np.unravel_index(T["liv"], T["dims"]), 1)
    perm = [(t + shift) % order for t in range(order)]
    return _pack([T["dims"][q] for q in perm], co[:, perm], T["val"])


# ---------------------------------------------------------------------------
# The benchmark configurations
# ---------------------------------------------------------------------------

def config_fd2d(n=16):
    """2D 5-point Dirichlet Laplacian on n x n composed with itself:
    A[i,j,k,l] contracted over (k,l) with A over (i,j)."""
    A = laplacian((n, n))
    return {"name": f"fd2d_laplacian_sq_{n}x{n}", "A": A, "B": A,
            "modes_a": [2, 3], "modes_b": [0, 1]}


def config_fd3d(n=64, seed=2):
    """3D 7-point Laplacian on n^3 composed with a seeded U(-1,1) x-derivative
    (Eq. 1 pattern along the first axis), plus the permutation of the result
    to mode order (k,l,m,i,j,n) (listed most significant first)."""
    L = laplacian((n, n, n))
    D = derivative_x((n, n, n), coeffs="uniform", seed=seed)
    # (k,l,m,i,j,n) most significant first = modes 2,3,4,0,1,5; sig is least significant first
    return {"name": f"fd3d_laplacian_dx_{n}^3", "A": L, "B": D,
            "modes_a": [3, 4, 5], "modes_b": [0, 1, 2],
            "permute_sig": [5, 1, 0, 4, 3, 2]}


def config_rmat_dcsr(bits=(20, 20, 12), nnz=10_000_000, seeds=(3, 4)):
    """R-MAT order-3 pair contracted over modes {1,2} x {1,2} (a_ijk b_ljk,
    the column-sparse x row-sparse form): the DCSR branch."""
    A = rmat3(bits, nnz, seeds[0])
    B = rmat3(bits, nnz, seeds[1])
    return {"name": f"rmat_{'x'.join(str(1 << b) for b in bits)}_{nnz}_a_ijk_b_ljk",
            "A": A, "B": B, "modes_a": [1, 2], "modes_b": [1, 2]}


def config_rmat_na(bits=(14, 14, 12), nnz=1 << 18, seeds=(5, 6)):
    """R-MAT order-3 pair with mode 2 of A contracted with mode 0 of B, where
    B is the same generator with its modes rotated so that the contracted
    mode comes first: the row-sparse x column-sparse (CSRNA) branch."""
    A = rmat3(bits, nnz, seeds[0])
    B = rotate_modes(rmat3(bits, nnz, seeds[1]), 2)
    return {"name": f"rmat_{'x'.join(str(1 << b) for b in bits)}_{nnz}_mode2_x_mode0",
            "A": A, "B": B, "modes_a": [2], "modes_b": [0]}


# ---------------------------------------------------------------------------
# Batched workload: uneven FD compositions and R-MAT products
# ---------------------------------------------------------------------------

STENCIL_2D = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
STENCIL_3D = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


def rmat3_torch(bits, nnz, seed, device="cuda", probs=RMAT_PROBS):
    """rmat3's distribution drawn with torch's seeded generator on `device`
    (fast for many large tensors; a different random stream from rmat3)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    p = torch.tensor(probs, dtype=torch.float64)
    p = p / p.sum()
    cum = torch.cumsum(p, 0).to(device)
    p0_zero, p1_zero = float(p[0] + p[1]), float(p[0] + p[2])
    p2_given = (float(p[0] / (p[0] + p[1])), float(p[2] / (p[2] + p[3])))
    bits = [int(b) for b in bits]
    dims = [1 << b for b in bits]
    L = max(bits)

    def draw(count):
        co = torch.zeros((count, 3), dtype=torch.int64, device=device)
        for t in range(L):
            act = [t < b for b in bits]
            b0 = b1 = None
            if act[0] and act[1]:
                q = torch.searchsorted(cum, torch.rand(count, generator=g, device=device, dtype=torch.float64),
                                       right=True).clamp_(max=3)
                b0, b1 = q >> 1, q & 1
            elif act[0]:
                b0 = (torch.rand(count, generator=g, device=device, dtype=torch.float64) >= p0_zero).long()
            elif act[1]:
                b1 = (torch.rand(count, generator=g, device=device, dtype=torch.float64) >= p1_zero).long()
            if act[2]:
                u = torch.rand(count, generator=g, device=device, dtype=torch.float64)
                if b0 is not None:
                    thr = torch.where(b0 == 0, p2_given[0], p2_given[1])
                else:
                    thr = torch.full((count,), p0_zero, device=device, dtype=torch.float64)
                co[:, 2] |= (u >= thr).long() << (bits[2] - 1 - t)
            if b0 is not None:
                co[:, 0] |= b0 << (bits[0] - 1 - t)
            if b1 is not None:
                co[:, 1] |= b1 << (bits[1] - 1 - t)
        vals = torch.rand(count, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0
        return co, vals

    all_liv = torch.empty(0, dtype=torch.int64, device=device)
    all_val = torch.empty(0, dtype=torch.float64, device=device)
    need = nnz
    while True:
        co, vals = draw(int(need * 1.05) + 64)
        liv = (co[:, 0] * dims[1] + co[:, 1]) * dims[2] + co[:, 2]
        all_liv = torch.cat([all_liv, liv])
        all_val = torch.cat([all_val, vals])
        order = torch.sort(all_liv, stable=True).indices
        s = all_liv[order]
        first = torch.ones_like(s, dtype=torch.bool)
        first[1:] = s[1:] != s[:-1]
        keep = order[first]                     # first draw of every distinct LIV
        if keep.numel() >= nnz:
            keep = torch.sort(keep).values[:nnz]
            liv, val = all_liv[keep], all_val[keep]
            o = torch.argsort(liv)
            return {"dims": dims, "sig": [2, 1, 0], "liv": liv[o], "val": val[o]}
        need = nnz - keep.numel()


def _log_uniform(rng, lo, hi):
    return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))


BATCH_KINDS = ("fd2d", "fd3d", "rmat_eq14", "rmat_eq16", "rmat_sop")


def batch_item(i, count, seed, attempt=0, fd2d=(16, 256), fd3d=(8, 40), rmat_nnz=(1e3, 1e6),
               ratio=(1.0, 500.0), device="cuda"):
    """Item i of a batch of `count` (see batch_problems), drawn from its own
    seed sequence (seed, i, attempt) so that any item can be redrawn alone."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(i), int(attempt)]))
    if i < count // 4:
        n = int(round(_log_uniform(rng, *fd2d)))
        A = stencil_operator((n, n), STENCIL_2D, rng.uniform(-1, 1, len(STENCIL_2D)))
        return A, A, [2, 3], [0, 1], "fd2d"
    if i < count // 2:
        n = int(round(_log_uniform(rng, *fd3d)))
        A = stencil_operator((n, n, n), STENCIL_3D, rng.uniform(-1, 1, len(STENCIL_3D)))
        return A, A, [3, 4, 5], [0, 1, 2], "fd3d"
    form = int(rng.integers(0, 3))
    nnz = int(_log_uniform(rng, *rmat_nnz))
    rho = _log_uniform(rng, *ratio)
    s1, s2 = int(rng.integers(0, 2**31)), int(rng.integers(0, 2**31))
    if form < 2:
        # a_ijk with three equal dims; contracted dims (j,k) or (k) give the ratio
        b = max(2, int(np.ceil(np.log2(np.sqrt(rho * nnz)))))
        bits = (b, b, b)
    else:
        # M x N x N with M = N^2 (Sec. 5.2.5): flattened as in Eq. 14 both
        # operands are N^2 x N^2 with row- and column-sparsity N^2 / nnz
        b = max(2, int(np.ceil(np.log2(rho * nnz) / 2)))
        bits = (2 * b, b, b)
    A = rmat3_torch(bits, nnz, s1, device)
    B = rmat3_torch(bits, nnz, s2, device)
    if form == 1:
        return A, B, [2], [2], "rmat_eq16"
    return A, B, [1, 2], [1, 2], ("rmat_eq14" if form == 0 else "rmat_sop")


def batch_problems(count=4096, seed=100, admit=None, max_attempts=64, **kw):
    """The batched workload: count/4 2D and count/4 3D FD operators with one
    U(-1,1) coefficient per stencil position, each composed with itself over
    its input-grid modes (grid sides log-uniform), and count/2 R-MAT pairs in
    one of the paper's three forms -- a_ijk b_ljk (Eq. 14), a_ijk b_lmk
    (Eq. 16) or M x N x N with M = N^2 (Sec. 5.2.5) -- with nnz log-uniform
    and hyper-sparsity ratio log-uniform.  `admit(A, B, modes_a, modes_b)`,
    when given, decides whether a drawn item is kept; a rejected item is
    redrawn from the next attempt's seed.  Returns (A, B, modes_a, modes_b,
    kind) tuples; R-MAT tensors live on `device` as torch tensors, FD ones
    as numpy arrays.  Keyword arguments go to batch_item."""
    out = []
    for i in range(count):
        for attempt in range(max_attempts):
            item = batch_item(i, count, seed, attempt, **kw)
            if admit is None or admit(*item[:4]):
                out.append(item)
                break
        else:
            raise RuntimeError(f"batch item {i}: no admissible draw in {max_attempts} attempts")
    return out


# ---------------------------------------------------------------------------
# The combinatorial Laplacian of Eq. 4 (Sec. 2, Sec. 6)
# ---------------------------------------------------------------------------

def fd_matrix(N):
    """The N x N FD matrix of Eq. 1 as a second-order LCO tensor d[i, i']."""
    r, c, v = fd_matrix_entries(N, "eq1")
    return _pack([N, N], np.stack([r, c], 1), v)


def kronecker_delta(N):
    """delta[j, l] = 1 for j == l (N entries)."""
    i = np.arange(N, dtype=np.int64)
    return _pack([N, N], np.stack([i, i], 1), np.ones(N))


def quadratic_field(N):
    """x[k, l] = k^2 + l^2 on an N x N grid (every point an entry)."""
    k, l = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    co = np.stack([k.ravel(), l.ravel()], 1)
    return _pack([N, N], co, (k.ravel() ** 2 + l.ravel() ** 2).astype(np.float64))


def relabel(T, sig):
    """The same entries read with another significance order: the tensor
    whose mode m is T's mode m, with `sig` as its lexicographic order (no
    data moves; used to name a product's modes like another's)."""
    return {"dims": list(T["dims"]), "sig": list(sig), "liv": T["liv"], "val": T["val"]}


def config_eq17(N=2047):
    """Eq. 17, b_ii'jl d_i'k with b_ii'jl = d_ii' delta_jl (Sec. 6): b is an
    N^3 x N row-sparse matrix once flattened, d the N x N FD matrix of
    Eq. 1; b is built row-major (i, i', j, l), so the product first
    rearranges it (the rearrangement the paper's timing includes)."""
    r, c, v = fd_matrix_entries(N, "eq1")
    j = np.arange(N, dtype=np.int64)
    co = np.stack([np.repeat(r, N), np.repeat(c, N), np.tile(j, r.shape[0]), np.tile(j, r.shape[0])], 1)
    b = _pack([N] * 4, co, np.repeat(v, N))
    return {"name": f"eq17_b_d_N{N}", "A": b, "B": fd_matrix(N), "modes_a": [1], "modes_b": [0]}


def wide_tensor(dims, sig, nnz, seed):
    """A tensor whose dims multiply past 2^63 (wide LIVs: unsigned 128-bit,
    stored as an (nnz, 2) uint64 array, low word first): nnz distinct LIVs
    drawn uniformly from [0, prod dims), ascending, values U(-1, 1).  The
    LIVs are drawn directly (no coordinates); sig only labels the order."""
    total = 1
    for d in dims:
        total *= int(d)
    if total > (1 << 127) - 1:
        raise ValueError("dims multiply past 2^127 - 1")
    nnz = min(int(nnz), total)
    rng = np.random.default_rng(seed)
    hi_max = total >> 64
    got = np.empty((0, 2), dtype=np.uint64)
    while got.shape[0] < nnz:
        m = int((nnz - got.shape[0]) * 1.2) + 16
        lo = rng.integers(0, 1 << 64, size=m, dtype=np.uint64)
        hi = rng.integers(0, hi_max + 1, size=m, dtype=np.uint64) if hi_max > 0 else np.zeros(m, np.uint64)
        if hi_max == 0:
            lo = lo % np.uint64(total)
        # keep draws below total: only the top high word can overshoot
        top_lo = np.uint64(total & ((1 << 64) - 1))
        ok = (hi < np.uint64(hi_max)) | ((hi == np.uint64(hi_max)) & (lo < top_lo)) if hi_max > 0 else np.ones(m, bool)
        cand = np.concatenate([got, np.stack([lo[ok], hi[ok]], 1)])
        order = np.lexsort((cand[:, 0], cand[:, 1]))
        cand = cand[order]
        keep = np.ones(cand.shape[0], bool)
        keep[1:] = (cand[1:, 0] != cand[:-1, 0]) | (cand[1:, 1] != cand[:-1, 1])
        got = cand[keep]
    if got.shape[0] > nnz:
        pick = np.sort(rng.choice(got.shape[0], size=nnz, replace=False))
        got = got[pick]
    return {"dims": [int(d) for d in dims], "sig": list(sig), "liv": np.ascontiguousarray(got),
            "val": rng.uniform(-1, 1, nnz)}
