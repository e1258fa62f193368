"""Pins for the oracle's contraction, flop count and Table-4 dispatch (Sec. 5).
CPU only."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth


def _dense(T):
    a = np.zeros(T["dims"])
    co = oracle.delinearise(T["dims"], T["sig"], T["liv"])
    a[tuple(co.T)] = T["val"]
    return a


def _mask(T):
    a = np.zeros(T["dims"])
    co = oracle.delinearise(T["dims"], T["sig"], T["liv"])
    a[tuple(co.T)] = 1.0
    return a


def _einsum_spec(order_a, order_b, modes_a, modes_b):
    letters = "abcdefghijklmnopqrstuvwxyz"
    la = list(letters[:order_a])
    lb = list(letters[order_a:order_a + order_b])
    for ma, mb in zip(modes_a, modes_b):
        lb[mb] = la[ma]
    free_a = [la[t] for t in range(order_a) if t not in modes_a]
    free_b = [lb[t] for t in range(order_b) if t not in modes_b]
    return "".join(la) + "," + "".join(lb) + "->" + "".join(free_a + free_b)


def _check_against_einsum(A, B, ma, mb):
    liv, val, ab = oracle.contract(A, B, ma, mb)
    spec = _einsum_spec(len(A["dims"]), len(B["dims"]), ma, mb)
    dense = np.einsum(spec, _dense(A), _dense(B))
    count = np.einsum(spec, _mask(A), _mask(B))       # number of products per entry
    absd = np.einsum(spec, np.abs(_dense(A)), np.abs(_dense(B)))
    out_dims = [A["dims"][t] for t in range(len(A["dims"])) if t not in ma] + \
               [B["dims"][t] for t in range(len(B["dims"])) if t not in mb]
    if len(out_dims) == 0:
        expect_liv = np.array([0], np.int64) if count > 0 else np.empty(0, np.int64)
        expect_val = np.array([dense]) if count > 0 else np.empty(0)
    else:
        nzs = np.argwhere(count > 0)
        expect_liv = np.ravel_multi_index(tuple(nzs.T), out_dims).astype(np.int64) if nzs.size else \
            np.empty(0, np.int64)
        expect_val = dense[tuple(nzs.T)] if nzs.size else np.empty(0)
        absd = absd[tuple(nzs.T)] if nzs.size else np.empty(0)
    order = np.argsort(expect_liv)
    assert np.array_equal(liv, expect_liv[order])                 # pattern: exact
    assert np.all(np.abs(val - expect_val[order]) <= 1e-13 * np.maximum(absd[order] if np.ndim(absd) else absd, 1e-300))
    assert np.allclose(ab, absd[order] if np.ndim(absd) else absd, rtol=1e-13, atol=0)
    f = oracle.flops(A, B, ma, mb)
    assert f == int(round(float(np.sum(count))))
    return liv, val


def _partial_matchings(order_a, order_b):
    """All partial permutations between the modes of A and B (Sec. 3.1)."""
    out = []
    for i in range(0, min(order_a, order_b) + 1):
        for sa in itertools.combinations(range(order_a), i):
            for sb in itertools.permutations(range(order_b), i):
                out.append((list(sa), list(sb)))
    return out


def test_partial_permutation_count():
    """P = sum_i i! C(N,i)^2 (Sec. 3.1): 34 matchings for two order-3 tensors."""
    for N in range(1, 6):
        P = sum(math.factorial(i) * math.comb(N, i) ** 2 for i in range(N + 1))
        assert len(_partial_matchings(N, N)) == P
    assert len(_partial_matchings(3, 3)) == 34


def _rand_tensor(dims, density, rng, sig=None):
    total = int(np.prod(dims))
    nnz = max(1, int(total * density))
    liv = np.sort(rng.choice(total, size=nnz, replace=False)).astype(np.int64)
    T = {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
         "val": rng.uniform(-1, 1, nnz)}
    if sig is not None:
        lo, vo = oracle.permute(T["dims"], T["sig"], sig, T["liv"], T["val"])
        T = {"dims": list(dims), "sig": list(sig), "liv": lo, "val": vo}
    return T


def test_every_matching_of_order3_against_einsum():
    """Brute force: all 34 matchings of two 3x3x3 tensors, dense einsum as the reference."""
    rng = np.random.default_rng(7)
    A = _rand_tensor([3, 3, 3], 0.4, rng)
    B = _rand_tensor([3, 3, 3], 0.4, rng, sig=[1, 0, 2])     # B in a non-row-major order
    for ma, mb in _partial_matchings(3, 3):
        _check_against_einsum(A, B, ma, mb)


def test_mixed_orders_and_dims_against_einsum():
    rng = np.random.default_rng(8)
    A = _rand_tensor([2, 3, 4, 2], 0.5, rng, sig=[2, 0, 3, 1])
    B = _rand_tensor([4, 5, 2], 0.5, rng)
    for ma, mb in [([2], [0]), ([2, 3], [0, 2]), ([0, 2], [2, 0]), ([], []), ([3, 0, 2], [2, 2, 0])]:
        if len(set(mb)) != len(mb):
            continue
        _check_against_einsum(A, B, ma, mb)


def test_laplacian_squared_closed_form():
    """The 5-point Laplacian composed with itself on 16x16 (Dirichlet) is the
    13-point biharmonic stencil: diagonal 16 + deg(p) (20 interior, 19 edge,
    18 corner), -8 at axial distance 1, 2 at diagonal, 1 at axial distance 2."""
    cfg = synth.config_fd2d(16)
    liv, val, ab = oracle.contract(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert liv.shape[0] == 3012
    assert oracle.flops(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"]) == 5832
    co = np.stack(np.unravel_index(liv, [16] * 4), 1)
    i, j, k, l = co.T
    di, dj = k - i, l - j
    deg = (i > 0).astype(int) + (i < 15) + (j > 0) + (j < 15)
    expect = np.full(liv.shape[0], np.nan)
    diag = (di == 0) & (dj == 0)
    expect[diag] = 16 + deg[diag]
    expect[(np.abs(di) + np.abs(dj) == 1)] = -8
    expect[(np.abs(di) == 1) & (np.abs(dj) == 1)] = 2
    expect[((np.abs(di) == 2) & (dj == 0)) | ((np.abs(dj) == 2) & (di == 0))] = 1
    assert not np.any(np.isnan(expect))
    assert np.array_equal(val, expect)            # small integers: bit-exact
    counts = {20: 196, 19: 56, 18: 4}
    for v, c in counts.items():
        assert int(np.sum(diag & (val == v))) == c
    assert int(np.sum(val == -8)) == 960 and int(np.sum(val == 2)) == 900
    assert int(np.sum(val == 1)) == 896


def test_fd_matrix_exact_on_quadratics():
    """Eq. 1 is O(h^2): it differentiates x^2 exactly on every row, boundary
    rows included (this pins the sign reading of the last row)."""
    for N in (3, 5, 11):
        r, c, v = synth.fd_matrix_entries(N)
        D = sp.csr_matrix((v, (r, c)), shape=(N, N))
        x = np.arange(N, dtype=float)
        assert np.allclose(D @ (x ** 2), 2 * x, rtol=0, atol=1e-12)
        assert np.allclose(D @ x, np.ones(N), rtol=0, atol=1e-12)


def _stencil_of(T, center):
    """Offsets and coefficients of a stencil operator's row at an interior point."""
    d = len(T["dims"]) // 2
    co = np.stack(np.unravel_index(T["liv"], T["dims"]), 1)
    rows = np.all(co[:, :d] == np.asarray(center)[None, :], axis=1)
    return {tuple((co[e, d:] - co[e, :d]).tolist()): T["val"][e] for e in np.nonzero(rows)[0]}


def test_stencil_composition_interior_closed_form():
    """Interior rows of a composition of constant stencils are the
    convolution of the two stencils (the 7-point Laplacian after an Eq. 1
    x-derivative on 8^3)."""
    n = 8
    L = synth.laplacian((n, n, n))
    D = synth.derivative_x((n, n, n), coeffs="eq1")
    liv, val, _ = oracle.contract(L, D, [3, 4, 5], [0, 1, 2])
    sl = _stencil_of(L, (4, 4, 4))
    sd = _stencil_of(D, (4, 4, 4))
    conv = {}
    for o1, c1 in sl.items():
        for o2, c2 in sd.items():
            o = tuple(a + b for a, b in zip(o1, o2))
            conv[o] = conv.get(o, 0.0) + c1 * c2
    C = {"dims": [n] * 6, "liv": liv, "val": val}
    got = _stencil_of(C, (4, 4, 4))
    assert set(got) == set(conv)          # structural zeros (the diagonal) are kept
    for o in conv:
        assert abs(got[o] - conv[o]) <= 1e-15
    assert got[(0, 0, 0)] == 0.0


def test_freivalds_probe_fd3d_small():
    """C x = A (B x) for random x, with A, B, C as scipy CSR matrices (Freivalds)."""
    cfg = synth.config_fd3d(n=10, seed=2)
    A, B = cfg["A"], cfg["B"]
    liv, val, ab = oracle.contract(A, B, cfg["modes_a"], cfg["modes_b"])
    m = k = n = 1000
    Am = sp.csr_matrix((A["val"], (A["liv"] // k, A["liv"] % k)), shape=(m, k))
    Bm = sp.csr_matrix((B["val"], (B["liv"] // n, B["liv"] % n)), shape=(k, n))
    Cm = sp.csr_matrix((val, (liv // n, liv % n)), shape=(m, n))
    x = np.random.default_rng(0).standard_normal(n)
    absC = sp.csr_matrix((ab, (liv // n, liv % n)), shape=(m, n))
    err = np.abs(Cm @ x - Am @ (Bm @ x))
    bound = 1e-13 * (abs(Am) @ (abs(Bm) @ np.abs(x))) + 1e-13 * (absC @ np.abs(x))
    assert np.all(err <= bound + 1e-300)


def test_empty_operands():
    A = {"dims": [3, 3], "sig": [1, 0], "liv": np.empty(0, np.int64), "val": np.empty(0)}
    B = {"dims": [3, 3], "sig": [1, 0], "liv": np.array([0, 4], np.int64), "val": np.array([1.0, 2.0])}
    liv, val, ab = oracle.contract(A, B, [1], [0])
    assert liv.shape[0] == 0
    liv, val, ab = oracle.contract(B, A, [1], [0])
    assert liv.shape[0] == 0


def test_mismatched_dims_rejected():
    A = {"dims": [3, 4], "sig": [1, 0], "liv": np.array([1], np.int64), "val": np.array([1.0])}
    with pytest.raises(oracle.OracleError):
        oracle.contract(A, A, [1], [1 - 1 + 0])        # 4 vs 3


# --------------------------- Table 4 dispatch ---------------------------

# (A class, B class) -> cell, classes in order S, R, C, I (Table 4)
TABLE4 = {
    ("S", "S"): "CSC/CSR", ("S", "R"): "CSC", ("S", "C"): "CSC", ("S", "I"): "CSC",
    ("C", "S"): "CSR", ("C", "R"): "DCSC/DCSR", ("C", "C"): "DCSC", ("C", "I"): "DCSC",
    ("R", "S"): "CSR", ("R", "R"): "DCSR", ("R", "C"): "CSCNA/CSRNA", ("R", "I"): "CSCNA",
    ("I", "S"): "CSR", ("I", "R"): "DCSR", ("I", "C"): "CSRNA", ("I", "I"): "SOP",
}


def _shape_for(ca, cb, base=1000):
    """m, k, n, nnz_a, nnz_b realising the requested classes (ratio 10 vs 1)."""
    nnz = base
    m = 10 * nnz if ca in ("R", "I") else nnz
    k_a = ca in ("C", "I")
    k_b = cb in ("R", "I")
    n = 10 * nnz if cb in ("C", "I") else nnz
    # k is shared; choose nnz_a, nnz_b so that k/nnz hits the wanted side for each
    k = 10 * nnz
    nnz_a = nnz if k_a else 10 * nnz
    nnz_b = nnz if k_b else 10 * nnz
    if ca in ("R", "I"):
        m = 10 * nnz_a
    else:
        m = nnz_a
    if cb in ("C", "I"):
        n = 10 * nnz_b
    else:
        n = nnz_b
    return m, k, n, nnz_a, nnz_b


@pytest.mark.parametrize("ca,cb", list(TABLE4))
def test_table4_cells(ca, cb):
    m, k, n, na, nb = _shape_for(ca, cb)
    names = "SRCI"
    assert names[oracle.sparsity_class(m, k, na)] == ca
    assert names[oracle.sparsity_class(k, n, nb)] == cb
    cell = TABLE4[(ca, cb)]
    if "/" in cell:
        col, row = cell.split("/")
        # fewer rearrangements decides ...
        assert oracle.dispatch(m, k, n, na, nb, perm_row=0, perm_col=1) == row
        assert oracle.dispatch(m, k, n, na, nb, perm_row=2, perm_col=1) == col
        # ... and with a tie the column variant is chosen iff n > m
        expect = col if n > m else row
        assert oracle.dispatch(m, k, n, na, nb, 1, 1) == expect
    else:
        for pr, pc in [(0, 0), (0, 2), (2, 0)]:
            assert oracle.dispatch(m, k, n, na, nb, pr, pc) == cell


def test_ratio_threshold_is_three():
    """dim/nnz > 3 is hyper-sparse; exactly 3 is not (Secs. 5.2.3-5.2.5)."""
    assert oracle.sparsity_class(300, 10, 100) == 0
    assert oracle.sparsity_class(301, 10, 100) == 1
    assert oracle.sparsity_class(10, 301, 100) == 2
    assert oracle.sparsity_class(301, 301, 100) == 3
    assert oracle.sparsity_class(5, 5, 0) == 3


def test_orientation_tie_break():
    """n > m picks the column variant, otherwise the row variant (Sec. 5.2.2)."""
    assert oracle.dispatch(100, 100, 101, 1000, 1000) == "CSC"
    assert oracle.dispatch(100, 100, 100, 1000, 1000) == "CSR"
    assert oracle.dispatch(101, 100, 100, 1000, 1000) == "CSR"


def test_configs_take_the_named_branches():
    """The workloads exercise the branches they are meant to: 2D/3D FD -> CSR,
    the R-MAT a_ijk b_ljk form -> DCSR, the mode-2 x mode-0 form -> CSRNA."""
    assert oracle.dispatch(256, 256, 256, 1216, 1216, 0, 2) == "CSR"
    assert oracle.dispatch(1 << 18, 1 << 18, 1 << 18, 1810432, 532480, 0, 2) == "CSR"
    assert oracle.dispatch(1 << 20, 1 << 32, 1 << 20, 10_000_000, 10_000_000, 1, 1) == "DCSR"
    assert oracle.dispatch(1 << 28, 1 << 12, 1 << 28, 1 << 18, 1 << 18, 0, 2) == "CSRNA"


def _rt(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, liv.shape[0])}


def _as_tensor(dims, liv, val):
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv, "val": val}


def test_chained_products_associate():
    """(A x B) x C = A x (B x C) for a chain of matrix-like contractions: the
    output mode order (A's free modes, then B's) must line up across both
    groupings.  Entry patterns agree exactly; values to rounding."""
    A = _rt([6, 7, 5], 90, 101)          # (i, j, k)
    B = _rt([5, 8], 25, 102)             # (k, l)
    Cm = _rt([8, 4, 3], 60, 103)         # (l, m, n)
    l1, v1, _ = oracle.contract(A, B, [2], [0])                        # (i, j, l)
    left = oracle.contract(_as_tensor([6, 7, 8], l1, v1), Cm, [2], [0])  # (i, j, m, n)
    l2, v2, _ = oracle.contract(B, Cm, [1], [0])                       # (k, m, n)
    right = oracle.contract(A, _as_tensor([5, 4, 3], l2, v2), [2], [0])  # (i, j, m, n)
    dense_left = np.zeros([6, 7, 4, 3]); dense_right = np.zeros([6, 7, 4, 3])
    dense_left.reshape(-1)[left[0]] = left[1]
    dense_right.reshape(-1)[right[0]] = right[1]
    assert np.allclose(dense_left, dense_right, rtol=0, atol=1e-12)


def test_swapping_operands_transposes_the_product():
    """contract(B, A) has B's free modes first; moving them behind A's gives
    contract(A, B) exactly (same products, same summation order per entry)."""
    A = _rt([5, 6, 4], 70, 111)          # (i, k, j)
    B = _rt([6, 3, 7], 60, 112)          # (k, l, m)
    la, va, _ = oracle.contract(A, B, [1], [0])   # (i, j, l, m)
    lb, vb, _ = oracle.contract(B, A, [0], [1])   # (l, m, i, j)
    # (l, m, i, j) row-major -> (i, j, l, m) row-major: sig lists modes least significant first
    lt, vt = oracle.permute([3, 7, 5, 4], [3, 2, 1, 0], [1, 0, 3, 2], lb, vb)
    assert np.array_equal(lt, la)
    assert np.allclose(vt, va, rtol=0, atol=1e-15)


def test_contraction_is_bilinear():
    """contract(A + 2 A', B) = contract(A, B) + 2 contract(A', B), with the
    sum taken by the oracle's add: catches dropped terms and sign errors."""
    A = _rt([4, 6], 14, 121)
    A2 = _rt([4, 6], 12, 122)
    B = _rt([6, 5], 16, 123)
    s_liv, s_val = oracle.add(1.0, A, 2.0, A2)
    lhs_l, lhs_v, _ = oracle.contract(_as_tensor([4, 6], s_liv, s_val), B, [1], [0])
    l1, v1, _ = oracle.contract(A, B, [1], [0])
    l2, v2, _ = oracle.contract(A2, B, [1], [0])
    rhs_l, rhs_v = oracle.add(1.0, _as_tensor([4, 5], l1, v1), 2.0, _as_tensor([4, 5], l2, v2))
    d_l = np.zeros(20); d_r = np.zeros(20)
    d_l[lhs_l] = lhs_v
    d_r[rhs_l] = rhs_v
    assert np.allclose(d_l, d_r, rtol=0, atol=1e-13)
