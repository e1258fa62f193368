"""GPU parity of the contraction (every poly-algorithm branch) against the
oracle: index patterns bit-exact, FP64 values within 1e-13 * sum |a||b|."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches, dev, host

pytestmark = pytest.mark.gpu

ALL_ALGS = list(lco.ALG_NAMES)


def _rand(dims, density, seed, sig=None, nnz=None):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    nnz = nnz if nnz is not None else max(1, int(total * density))
    if total <= 4 * nnz:
        liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False))
    else:
        liv = np.unique(rng.integers(0, total, size=int(nnz * 1.3) + 8))[:nnz]
    liv = np.sort(liv).astype(np.int64)
    T = {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
         "val": rng.uniform(-1, 1, liv.shape[0])}
    if sig is not None:
        lo, vo = oracle.permute(T["dims"], T["sig"], sig, T["liv"], T["val"])
        T = {"dims": list(dims), "sig": list(sig), "liv": lo, "val": vo}
    return T


def _run(A, B, ma, mb, alg=None):
    C, info = lco.contract(dev(A), dev(B), ma, mb, alg=alg, return_info=True)
    assert info["status"] == 0
    if alg is not None:
        assert info["alg"] == alg
    return C, info


def test_fd2d_laplacian_squared_closed_form_bit_exact():
    """16x16 5-point Laplacian composed with itself: 3012 entries of the
    13-point biharmonic stencil; small integers, so bit-exact."""
    cfg = synth.config_fd2d(16)
    C, info = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert info["alg"] == "CSR" and info["f"] == 5832 and info["nnz_c"] == 3012
    liv, val = host(C)
    rl, rv, _ = oracle.contract(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert np.array_equal(liv, rl) and np.array_equal(val, rv)


@pytest.mark.parametrize("alg", ALL_ALGS)
def test_every_branch_fd2d(alg):
    cfg = synth.config_fd2d(16)
    C, _ = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"], alg)
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"], tol=0.0)


@pytest.mark.parametrize("alg", ALL_ALGS)
def test_every_branch_random_mixed_orders(alg):
    A = _rand([6, 7, 8, 5], 0.15, 11, sig=[2, 0, 3, 1])
    B = _rand([8, 9, 6], 0.2, 12)
    for ma, mb in [([2], [0]), ([2, 0], [0, 2]), ([0, 2], [2, 0]), ([], [])]:
        C, _ = _run(A, B, ma, mb, alg)
        assert_contract_matches(C, A, B, ma, mb)


def test_all_34_matchings_order3():
    """Every partial permutation of modes between two 5x5x5 tensors (Sec. 3.1: 34 matchings)."""
    A = _rand([5, 5, 5], 0.3, 13)
    B = _rand([5, 5, 5], 0.3, 14, sig=[1, 2, 0])
    count = 0
    for i in range(4):
        for sa in itertools.combinations(range(3), i):
            for sb in itertools.permutations(range(3), i):
                C, _ = _run(A, B, list(sa), list(sb))
                assert_contract_matches(C, A, B, list(sa), list(sb))
                count += 1
    assert count == 34


@pytest.mark.parametrize("alg", ALL_ALGS)
def test_every_branch_hypersparse_rmat(alg):
    """Small R-MAT pair in the a_ijk b_ljk form (column-sparse x row-sparse)."""
    A = synth.rmat3((9, 9, 6), 20_000, 21)
    B = synth.rmat3((9, 9, 6), 20_000, 22)
    C, _ = _run(A, B, [1, 2], [1, 2], alg)
    assert_contract_matches(C, A, B, [1, 2], [1, 2])


@pytest.mark.parametrize("alg", ["CSRNA", "CSR", "SOP"])
def test_rmat_mode2_x_mode0_small(alg):
    cfg = synth.config_rmat_na(bits=(10, 10, 8), nnz=1 << 14, seeds=(5, 6))
    C, _ = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"], alg)
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])


def test_heavy_rows_take_the_spill_path():
    """Rows with thousands of products exceed the shared-memory chunk and are
    sorted and reduced in global scratch."""
    rng = np.random.default_rng(30)
    # A: 3 rows, each hitting 40 dense R rows of 300 entries -> 12000 products per row
    a_co = np.array([(r, c) for r in range(3) for c in range(0, 80, 2)])
    A = {"dims": [3, 80], "sig": [1, 0],
         "liv": np.ravel_multi_index(tuple(a_co.T), (3, 80)).astype(np.int64), "val": rng.uniform(-1, 1, len(a_co))}
    b_co = np.array([(c, j) for c in range(80) for j in rng.choice(1000, 300, replace=False)])
    b_liv = np.sort(np.ravel_multi_index(tuple(b_co.T), (80, 1000))).astype(np.int64)
    B = {"dims": [80, 1000], "sig": [1, 0], "liv": b_liv, "val": rng.uniform(-1, 1, len(b_liv))}
    for alg in ("CSR", "CSRNA", "DCSR"):
        C, info = _run(A, B, [1], [0], alg)
        assert info["f"] == 3 * 40 * 300
        assert_contract_matches(C, A, B, [1], [0])


def test_empty_and_disjoint():
    A = _rand([10, 10], 0.2, 40)
    E = {"dims": [10, 10], "sig": [1, 0], "liv": np.empty(0, np.int64), "val": np.empty(0)}
    C, info = _run(A, E, [1], [0])
    assert C.nnz == 0 and info["f"] == 0
    C, info = _run(E, A, [1], [0])
    assert C.nnz == 0
    # no matching contracted index at all
    A1 = {"dims": [4, 4], "sig": [1, 0], "liv": np.array([0, 4], np.int64), "val": np.array([1.0, 2.0])}
    B1 = {"dims": [4, 4], "sig": [1, 0], "liv": np.array([5, 6], np.int64), "val": np.array([1.0, 2.0])}
    C, info = _run(A1, B1, [1], [0])
    assert C.nnz == 0 and info["f"] == 0


def test_outer_and_full_contraction():
    A = _rand([6, 5], 0.4, 41)
    B = _rand([6, 5], 0.4, 42)
    C, _ = _run(A, B, [], [])                 # outer product, order 4
    assert_contract_matches(C, A, B, [], [])
    C, _ = _run(A, B, [0, 1], [0, 1])         # scalar
    assert_contract_matches(C, A, B, [0, 1], [0, 1])


def test_capacity_error_reported():
    cfg = synth.config_fd2d(8)
    A, B = dev(cfg["A"]), dev(cfg["B"])
    plan = lco.ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, cfg["modes_a"], cfg["modes_b"])
    plan.ensure_workspace(10)
    c_liv = torch.empty(10, dtype=torch.int64, device="cuda")
    c_val = torch.empty(10, dtype=torch.float64, device="cuda")
    plan.run(A, B, c_liv, c_val)
    r = plan.result()
    assert r["status"] == 8 and r["f"] > 10


def test_fd3d_full_size_against_oracle():
    """The 64^3 7-point Laplacian x seeded U(-1,1) x-derivative at full size,
    in the launch configuration the benchmark times, element by element."""
    cfg = synth.config_fd3d()
    C, info = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert info["alg"] == "CSR" and info["f"] == 3_669_504 and info["nnz_c"] == 3_382_784
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])


def test_rmat_na_full_size_against_oracle():
    """2^14 x 2^14 x 2^12 R-MAT pair, mode 2 x mode 0 (CSRNA) at 2^18 nnz each."""
    cfg = synth.config_rmat_na()
    C, info = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert info["alg"] == "CSRNA"
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])


def test_rmat_dcsr_reduced_size_against_oracle():
    """a_ijk b_ljk on 2^16 x 2^16 x 2^10 R-MAT tensors (1M nnz each): DCSR with
    B permuted (i,j,k) -> (j,k,i)."""
    cfg = synth.config_rmat_dcsr(bits=(16, 16, 10), nnz=1_000_000, seeds=(3, 4))
    C, info = _run(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert info["alg"] == "DCSR" and info["permute_b"] == 1
    assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])


def _matrix_pair(rows_spec, n_cols_r=4000, seed=50):
    """A: one row per spec entry (n_entries, products per entry) over a shared
    contracted range; B: rows with the requested lengths.  Returns host dicts."""
    rng = np.random.default_rng(seed)
    k = sum(ne for ne, _ in rows_spec) + 1
    a_co, b_rows = [], {}
    c = 0
    for r, (ne, pl) in enumerate(rows_spec):
        for _ in range(ne):
            a_co.append((r, c))
            b_rows[c] = np.sort(rng.choice(n_cols_r, size=min(pl, n_cols_r), replace=False))
            c += 1
    a_co = np.array(a_co, dtype=np.int64)
    A = {"dims": [len(rows_spec), k], "sig": [1, 0],
         "liv": np.ravel_multi_index(tuple(a_co.T), (len(rows_spec), k)).astype(np.int64),
         "val": rng.uniform(-1, 1, len(a_co))}
    b_co = np.array([(cc, j) for cc, js in b_rows.items() for j in js], dtype=np.int64)
    b_liv = np.sort(np.ravel_multi_index(tuple(b_co.T), (k, n_cols_r))).astype(np.int64)
    B = {"dims": [k, n_cols_r], "sig": [1, 0], "liv": b_liv, "val": rng.uniform(-1, 1, len(b_liv))}
    return A, B


@pytest.mark.parametrize("alg", ["CSR", "CSRNA", "DCSR"])
def test_row_kinds_in_one_product(alg):
    """Light rows merged by a lane (<= 8 runs), light rows with more runs
    (sorted by the whole warp), heavy rows reduced in shared memory and a
    heavy row reduced in global scratch, mixed in one contraction."""
    spec = ([(5, 3)] * 40 + [(12, 3)] * 10 + [(20, 15)] * 3 + [(1, 1)] * 30 +
            [(40, 40)] * 2 + [(3, 2)] * 20 + [(30, 120)] + [(6, 2)] * 50)
    A, B = _matrix_pair(spec, n_cols_r=50, seed=51)     # few columns: many duplicates
    C, info = _run(A, B, [1], [0], alg)
    assert_contract_matches(C, A, B, [1], [0])
    A, B = _matrix_pair(spec, n_cols_r=100000, seed=52)  # many columns: few duplicates
    C, info = _run(A, B, [1], [0], alg)
    assert_contract_matches(C, A, B, [1], [0])


def test_row_kinds_placed_through_scratch():
    """With more than 65,536 entries in L the row kernel writes each 32-row
    tile at the product offset of its first row and a compaction pass places
    the tiles: every row kind mixed, checked against the oracle and bit for
    bit against SOP (which has no row tiles)."""
    spec = ([(5, 3)] * 40 + [(12, 3)] * 10 + [(20, 15)] * 3 + [(1, 1)] * 30 +
            [(40, 40)] * 2 + [(3, 2)] * 20 + [(30, 120)] + [(6, 2)] * 50 + [(1, 400)] * 2) * 80
    A, B = _matrix_pair(spec, n_cols_r=3000, seed=53)
    assert len(A["liv"]) > 65536
    ref, _ = _run(A, B, [1], [0], "SOP")
    assert_contract_matches(ref, A, B, [1], [0])
    for alg in ("CSR", "CSRNA", "DCSR"):
        C, _ = _run(A, B, [1], [0], alg)
        assert torch.equal(C.liv, ref.liv), alg
        assert torch.equal(C.val.view(torch.int64), ref.val.view(torch.int64)), alg


def test_plan_reuse_gives_identical_results():
    """Running the same plan twice (as the benchmark does) reproduces C bit-for-bit."""
    cfg = synth.config_fd3d(n=24, seed=2)
    A, B = dev(cfg["A"]), dev(cfg["B"])
    plan = lco.ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, cfg["modes_a"], cfg["modes_b"])
    plan.ensure_workspace(0)
    plan.symbolic(A, B)
    f = plan.result()["f"]
    plan.ensure_workspace(f)
    outs = []
    for _ in range(2):
        c_liv = torch.empty(f, dtype=torch.int64, device="cuda")
        c_val = torch.empty(f, dtype=torch.float64, device="cuda")
        plan.run(A, B, c_liv, c_val)
        r = plan.result()
        assert r["status"] == 0
        outs.append((c_liv[:r["nnz_c"]].clone(), c_val[:r["nnz_c"]].clone()))
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1].view(torch.int64), outs[1][1].view(torch.int64))


def test_results_are_deterministic_on_every_branch():
    """Every branch sums each output's products in generation order, so two
    runs give the same bits, heavy rows included."""
    A = synth.rmat3((9, 6, 6), 30000, seed=41)
    B = synth.rmat3((9, 6, 6), 30000, seed=42)
    for alg in ("CSR", "CSRNA", "DCSR", "SOP", "CSC", "CSCNA", "DCSC"):
        C1, info = _run(A, B, [1, 2], [1, 2], alg)
        C2, _ = _run(A, B, [1, 2], [1, 2], alg)
        assert torch.equal(C1.liv, C2.liv), alg
        assert torch.equal(C1.val.view(torch.int64), C2.val.view(torch.int64)), alg
        assert_contract_matches(C1, A, B, [1, 2], [1, 2])


def test_single_entry_heavy_rows_are_copies():
    """Rows of A with one entry that meets an R row of thousands of entries
    (the row-sparse x column-sparse shape of the R-MAT mode-2 product) are
    scaled copies of that R row; mixed with multi-entry heavy rows and light
    rows, for every row-oriented branch."""
    rng = np.random.default_rng(31)
    k, n = 64, 5000
    b_rows = {c: np.sort(rng.choice(n, size=(3000 if c % 8 == 0 else 5), replace=False)) for c in range(k)}
    b_co = np.array([(c, j) for c in range(k) for j in b_rows[c]])
    B = {"dims": [k, n], "sig": [1, 0], "liv": (b_co[:, 0] * n + b_co[:, 1]).astype(np.int64),
         "val": rng.uniform(-1, 1, len(b_co))}
    a_co = [(r, (r * 8) % k) for r in range(40)]                   # one entry on a long R row
    a_co += [(40 + r, c) for r in range(4) for c in (0, 8, 16)]     # multi-entry heavy rows
    a_co += [(50 + r, c) for r in range(30) for c in (1, 2, 3)]     # light rows
    a_co += [(90, 5)]                                               # one entry on a short row
    a_co = np.array(sorted(a_co))
    A = {"dims": [100, k], "sig": [1, 0], "liv": (a_co[:, 0] * k + a_co[:, 1]).astype(np.int64),
         "val": rng.uniform(-1, 1, len(a_co))}
    for alg in ("CSR", "CSRNA", "DCSR"):
        C, info = _run(A, B, [1], [0], alg)
        assert_contract_matches(C, A, B, [1], [0])


def test_row_branches_are_bit_identical():
    """Every row branch (and the one-CTA path) multiplies each pair once,
    rounds the product, and adds the products of an output in generation
    order; so CSR, CSRNA, DCSR, SOP and the automatic plan agree bit for bit."""
    rng = np.random.default_rng(44)
    A = synth.stencil_operator((12, 12), synth.STENCIL_2D, rng.uniform(-1, 1, 5))
    R1 = synth.rmat3((7, 7, 5), 6000, seed=45)
    R2 = synth.rmat3((7, 7, 5), 6000, seed=46)
    for X, Y, ma, mb in ((A, A, [2, 3], [0, 1]), (R1, R2, [1, 2], [1, 2])):
        ref = None
        for alg in (None, "CSR", "CSRNA", "DCSR", "SOP"):
            C, _ = _run(X, Y, ma, mb, alg)
            if ref is None:
                ref = C
                assert_contract_matches(C, X, Y, ma, mb)
                continue
            assert torch.equal(C.liv, ref.liv), alg
            assert torch.equal(C.val.view(torch.int64), ref.val.view(torch.int64)), alg


def _heavy_case(seed, nrows, ent, rlen, ncol, window):
    """A with `nrows` rows of `ent` entries, each meeting an R row of `rlen`
    entries: every row has ent * rlen > 256 products (a heavy row).  With
    `window`, R's columns of the rows an A row meets lie within `window`
    consecutive columns (the dense-window accumulator fits); the R rows of
    one A row overlap in columns, so outputs sum several products."""
    rng = np.random.default_rng(seed)
    k = nrows * ent
    a_co = np.array([(r, r * ent + t) for r in range(nrows) for t in range(ent)])
    A = {"dims": [nrows, k], "sig": [1, 0], "liv": np.ravel_multi_index(tuple(a_co.T), (nrows, k)).astype(np.int64),
         "val": rng.uniform(-1, 1, len(a_co))}
    b_co = []
    for c in range(k):
        base = (c // ent) * 37 % max(ncol - window, 1)
        cols = base + rng.choice(window, rlen, replace=False) if window else rng.choice(ncol, rlen, replace=False)
        b_co += [(c, j) for j in cols]
    b_co = np.array(b_co)
    b_liv = np.sort(np.ravel_multi_index(tuple(b_co.T), (k, ncol))).astype(np.int64)
    B = {"dims": [k, ncol], "sig": [1, 0], "liv": b_liv, "val": rng.uniform(-1, 1, len(b_liv))}
    return A, B


@pytest.mark.parametrize("window", [400, 12000, 0])
def test_heavy_rows_accumulators(window):
    """Heavy rows (more than 256 products, up to 2048) of the accumulator
    plans (CSR, CSC, DCSR) go through the shared-memory accumulator: a dense
    column window when the row's columns span at most 16384 (window 400 and
    12000), else a column hash (window 0: columns spread over 2^20); the
    no-accumulator plans (CSRNA, CSCNA) expand, sort and sum.  Each matches
    the oracle, and every branch gives the same bits (products summed per
    column in entry order)."""
    A, B = _heavy_case(50 + window, nrows=24, ent=40, rlen=30, ncol=1 << 20, window=window)
    ref = None
    for alg in ("CSR", "CSRNA", "DCSR", "CSC", "CSCNA", "SOP"):
        C, info = _run(A, B, [1], [0], alg)
        assert info["f"] == 24 * 40 * 30
        if ref is None:
            ref = C
        assert_contract_matches(C, A, B, [1], [0])
        if list(C.sig) != list(ref.sig):
            # column variants give C column-major: compare in row-major order
            C = lco.radix_permute(C, ref.sig)
        assert torch.equal(C.liv, ref.liv), alg
        assert torch.equal(C.val.view(torch.int64), ref.val.view(torch.int64)), alg


def test_heavy_rows_at_the_accumulator_limits():
    """2048 products in a row (the accumulators' capacity) and one beyond it
    (the sort-based path), with many products per output column."""
    for ent, rlen in ((64, 32), (41, 50)):
        A, B = _heavy_case(60 + ent, nrows=8, ent=ent, rlen=rlen, ncol=4096, window=200)
        for alg in ("CSR", "CSRNA"):
            C, info = _run(A, B, [1], [0], alg)
            assert_contract_matches(C, A, B, [1], [0])


def test_radix_order_hint_gives_identical_products():
    """The operand permutation's sort order is a tuning choice: B of a_ijk
    b_ljk is rearranged to matrix order by a two-pass key whose high-digit
    buckets fit one CTA (high digit first on the device) or, with the hint,
    by LSD passes; the products are bit-identical and match the oracle."""
    A = _rand([64, 48, 40], None, 21, nnz=30_000)
    B = _rand([50, 48, 40], None, 22, nnz=30_000)
    ma, mb = [1, 2], [1, 2]
    out = []
    for order in (0, 1):
        C, info = lco.contract(dev(A), dev(B), ma, mb, return_info=True, radix_order=order)
        assert info["status"] == 0 and info["permute_b"]
        out.append(assert_contract_matches(C, A, B, ma, mb))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1].view(np.int64), out[1][1].view(np.int64))
