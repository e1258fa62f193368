"""Pins for the oracle's linearisation, LIV shuffle, RP classification and
permutation (Secs. 3.1 and 4.1).  CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table1():
    dims, sig, rows = None, None, []
    with open(os.path.join(GOLDEN, "table1_co_vs_lco.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("# dims:"):
                dims = [int(x) for x in line.split(":")[1].split()]
            elif line.startswith("# sig:"):
                sig = [int(x) for x in line.split(":")[1].split()]
            elif line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    rows = np.array(rows, dtype=np.int64)
    return dims, sig, rows[:, :3], rows[:, 3]


def test_table1_linearise():
    """Table 1: CO {1,0,0}.. in a 4x4x4 tensor, order {0,1,2} -> LCO 1,18,20,43,49,58."""
    dims, sig, co, liv = _read_table1()
    assert np.array_equal(oracle.linearise(dims, sig, co), liv)
    assert np.array_equal(oracle.delinearise(dims, sig, liv), co)


def test_liv_formula_brute_force():
    """LIV = i + n_i (j + n_j k) for order {0,1,2}, checked over every coordinate,
    and every other order as the same sum with the strides permuted."""
    dims = [3, 4, 5]
    co = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int64)
    expect = co[:, 0] + dims[0] * (co[:, 1] + dims[1] * co[:, 2])
    assert np.array_equal(oracle.linearise(dims, [0, 1, 2], co), expect)
    for sig in itertools.permutations(range(3)):
        stride, s = {}, 1
        for mode in sig:               # sig[0] least significant
            stride[mode] = s
            s *= dims[mode]
        exp = sum(co[:, m] * stride[m] for m in range(3))
        got = oracle.linearise(dims, list(sig), co)
        assert np.array_equal(got, exp)
        # bijection onto 0..prod-1
        assert np.array_equal(np.sort(got), np.arange(np.prod(dims)))


def test_relinearise_roundtrip_and_table1():
    dims, sig, co, liv = _read_table1()
    for new in itertools.permutations(range(3)):
        r = oracle.relinearise(dims, sig, list(new), liv)
        assert np.array_equal(r, oracle.linearise(dims, list(new), co))
        back = oracle.relinearise(dims, list(new), sig, r)
        assert np.array_equal(back, liv)


def test_overflow_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.relinearise([1 << 32, 1 << 32], [0, 1], [1, 0], np.array([0], np.int64))
    with pytest.raises(oracle.OracleError):
        oracle.relinearise([1 << 62, 2], [0, 1], [1, 0], np.array([0], np.int64))
    # 7 * 1317624576693539401 = 2^63 - 1, the largest product that fits
    dims = [7, 1317624576693539401]
    top = (1 << 63) - 2
    r = oracle.relinearise(dims, [0, 1], [1, 0], np.array([top], np.int64))
    assert r[0] == (top % 7) * dims[1] + top // 7


def _fig2():
    d = {}
    with open(os.path.join(GOLDEN, "fig2_rp_example.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                d[k] = [int(x) for x in v]
    return d


def test_fig2_classification_and_divisors():
    """Fig. 2: {0,1,2} -> {1,0,2} on 10x3x2: i rearranges, j and k rest; /30 and /3."""
    g = _fig2()
    assert list(oracle.rp_classify(g["sig_old"], g["sig_new"])) == g["rearrangement"]
    mt, ml, nr = oracle.rp_keyspec(g["dims"], g["sig_old"], g["sig_new"])
    assert (mt, ml, nr) == (g["m_top"][0], g["m_low"][0], 1)


def test_min_permutation_of_table2_needs_one_index():
    """Table 2 / Sec. 4.2: {0,1,2,3} -> {1,0,2,3} rearranges a single index."""
    r = oracle.rp_classify([0, 1, 2, 3], [1, 0, 2, 3])
    assert list(r) == [1, 0, 0, 0]
    mt, ml, nr = oracle.rp_keyspec([5, 6, 7, 8], [0, 1, 2, 3], [1, 0, 2, 3])
    assert (mt, ml, nr) == (30, 6, 1)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_final_index_always_resting(order):
    """Sec. 4.1: the final (least significant) index of the new order is always resting."""
    base = list(range(order))
    for new in itertools.permutations(base):
        r = oracle.rp_classify(base, list(new))
        assert r[new[0]] == 0
        assert (r.sum() == 0) == (list(new) == base)


def _rand_tensor(dims, nnz, rng):
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False)).astype(np.int64)
    val = rng.standard_normal(liv.shape[0])
    return liv, val


def _check_permute_case(dims, so, sn, liv, val):
    lo, vo = oracle.permute(dims, so, sn, liv, val)
    # definition-level properties
    assert np.all(np.diff(lo) > 0)
    co_in = oracle.delinearise(dims, so, liv)
    co_out = oracle.delinearise(dims, sn, lo)
    a = {tuple(c): v for c, v in zip(co_in.tolist(), val.tolist())}
    b = {tuple(c): v for c, v in zip(co_out.tolist(), vo.tolist())}
    assert a == b
    # inverse permutation restores the input bit-exactly
    lb, vb = oracle.permute(dims, sn, so, lo, vo)
    assert np.array_equal(lb, liv) and np.array_equal(vb.view(np.int64), val.view(np.int64))
    # the RP algorithm (regions + stable sort on the shaved key) agrees
    lr, vr = oracle.rp_permute(dims, so, sn, liv, val)
    assert np.array_equal(lr, lo) and np.array_equal(vr.view(np.int64), vo.view(np.int64))
    return lo, vo


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_all_order_pairs_small(order):
    rng = np.random.default_rng(10 + order)
    dims = [int(x) for x in rng.integers(2, 5, size=order)]
    liv, val = _rand_tensor(dims, max(1, int(np.prod(dims)) // 3), rng)
    for so in itertools.permutations(range(order)):
        so = list(so)
        src, _ = oracle.permute(dims, list(range(order)), so, liv, val)
        sval = rng.standard_normal(src.shape[0])
        for sn in itertools.permutations(range(order)):
            _check_permute_case(dims, so, list(sn), src, sval)


def test_all_order6_permutations():
    """All 719 non-identity order-6 permutations (and 23 of order 4, Sec. 4.2)."""
    rng = np.random.default_rng(6)
    dims = [2, 3, 2, 3, 2, 2]
    liv, val = _rand_tensor(dims, 150, rng)
    base = list(range(6))
    for sn in itertools.permutations(base):
        _check_permute_case(dims, base, list(sn), liv, val)


def test_composition():
    """perm q after perm p equals the single permutation to q."""
    rng = np.random.default_rng(3)
    dims = [4, 3, 5, 2]
    liv, val = _rand_tensor(dims, 60, rng)
    p, q = [2, 0, 3, 1], [1, 3, 0, 2]
    l1, v1 = oracle.permute(dims, [0, 1, 2, 3], p, liv, val)
    l2, v2 = oracle.permute(dims, p, q, l1, v1)
    l3, v3 = oracle.permute(dims, [0, 1, 2, 3], q, liv, val)
    assert np.array_equal(l2, l3) and np.array_equal(v2, v3)


def test_shaving_is_tight():
    """Dropping the lowest rearrangement index from the shaved key breaks the
    sort for some input: the classification does not mark it resting."""
    rng = np.random.default_rng(4)
    dims = [4, 4, 4]
    so, sn = [0, 1, 2], [1, 0, 2]      # index 0 must be sorted on
    liv, val = _rand_tensor(dims, 40, rng)
    full, _ = oracle.permute(dims, so, sn, liv, val)
    newliv = oracle.relinearise(dims, so, sn, liv)
    mt, ml, _ = oracle.rp_keyspec(dims, so, sn)
    coarse = (newliv % mt) // (ml * dims[0])          # key without index 0
    order = np.lexsort((np.arange(liv.shape[0]), coarse, newliv // mt))
    assert not np.array_equal(newliv[order], full)
    shaved = (newliv % mt) // ml
    order = np.lexsort((np.arange(liv.shape[0]), shaved, newliv // mt))
    assert np.array_equal(newliv[order], full)


def test_empty_and_single():
    dims = [3, 3]
    lo, vo = oracle.permute(dims, [0, 1], [1, 0], np.empty(0, np.int64), np.empty(0))
    assert lo.shape == (0,)
    lo, vo = oracle.permute(dims, [0, 1], [1, 0], np.array([5], np.int64), np.array([2.5]))
    assert lo.tolist() == [7] and vo.tolist() == [2.5]
