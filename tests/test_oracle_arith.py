"""Pins for the oracle's sort and add (Sec. 3.2; the sum of Eq. 4) and for
the combinatorial Laplacian chain of Sec. 6 computed with the oracle."""
import numpy as np
import pytest

import oracle
import synth


def _rand(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, liv.shape[0])}


def test_sort_of_a_shuffle_restores_the_tensor():
    T = _rand([30, 40, 50], 5000, 1)
    perm = np.random.default_rng(2).permutation(5000)
    l, v = oracle.sort(T["liv"][perm], T["val"][perm])
    assert np.array_equal(l, T["liv"]) and np.array_equal(v, T["val"])


def test_sort_is_stable_and_matches_a_library_stable_sort():
    rng = np.random.default_rng(3)
    liv = rng.integers(0, 50, 2000).astype(np.int64)        # many equal keys
    val = np.arange(2000, dtype=np.float64)                   # values record the input position
    l, v = oracle.sort(liv, val)
    o = np.argsort(liv, kind="stable")
    assert np.array_equal(l, liv[o]) and np.array_equal(v, val[o])


def _dense(T):
    d = np.zeros(int(np.prod(T["dims"])))
    d[T["liv"]] = T["val"]
    return d


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (2.0, -0.5), (0.0, 3.0)])
def test_add_against_dense_sum(alpha, beta):
    A, B = _rand([8, 9, 10], 300, 4), _rand([8, 9, 10], 300, 5)
    l, v = oracle.add(alpha, A, beta, B)
    assert np.array_equal(l, np.union1d(A["liv"], B["liv"]))      # the union, structural entries kept
    ref = alpha * _dense(A) + beta * _dense(B)
    assert np.allclose(v, ref[l], rtol=0, atol=1e-15)


def test_add_keeps_cancelled_entries_and_commutes():
    A = _rand([20, 20], 150, 6)
    l, v = oracle.add(1.0, A, -1.0, A)
    assert np.array_equal(l, A["liv"]) and np.all(v == 0.0)         # reading: structural zeros kept
    B = _rand([20, 20], 150, 7)
    l1, v1 = oracle.add(1.0, A, 1.0, B)
    l2, v2 = oracle.add(1.0, B, 1.0, A)
    assert np.array_equal(l1, l2) and np.array_equal(v1, v2)


def test_add_disjoint_supports_is_concatenation_in_order():
    A = {"dims": [100], "sig": [0], "liv": np.arange(0, 100, 2, dtype=np.int64), "val": np.ones(50)}
    B = {"dims": [100], "sig": [0], "liv": np.arange(1, 100, 2, dtype=np.int64), "val": 2 * np.ones(50)}
    l, v = oracle.add(1.0, A, 1.0, B)
    assert np.array_equal(l, np.arange(100)) and np.array_equal(v, np.tile([1.0, 2.0], 50))


def laplacian_chain(N):
    """Eq. 4 evaluated left to right with the oracle: two outer products with
    delta, two Eq. 17 products, the re-sort of the second term and the sum."""
    d, dl = synth.fd_matrix(N), synth.kronecker_delta(N)
    rm = [3, 2, 1, 0]
    # b_y[i,i',j,l] = d[i,i'] delta[j,l];  c_y[i,j,l,k] = b_y[i,i',j,l] d[i',k]
    by = dict(zip(("liv", "val"), oracle.contract(d, dl, [], [])[:2]), dims=[N] * 4, sig=rm)
    cy = dict(zip(("liv", "val"), oracle.contract(by, d, [1], [0])[:2]), dims=[N] * 4, sig=rm)
    # b_x[j,j',i,k] = d[j,j'] delta[i,k];  c_x[j,i,k,l] = b_x[j,j',i,k] d[j',l]
    cx = dict(zip(("liv", "val"), oracle.contract(by, d, [1], [0])[:2]), dims=[N] * 4, sig=rm)
    # c_x read with c_y's mode names (i,j,l,k): c_x's most significant mode j is
    # c_y's mode 1, then i (0), k (3), l (2): sig (least significant first) [2,3,0,1]
    cx_named = synth.relabel(cx, [2, 3, 0, 1])
    pl, pv = oracle.permute(cx_named["dims"], cx_named["sig"], rm, cx_named["liv"], cx_named["val"])
    al, av = oracle.add(1.0, cy, 1.0, {"liv": pl, "val": pv})
    return {"dims": [N] * 4, "sig": rm, "liv": al, "val": av}


@pytest.mark.parametrize("N", [7, 15])
def test_laplacian_chain_on_quadratics_is_exactly_four(N):
    """d (Eq. 1) is exact on quadratics: d d (i^2) = 2 on every row, so the
    combinatorial Laplacian of Eq. 4, a_ijkl, maps x_kl = k^2 + l^2 to 4 at
    every (i, j) -- exactly, as every value is a small dyadic rational."""
    a = laplacian_chain(N)
    x = synth.quadratic_field(N)
    yl, yv, _ = oracle.contract(a, x, [3, 2], [0, 1])      # a is named (i,j,l,k): contract l,k with x's k,l
    assert np.array_equal(yl, np.arange(N * N)) and np.all(yv == 4.0)
