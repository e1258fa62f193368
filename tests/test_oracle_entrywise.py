"""Pins for the oracle's contraction with entrywise (shared, unsummed) modes
(Sec. 5: such a product is one matrix product per value of the shared
indices): dense einsum brute force on tiny tensors, and slice by slice."""

import numpy as np
import pytest

import oracle


def _rand(dims, density, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    n = max(1, int(total * density))
    liv = np.sort(rng.choice(total, size=n, replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, n)}


def _dense(T):
    d = np.zeros(int(np.prod(T["dims"])))
    d[T["liv"]] = T["val"]
    return d.reshape(T["dims"])


def _pattern(T):
    d = np.zeros(int(np.prod(T["dims"])), dtype=np.int64)
    d[T["liv"]] = 1
    return d.reshape(T["dims"])


CASES = [
    # (A dims, B dims, modes_a, modes_b, entry_a, entry_b, einsum)
    ((3, 4, 5), (3, 5, 6), [2], [1], [0], [0], "hik,hkj->hij"),
    ((4, 5, 3), (6, 3, 5), [1], [2], [2], [1], "ikh,jhk->hij"),
    ((2, 3, 4, 5), (5, 2, 3, 6), [3], [0], [0, 1], [1, 2], "hgik,khgj->hgij"),
    ((3, 4), (3, 5), [], [], [0], [0], "hi,hj->hij"),              # entrywise outer product
    ((3, 4), (4, 3), [1], [0], [0], [1], "hk,kh->h"),              # entrywise inner product
]


@pytest.mark.parametrize("case", CASES)
def test_entrywise_against_dense_einsum(case):
    da, db, ma, mb, ea, eb, sub = case
    A, B = _rand(da, 0.5, 1), _rand(db, 0.5, 2)
    liv, val, _ = oracle.contract(A, B, ma, mb, ea, eb)
    ref = np.einsum(sub, _dense(A), _dense(B))
    pat = np.einsum(sub, _pattern(A), _pattern(B))          # products per output entry
    assert np.array_equal(liv, np.flatnonzero(pat.ravel()))
    assert np.allclose(val, ref.ravel()[liv], rtol=0, atol=1e-14)


def test_each_slice_is_a_plain_product():
    """For a fixed value h of the shared index the result is the ordinary
    contraction of A's and B's h-slices."""
    A, B = _rand((4, 6, 7), 0.3, 3), _rand((4, 7, 5), 0.3, 4)
    liv, val, _ = oracle.contract(A, B, [2], [1], [0], [0])
    for h in range(4):
        sa = {"dims": [6, 7], "sig": [1, 0], "liv": A["liv"][A["liv"] // 42 == h] - h * 42,
              "val": A["val"][A["liv"] // 42 == h]}
        sb = {"dims": [7, 5], "sig": [1, 0], "liv": B["liv"][B["liv"] // 35 == h] - h * 35,
              "val": B["val"][B["liv"] // 35 == h]}
        l, v, _ = oracle.contract(sa, sb, [1], [0])
        sel = liv // 30 == h
        assert np.array_equal(liv[sel] - h * 30, l)
        assert np.array_equal(val[sel], v)


def test_entrywise_validation():
    A, B = _rand((3, 4), 0.5, 5), _rand((3, 4), 0.5, 6)
    with pytest.raises(Exception):
        oracle.contract(A, B, [1], [1], [1], [1])   # a mode both contracted and entrywise
    with pytest.raises(Exception):
        oracle.contract(A, B, [], [], [0], [1])     # dims differ (3 vs 4)
