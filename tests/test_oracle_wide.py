"""Pins for the oracle's wide-LIV re-linearisation and permutation (unsigned
128-bit LIVs, Sec. 3.1's future work on LIVs past 2^63 - 1; Sec. 7).

Each pin checks the oracle against something other than its own formula:
the 64-bit oracle (pinned separately) where the dims allow both; bit-field
shuffles where every dim is a power of two (a LIV is then a concatenation of
bit fields); the round trip back to the old order; and coordinates kept
with their values."""
import numpy as np
import pytest

import oracle
import synth


def _ints(liv):
    return [int(a) | (int(b) << 64) for a, b in liv]


def _pairs(ints):
    return np.array([[x & ((1 << 64) - 1), x >> 64] for x in ints], dtype=np.uint64).reshape(-1, 2)


def test_equals_the_64_bit_oracle_where_both_apply():
    rng = np.random.default_rng(1)
    dims = [37, 50, 29, 41]
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=4000, replace=False)).astype(np.int64)
    val = rng.uniform(-1, 1, liv.shape[0])
    for new_sig in ([0, 1, 2, 3], [2, 0, 3, 1], [3, 1, 0, 2]):
        l64, v64 = oracle.permute(dims, [3, 2, 1, 0], new_sig, liv, val)
        wl, wv = oracle.permute_wide(dims, [3, 2, 1, 0], new_sig, _pairs(liv.tolist()), val)
        assert _ints(wl) == [int(x) for x in l64]
        assert np.array_equal(wv, v64)


def test_power_of_two_dims_are_bit_field_shuffles():
    # dims 2^41, 2^40, 2^30, 2^13: a LIV is four bit fields; re-linearising
    # moves whole fields, which shifts and masks compute without division
    widths = [41, 40, 30, 13]
    dims = [1 << w for w in widths]
    T = synth.wide_tensor(dims, [3, 2, 1, 0], 3000, seed=2)

    def fields(x, sig):
        out = {}
        for m in sig:                       # least significant field first
            out[m] = x & ((1 << widths[m]) - 1)
            x >>= widths[m]
        return out

    def join(f, sig):
        x, sh = 0, 0
        for m in sig:
            x |= f[m] << sh
            sh += widths[m]
        return x

    for new_sig in ([0, 1, 2, 3], [1, 3, 0, 2]):
        got = _ints(oracle.relinearise_wide(dims, [3, 2, 1, 0], new_sig, T["liv"]))
        want = [join(fields(x, [3, 2, 1, 0]), new_sig) for x in _ints(T["liv"])]
        assert got == want


def test_round_trip_restores_the_tensor():
    dims = [(1 << 40) + 7, (1 << 35) - 3, 999_983, 1 << 20]   # product ~2^115
    T = synth.wide_tensor(dims, [3, 2, 1, 0], 5000, seed=3)
    l1, v1 = oracle.permute_wide(dims, [3, 2, 1, 0], [1, 3, 0, 2], T["liv"], T["val"])
    l2, v2 = oracle.permute_wide(dims, [1, 3, 0, 2], [3, 2, 1, 0], l1, v1)
    assert np.array_equal(l2, T["liv"]) and np.array_equal(v2, T["val"])


def test_coordinates_keep_their_values_and_the_output_is_sorted():
    dims = [(1 << 50) + 1, (1 << 45) - 5, 12345]
    T = synth.wide_tensor(dims, [2, 1, 0], 3000, seed=4)
    new_sig = [0, 2, 1]
    lo, vo = oracle.permute_wide(dims, [2, 1, 0], new_sig, T["liv"], T["val"])

    def coords(x, sig):
        c = [0] * len(dims)
        for m in sig:
            x, c[m] = divmod(x, dims[m])
        return tuple(c)

    before = {coords(x, [2, 1, 0]): v for x, v in zip(_ints(T["liv"]), T["val"])}
    after_ints = _ints(lo)
    after = {coords(x, new_sig): v for x, v in zip(after_ints, vo)}
    assert before == after
    assert all(a < b for a, b in zip(after_ints, after_ints[1:]))


def test_limits():
    # dims multiplying past 2^127 - 1 are rejected
    with pytest.raises(oracle.OracleError):
        oracle.permute_wide([(1 << 63) - 1, (1 << 63) - 1, 4], [2, 1, 0], [0, 1, 2],
                            np.zeros((1, 2), np.uint64), np.zeros(1))
    # a LIV outside [0, prod dims) is rejected
    with pytest.raises(oracle.OracleError):
        oracle.relinearise_wide([1 << 40, 1 << 40], [1, 0], [0, 1], _pairs([1 << 80]))
    # empty tensors are fine
    lo, vo = oracle.permute_wide([1 << 40, 1 << 40], [1, 0], [0, 1], np.zeros((0, 2), np.uint64), np.zeros(0))
    assert lo.shape == (0, 2) and vo.shape == (0,)


def test_relinearisations_compose():
    """Re-linearising from order a to b and then from b to c equals going
    from a to c directly."""
    dims = [(1 << 37) + 5, (1 << 33) - 1, 123_457, 77]
    T = synth.wide_tensor(dims, [3, 2, 1, 0], 2000, seed=5)
    a, b, c = [3, 2, 1, 0], [1, 3, 0, 2], [2, 0, 3, 1]
    ab = oracle.relinearise_wide(dims, a, b, T["liv"])
    abc = oracle.relinearise_wide(dims, b, c, ab)
    ac = oracle.relinearise_wide(dims, a, c, T["liv"])
    assert np.array_equal(abc, ac)
    assert not np.array_equal(ab, T["liv"])


def test_wide_generator_is_seeded_sorted_and_in_range():
    dims = [(1 << 40) + 11, (1 << 41) - 9, 9_999_991]
    total = dims[0] * dims[1] * dims[2]
    T1 = synth.wide_tensor(dims, [2, 1, 0], 20_000, seed=8)
    T2 = synth.wide_tensor(dims, [2, 1, 0], 20_000, seed=8)
    assert np.array_equal(T1["liv"], T2["liv"]) and np.array_equal(T1["val"], T2["val"])
    x = _ints(T1["liv"])
    assert len(x) == 20_000 and all(a < b for a, b in zip(x, x[1:])) and 0 <= x[0] and x[-1] < total
    # uniform over the index space: the high words spread over their range
    hi = T1["liv"][:, 1].astype(np.float64)
    assert hi.max() > 0.9 * (total >> 64) and hi.min() < 0.1 * (total >> 64)
    # a product that fits 64 bits gives high words of zero
    S = synth.wide_tensor([1000, 1000], [1, 0], 500, seed=9)
    assert not S["liv"][:, 1].any() and S["liv"][:, 0].max() < 1_000_000


def _wide_of(T):
    liv = np.asarray(T["liv"], dtype=np.int64)
    return {"dims": list(T["dims"]), "sig": list(T["sig"]), "val": T["val"],
            "liv": np.stack([liv.view(np.uint64), np.zeros_like(liv).view(np.uint64)], 1)}


def _rand64(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=min(nnz, total), replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, liv.shape[0])}


@pytest.mark.parametrize("ma,mb", [([1], [0]), ([0], [1]), ([1, 2], [0, 1]), ([2, 0], [1, 2]), ([], [])])
def test_wide_contraction_equals_the_64_bit_oracle_where_both_apply(ma, mb):
    A = _rand64([6, 5, 4], 60, 31)
    B = _rand64([5, 4, 7], 70, 32)
    if ma == [0]:
        B = _rand64([5, 6, 3], 50, 33)
    if ma == [2, 0]:
        B = _rand64([3, 4, 6], 40, 34)
    l64, v64, a64 = oracle.contract(A, B, ma, mb)
    lw, vw, aw = oracle.contract_wide(_wide_of(A), _wide_of(B), ma, mb)
    assert _ints(lw) == [int(x) for x in l64]
    assert np.array_equal(vw, v64) and np.array_equal(aw, a64)


def test_wide_contraction_with_a_large_leading_mode():
    """A gains a leading free mode of size 2^62 + 3 (four large coordinates
    x), so C's LIVs pass 2^64.  Per value of x, C's slice is the 64-bit
    oracle's product of A's slice with B."""
    X = (1 << 62) + 3
    A = _rand64([7, 9], 40, 41)            # (i, k)
    B = _rand64([9, 6], 30, 42)            # (k, j)
    rng = np.random.default_rng(43)
    xs = [int(v) << 41 for v in np.sort(rng.choice(1 << 20, size=4, replace=False))]   # four large coordinates
    x_of = rng.integers(0, 4, size=len(A["liv"]))
    wide_a = sorted((int(xs[x]) * 63 + int(l), float(v)) for x, l, v in zip(x_of, A["liv"], A["val"]))
    Aw = {"dims": [X, 7, 9], "sig": [2, 1, 0], "liv": _pairs([w for w, _ in wide_a]),
          "val": np.array([v for _, v in wide_a])}
    lw, vw, _ = oracle.contract_wide(Aw, _wide_of(B), [2], [0])
    expect = []
    for x in range(4):
        sel = x_of == x
        if not sel.any():
            continue
        As = {"dims": [7, 9], "sig": [1, 0], "liv": A["liv"][sel], "val": A["val"][sel]}
        l64, v64, _ = oracle.contract(As, B, [1], [0])
        expect += [(int(xs[x]) * 42 + int(l), float(v)) for l, v in zip(l64, v64)]
    expect.sort()
    got = list(zip(_ints(lw), vw.tolist()))
    assert [g[0] for g in got] == [e[0] for e in expect]
    assert np.allclose([g[1] for g in got], [e[1] for e in expect], rtol=0, atol=1e-15)
    assert max(g[0] for g in got) >= 1 << 64


def test_wide_contraction_output_limit():
    # C's modes (2^62, 8) x (2^63 - 1) span ~2^128: past the wide limit
    A = {"dims": [1 << 62, 8, 1 << 40], "sig": [2, 1, 0], "liv": _pairs([5]), "val": np.ones(1)}
    B = {"dims": [1 << 40, (1 << 63) - 1], "sig": [1, 0], "liv": _pairs([7]), "val": np.ones(1)}
    with pytest.raises(oracle.OracleError):
        oracle.contract_wide(A, B, [2], [0])
