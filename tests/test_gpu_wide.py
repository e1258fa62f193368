"""GPU parity of the wide-LIV (unsigned 128-bit) re-linearisation and radix
permutation against the oracle: LIVs and values bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco
import synth

pytestmark = pytest.mark.gpu


def _dev(liv_u64, val=None):
    liv = torch.from_numpy(np.ascontiguousarray(liv_u64).view(np.int64)).cuda()
    return liv if val is None else (liv, torch.as_tensor(val, dtype=torch.float64).cuda())


def _host(liv):
    return liv.cpu().numpy().view(np.uint64)


def _check_permute(dims, sig, new_sig, nnz, seed):
    T = synth.wide_tensor(dims, sig, nnz, seed)
    liv, val = _dev(T["liv"], T["val"])
    lo, vo = lco.radix_permute_wide(dims, sig, new_sig, liv, val)
    torch.cuda.synchronize()
    rl, rv = oracle.permute_wide(dims, sig, new_sig, T["liv"], T["val"])
    assert np.array_equal(_host(lo), rl)
    assert np.array_equal(vo.cpu().numpy().view(np.int64), rv.view(np.int64))
    return lco.radix_permute_wide_info(dims, sig, new_sig, T["liv"].shape[0])


WIDE = [1 << 40, (1 << 40) - 3, (1 << 30) + 3, 1000]     # ~2^120


@pytest.mark.parametrize("new_sig,chunks", [([0, 1, 2, 3], 2), ([3, 2, 0, 1], 1), ([2, 3, 1, 0], 2),
                                            ([1, 0, 3, 2], 1)])
def test_wide_permutation_matches_oracle(new_sig, chunks):
    info = _check_permute(WIDE, [3, 2, 1, 0], new_sig, 60_003, seed=11)
    assert info["chunks"] == chunks


def test_three_key_chunks():
    # ~2^126.9; mode 2 moves above mode 1 and mode 0 drops to the bottom,
    # so the key is modes 2 and 1: 123 bits
    dims = [15, 1 << 61, 1 << 62]
    info = _check_permute(dims, [2, 1, 0], [0, 2, 1], 40_000, seed=12)
    assert info["chunks"] == 3 and info["key_bits"] > 108


@pytest.mark.parametrize("nnz", [0, 1, 7, 2049, 100_003])
def test_ragged_sizes(nnz):
    _check_permute(WIDE, [3, 2, 1, 0], [2, 0, 3, 1], nnz, seed=13 + nnz)


@pytest.mark.parametrize("dims,nnz", [([4, 1, 1], 3), ([1 << 61, 1 << 62, 1, 1], 30_001)])
def test_unit_dims_in_the_key(dims, nnz):
    # the swapped top modes have dim 1: the key range is 1 and the output
    # is the input order with every LIV unchanged
    order = len(dims)
    sig = list(range(order))
    info = _check_permute(dims, sig, sig[:-2] + [sig[-1], sig[-2]], nnz, seed=18 + order)
    assert info["n_rearr"] == 1 and info["chunks"] == 1


def test_same_order_is_a_copy():
    info = _check_permute(WIDE, [3, 2, 1, 0], [3, 2, 1, 0], 5000, seed=14)
    assert info["n_rearr"] == 0


def test_agrees_with_the_64_bit_path_where_both_apply():
    rng = np.random.default_rng(15)
    dims = [300, 200, 100, 50]
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=50_000, replace=False)).astype(np.int64)
    val = rng.uniform(-1, 1, liv.shape[0])
    t = lco.LcoTensor(dims, [3, 2, 1, 0], torch.as_tensor(liv).cuda(), torch.as_tensor(val).cuda())
    p64 = lco.radix_permute(t, [1, 3, 0, 2])
    wide = np.stack([liv.view(np.uint64), np.zeros_like(liv).view(np.uint64)], 1)
    wl, wv = _dev(wide, val)
    lo, vo = lco.radix_permute_wide(dims, [3, 2, 1, 0], [1, 3, 0, 2], wl, wv)
    h = _host(lo)
    assert np.array_equal(h[:, 1], np.zeros(h.shape[0], np.uint64))
    assert np.array_equal(h[:, 0].view(np.int64), p64.liv.cpu().numpy())
    assert torch.equal(vo.view(torch.int64), p64.val.view(torch.int64))


def test_relinearise_wide_matches_oracle():
    T = synth.wide_tensor(WIDE, [3, 2, 1, 0], 30_001, seed=16)
    out = lco.relinearise_wide(WIDE, [3, 2, 1, 0], [1, 3, 0, 2], _dev(T["liv"]))
    torch.cuda.synchronize()
    assert np.array_equal(_host(out), oracle.relinearise_wide(WIDE, [3, 2, 1, 0], [1, 3, 0, 2], T["liv"]))


def test_round_trip_on_the_device():
    T = synth.wide_tensor(WIDE, [3, 2, 1, 0], 20_000, seed=17)
    liv, val = _dev(T["liv"], T["val"])
    l1, v1 = lco.radix_permute_wide(WIDE, [3, 2, 1, 0], [0, 2, 1, 3], liv, val)
    l2, v2 = lco.radix_permute_wide(WIDE, [0, 2, 1, 3], [3, 2, 1, 0], l1, v1)
    assert torch.equal(l2, liv) and torch.equal(v2.view(torch.int64), val.view(torch.int64))


# ---------------------------------------------------------------------------
# Contraction of wide tensors (rank compression + the 64-bit product)
# ---------------------------------------------------------------------------

def _ints(l):
    return [int(a) | (int(b) << 64) for a, b in np.asarray(l, dtype=np.uint64)]


def _pairs(ints):
    return np.array([[x & ((1 << 64) - 1), x >> 64] for x in ints], dtype=np.uint64).reshape(-1, 2)


def _check_contract_wide(A, B, ma, mb):
    al, av = _dev(A["liv"], A["val"])
    bl, bv = _dev(B["liv"], B["val"])
    cl, cv, plan = lco.contract_wide(A["dims"], A["sig"], al, av, B["dims"], B["sig"], bl, bv, ma, mb)
    torch.cuda.synchronize()
    rl, rv, ra = oracle.contract_wide(A, B, ma, mb)
    got = _host(cl) if cl.shape[0] else np.empty((0, 2), np.uint64)
    assert got.shape == rl.shape, f"{got.shape[0]} entries, oracle {rl.shape[0]}"
    assert np.array_equal(got, rl), "index pattern differs from the oracle"
    err = np.abs(cv.cpu().numpy() - rv)
    assert np.all(err <= 1e-13 * ra), f"worst {err.max() if err.size else 0}"
    return plan, rl.shape[0]


def test_wide_contraction_agrees_with_64_bit_where_both_apply():
    rng = np.random.default_rng(70)
    dims_a, dims_b = [30, 40, 20], [20, 50, 40]
    A = {"dims": dims_a, "sig": [2, 1, 0], "liv": np.sort(rng.choice(30 * 40 * 20, 6000, replace=False))}
    B = {"dims": dims_b, "sig": [0, 2, 1], "liv": np.sort(rng.choice(20 * 50 * 40, 9000, replace=False))}
    A["val"], B["val"] = rng.uniform(-1, 1, 6000), rng.uniform(-1, 1, 9000)
    Aw = dict(A, liv=_pairs([int(x) for x in A["liv"]]))
    Bw = dict(B, liv=_pairs([int(x) for x in B["liv"]]))
    for ma, mb in (([2], [0]), ([1, 2], [2, 0]), ([1], [2])):
        plan, n = _check_contract_wide(Aw, Bw, ma, mb)
        C64 = lco.contract(lco.LcoTensor.from_host(A, "cuda"), lco.LcoTensor.from_host(B, "cuda"), ma, mb)
        assert n == C64.nnz


def test_wide_contraction_large_free_modes():
    """Row keys near 2^90 and column keys near 2^45 (C's LIVs near 2^126),
    a small contracted mode: every A entry meets B rows."""
    A = synth.wide_tensor([1 << 40, (1 << 40) - 3, 1000], [2, 1, 0], 20_000, seed=71)
    B = synth.wide_tensor([1000, (1 << 45) + 7, 3], [2, 1, 0], 30_000, seed=72)
    plan, n = _check_contract_wide(A, B, [2], [0])
    assert n > 100_000


def test_wide_contraction_with_a_wide_contracted_key():
    """The contracted pair spans ~2^100: B's rows are built from A's keys so
    that half of A's entries meet one, the others meet none (dropped from
    the rank matrix)."""
    rng = np.random.default_rng(73)
    K1, K2, I, J = (1 << 50) + 1, (1 << 50) - 5, 11, 9
    A = synth.wide_tensor([I, K1, K2], [2, 1, 0], 8000, seed=74)      # (i, k1, k2), row-major
    keys = sorted({x % (K1 * K2) for x in _ints(A["liv"])})
    keep = [k for k in keys if rng.random() < 0.5]
    b_ints = sorted({k * J + int(j) for k in keep for j in rng.choice(J, 3, replace=False)})
    B = {"dims": [K1, K2, J], "sig": [2, 1, 0], "liv": _pairs(b_ints), "val": rng.uniform(-1, 1, len(b_ints))}
    _check_contract_wide(A, B, [1, 2], [0, 1])


def test_wide_contraction_mixed_orders_and_empty():
    A = synth.wide_tensor([1 << 33, 17, (1 << 31) + 1], [0, 2, 1], 5000, seed=75)
    B = synth.wide_tensor([17, 1 << 35], [1, 0], 4000, seed=76)
    _check_contract_wide(A, B, [1], [0])
    E = {"dims": [17, 1 << 35], "sig": [1, 0], "liv": np.empty((0, 2), np.uint64), "val": np.empty(0)}
    el, ev = _dev(E["liv"], E["val"])
    al, av = _dev(A["liv"], A["val"])
    cl, cv, _ = lco.contract_wide(A["dims"], A["sig"], al, av, E["dims"], E["sig"], el, ev, [1], [0])
    assert cl.shape[0] == 0
