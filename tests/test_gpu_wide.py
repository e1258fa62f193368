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
