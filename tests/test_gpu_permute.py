"""GPU parity of the LIV shuffle and the radix permutation against the oracle
(bit-exact: LIVs are unique, so the output order is unique; values move
unchanged)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco
import synth
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _rand(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    nnz = min(nnz, total)
    if total <= 4 * nnz:
        liv = np.sort(rng.choice(total, size=nnz, replace=False))
    else:
        liv = np.unique(rng.integers(0, total, size=int(nnz * 1.2) + 8))[:nnz]
    liv = np.sort(liv).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.standard_normal(liv.shape[0])}


def _check_perm(T, new_sig):
    t = dev(T)
    out = lco.radix_permute(t, new_sig)
    rl, rv = oracle.permute(T["dims"], T["sig"], new_sig, T["liv"], T["val"])
    gl, gv = host(out)
    assert np.array_equal(gl, rl)
    assert np.array_equal(gv.view(np.int64), rv.view(np.int64))


def test_relinearise_matches_oracle():
    T = _rand([7, 31, 5, 63], 20000, 1)
    t = dev(T)
    for new in [[0, 1, 2, 3], [3, 2, 1, 0], [1, 3, 0, 2], [2, 0, 3, 1]]:
        got = lco.relinearise(t, new).cpu().numpy()
        assert np.array_equal(got, oracle.relinearise(T["dims"], T["sig"], new, T["liv"]))


def test_relinearise_table1():
    co = np.array([[1, 0, 0], [2, 0, 1], [0, 1, 1], [3, 2, 2], [1, 0, 3], [2, 2, 3]])
    liv = oracle.linearise([4, 4, 4], [2, 1, 0], co)     # row-major
    t = lco.LcoTensor([4, 4, 4], [2, 1, 0], torch.tensor(liv, device="cuda"),
                      torch.zeros(6, dtype=torch.float64, device="cuda"))
    got = lco.relinearise(t, [0, 1, 2]).cpu().numpy()
    assert got.tolist() == [1, 18, 20, 43, 49, 58]


def test_all_order4_permutations():
    """All 23 non-identity permutations of a 4th-order tensor (Sec. 4.2), on
    odd dims (2^k - 1 so that no division is a shift) and a ragged nnz."""
    T = _rand([15, 31, 7, 63], 40_001, 2)
    for sn in itertools.permutations(range(4)):
        _check_perm(T, list(sn))


def test_all_order6_permutations_small():
    T = _rand([3, 4, 5, 3, 4, 3], 1500, 3)
    for sn in itertools.permutations(range(6)):
        _check_perm(T, list(sn))


@pytest.mark.parametrize("nnz", [1, 2, 31, 4095, 4096, 4097, 8191, 70_001])
def test_ragged_sizes(nnz):
    T = _rand([64, 64, 64], nnz, 4 + nnz)
    _check_perm(T, [2, 0, 1])
    _check_perm(T, [1, 0, 2])


def test_empty():
    T = {"dims": [4, 5], "sig": [1, 0], "liv": np.empty(0, np.int64), "val": np.empty(0)}
    t = dev(T)
    out = lco.radix_permute(t, [0, 1])
    assert out.nnz == 0


def test_constant_digit_passes_skipped():
    """Keys whose high digits never vary: the passes are skipped on the device
    and the result still lands in the output buffer."""
    dims = [2, 4096, 4096]
    rng = np.random.default_rng(5)
    co = np.stack([np.zeros(5000, np.int64), rng.integers(0, 4096, 5000), rng.integers(0, 16, 5000)], 1)
    liv = np.unique(np.ravel_multi_index(tuple(co.T), dims)).astype(np.int64)
    T = {"dims": dims, "sig": [2, 1, 0], "liv": liv, "val": rng.standard_normal(liv.shape[0])}
    for sn in ([1, 2, 0], [0, 2, 1], [2, 0, 1]):
        _check_perm(T, sn)


def test_inverse_is_identity_on_device():
    T = _rand([64, 64, 64, 64], 300_000, 6)
    t = dev(T)
    p = lco.radix_permute(t, [1, 3, 0, 2])
    back = lco.radix_permute(p, T["sig"])
    assert torch.equal(back.liv, t.liv) and torch.equal(back.val.view(torch.int64), t.val.view(torch.int64))


def test_fd3d_result_permute_full_size():
    """The 64^3 Laplacian x derivative product permuted to (k,l,m,i,j,n),
    at full size (3.38M entries), compared with the oracle element by element."""
    cfg = synth.config_fd3d()
    liv, val, _ = oracle.contract(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    T = {"dims": [64] * 6, "sig": [5, 4, 3, 2, 1, 0], "liv": liv, "val": val}
    _check_perm(T, cfg["permute_sig"])


def test_rmat_b_permute_large():
    """R-MAT order-3 tensor, (i,j,k) -> (j,k,i): 32-bit shaved key, 1M entries."""
    T = synth.rmat3((20, 20, 12), 1_000_000, 4)
    _check_perm(T, [0, 2, 1])


@pytest.mark.parametrize("nnz", [4097, 70001])
def test_unaligned_buffers(nnz):
    """Input and output slices that are 8- but not 16-byte aligned (as in a
    batch's shared output buffer) take the direct-load path of the scatter;
    the result is unchanged."""
    T = _rand([64] * 4, nnz, seed=nnz)
    new_sig = [1, 3, 0, 2]
    rl, rv = oracle.permute(T["dims"], T["sig"], new_sig, T["liv"], T["val"])
    big_l = torch.zeros(nnz + 1, dtype=torch.int64, device="cuda")
    big_v = torch.zeros(nnz + 1, dtype=torch.float64, device="cuda")
    big_l[1:] = torch.from_numpy(T["liv"]).cuda()
    big_v[1:] = torch.from_numpy(T["val"]).cuda()
    out_l = torch.zeros(nnz + 1, dtype=torch.int64, device="cuda")
    out_v = torch.zeros(nnz + 1, dtype=torch.float64, device="cuda")
    p = lco.Permuter(T["dims"], T["sig"], new_sig, nnz)
    p(big_l[1:], big_v[1:], out_l[1:], out_v[1:])
    torch.cuda.synchronize()
    assert p.device_status() == 0
    assert np.array_equal(out_l[1:].cpu().numpy(), rl)
    assert np.array_equal(out_v[1:].cpu().numpy().view(np.int64), rv.view(np.int64))


def _run_with_path(T, new_sig):
    """Permutes through a Permuter and returns (liv, val, high_digit_first):
    the last from the radix engine's pass flags at the start of the
    workspace's region (after the 256-byte header): [17] is set when the
    device chose to sort by the high digit first."""
    t = dev(T)
    p = lco.Permuter(T["dims"], T["sig"], new_sig, T["liv"].shape[0], device="cuda")
    liv, val = p(t.liv, t.val)
    torch.cuda.synchronize()
    assert p.device_status() == 0
    flags = p.ws[256:256 + 32 * 4].view(torch.int32).cpu().numpy()
    return liv.cpu().numpy(), val.cpu().numpy(), bool(flags[17])


def test_high_digit_first_and_fallback():
    """Two-pass keys: with every high-digit bucket within one CTA's capacity
    the device sorts by the high digit first and each bucket locally by the
    low digit; one oversized bucket sends the same keys through the two LSD
    passes.  Both must equal the oracle bit for bit."""
    dims, sig, new = [256, 64, 64], [2, 1, 0], [0, 1, 2]
    # mode 0 keeps its place (resting): the key is (mode 2, mode 1), 12 bits
    info = lco.radix_permute_info(dims, sig, new)
    assert info["passes"] == 2 and info["key_bits"] == 12
    # uniform: high-digit (mode 2) buckets of ~3,000 entries
    T = _rand(dims, 200_000, 11)
    rl, rv = oracle.permute(dims, sig, new, T["liv"], T["val"])
    gl, gv, hdf = _run_with_path(T, new)
    assert hdf
    assert np.array_equal(gl, rl) and np.array_equal(gv.view(np.int64), rv.view(np.int64))
    # skewed: every (mode 0, mode 1) pair at mode 2 = 5, i.e. 16,384 entries
    # in one high-digit bucket, more than one CTA's 8,192
    rng = np.random.default_rng(12)
    co = np.stack([rng.integers(0, 256, 100_000), rng.integers(0, 64, 100_000), rng.integers(0, 64, 100_000)], 1)
    a, b = np.meshgrid(np.arange(256), np.arange(64), indexing="ij")
    hot = np.stack([a.ravel(), b.ravel(), np.full(a.size, 5)], 1)
    liv = np.unique(oracle.linearise(dims, sig, np.concatenate([co, hot])))
    S = {"dims": dims, "sig": sig, "liv": liv.astype(np.int64), "val": rng.standard_normal(liv.shape[0])}
    rl, rv = oracle.permute(dims, sig, new, S["liv"], S["val"])
    gl, gv, hdf = _run_with_path(S, new)
    assert not hdf
    assert np.array_equal(gl, rl) and np.array_equal(gv.view(np.int64), rv.view(np.int64))
