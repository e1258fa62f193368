"""GPU parity at the sizes the benchmarks run, element by element against the
oracle.

At full size the radix passes run thousands of tiles whose look-backs
overlap, two-pass keys have high-digit buckets too large for one CTA (so
the LSD passes run), and the DCSR entry cache packs row starts into 40
bits: none of this engages on small inputs.  These tests run them at full
size -- stand-alone permutations of 8M and 12M keys, the
hyper-sparse R-MAT product C3 (10M non-zeros per operand, DCSR, B permuted
with a 32-bit key in four passes) and the Sec. 6 product b_ii'jl d_i'k at
N = 2047 (b has 8.4M entries) -- and compare every LIV bit-exactly and every
value within |c - c_ref| <= 1e-13 sum |a||b|.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches, dev, host

pytestmark = pytest.mark.gpu


def _rand(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.unique(rng.integers(0, total, size=int(nnz * 1.05) + 8))
    liv = np.sort(rng.choice(liv, size=min(nnz, liv.shape[0]), replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1.0, 1.0, liv.shape[0])}


def _check_perm(T, new_sig, passes=None):
    info = lco.radix_permute_info(T["dims"], T["sig"], new_sig, nnz=T["liv"].shape[0])
    if passes is not None:
        assert info["passes"] == passes, info
    out = lco.radix_permute(dev(T), new_sig)
    rl, rv = oracle.permute(T["dims"], T["sig"], new_sig, T["liv"], T["val"])
    gl, gv = host(out)
    assert np.array_equal(gl, rl), "permuted LIVs differ from the oracle"
    assert np.array_equal(gv.view(np.int64), rv.view(np.int64)), "values were not moved bit-exactly"


@pytest.mark.parametrize("dims,nnz,new_sig,passes", [
    ([2047, 1023, 4095, 511], 8_000_003, [1, 3, 0, 2], 4),  # odd dims (no shifts), 32-bit key
    ([255, 511, 127, 1023], 8_000_003, [1, 3, 0, 2], 3),   # odd dims, 25-bit key
    ([255, 511, 127, 1023], 12_000_001, [3, 1, 2, 0], 2),  # odd dims, 15-bit key
    ([256, 512, 128, 1024], 12_000_000, [2, 0, 3, 1], 3),  # power-of-two dims (bit fields), 19-bit key
    ([4096, 4096, 4096], 8_000_000, [0, 2, 1], 3),         # order 3, 24-bit key
])
def test_full_size_permutations(dims, nnz, new_sig, passes):
    _check_perm(_rand(dims, nnz, seed=nnz % 1000 + len(dims)), new_sig, passes)


@pytest.fixture(scope="module")
def c3():
    return synth.config_rmat_dcsr()


def test_c3_b_permutation_full_size(c3):
    """C3's B (10M non-zeros, 2^20 x 2^20 x 2^12) into its matrix order
    (j,k,i): i is resting, the 32-bit key takes four passes."""
    _check_perm(c3["B"], [0, 2, 1])


def test_c3_contraction_full_size(c3):
    """C3 = A x_{1,2;1,2} B at full size: Table 4 picks DCSR, B is permuted,
    and the numeric phase reads the packed entry cache for every L entry."""
    A, B = dev(c3["A"]), dev(c3["B"])
    C, info = lco.contract(A, B, c3["modes_a"], c3["modes_b"], return_info=True)
    assert info["status"] == 0 and info["alg"] == "DCSR", info
    assert_contract_matches(C, c3["A"], c3["B"], c3["modes_a"], c3["modes_b"])


def test_eq17_full_size():
    """Sec. 6, Eq. 17 at N = 2^11 - 1: b (8,384,512 entries) times d, b
    rearranged on the device; 12,578,815 output entries."""
    cfg = synth.config_eq17(2047)
    C, info = lco.contract(dev(cfg["A"]), dev(cfg["B"]), cfg["modes_a"], cfg["modes_b"], return_info=True)
    assert info["status"] == 0, info
    liv, _ = assert_contract_matches(C, cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    assert liv.shape[0] == 12_578_815
    del C
    torch.cuda.empty_cache()
