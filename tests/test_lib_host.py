"""CPU-only checks of the CUDA library: it builds for sm_103a, loads, exports
every entry point include/lco.h declares, and its host-side planning (RP
classification, Table-4 dispatch) agrees with the oracle.  No kernel runs."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import paper_1802_02619_gb300 as lco

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"\b(lco_[a-z0-9_]+)\s*\(", text):
                names.add(m.group(1))
    return names


def test_library_loads_and_exports_header():
    lib = lco.load()
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert lib.lco_build_arch() == 1030


def test_every_binding_is_declared():
    declared = _declared_functions()
    for name in lco.exported_symbols():
        assert name in declared


def test_status_strings():
    lib = lco.load()
    assert lib.lco_status_str(0) == b"ok"
    assert b"capacity" in lib.lco_status_str(8)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_rp_classification_matches_oracle(order):
    rng = np.random.default_rng(order)
    dims = [int(x) for x in rng.integers(2, 6, size=order)]
    for so in itertools.permutations(range(order)):
        for sn in itertools.permutations(range(order)):
            info = lco.radix_permute_info(dims, list(so), list(sn), nnz=10)
            assert info["is_rearr"] == list(oracle.rp_classify(list(so), list(sn)))
            mt, ml, nr = oracle.rp_keyspec(dims, list(so), list(sn))
            assert info["n_rearr"] == nr
            if nr:
                assert (info["m_top"], info["m_low"]) == (mt, ml)
                total = int(np.prod(dims))
                assert (1 << info["key_bits"]) >= total // ml
                assert info["passes"] * info["digit_bits"] >= info["key_bits"]


def test_rp_fig2_and_c2_permute_keys():
    info = lco.radix_permute_info([10, 3, 2], [0, 1, 2], [1, 0, 2])
    assert (info["m_top"], info["m_low"], info["is_rearr"]) == (30, 3, [1, 0, 0])
    # 6th-order 64^6 row-major -> (k,l,m,i,j,n): key is (k,l,m), 18 bits
    info = lco.radix_permute_info([64] * 6, [5, 4, 3, 2, 1, 0], [5, 1, 0, 4, 3, 2])
    assert info["m_low"] == 64 ** 3 and info["key_bits"] == 18 and info["passes"] == 2


def test_invalid_arguments_rejected():
    with pytest.raises(lco.LcoError):
        lco.radix_permute_info([3, 3], [0, 0], [1, 0])
    with pytest.raises(lco.LcoError):
        lco.radix_permute_info([1 << 32, 1 << 32], [0, 1], [1, 0])
    with pytest.raises(lco.LcoError):
        lco.ContractPlan([3, 4], [1, 0], 5, [3, 4], [1, 0], 5, [1], [0])   # 4 vs 3: dims mismatch
    with pytest.raises(lco.LcoError):
        lco.ContractPlan([1 << 40, 4], [1, 0], 5, [4, 1 << 40], [1, 0], 5, [1], [0])   # m*n overflow


def _plan(m_dims, k_dims, n_dims, nnz_a, nnz_b, sig_a=None, sig_b=None, alg=None):
    """A: free dims m_dims then contracted k_dims; B: contracted then free."""
    a_dims = list(m_dims) + list(k_dims)
    b_dims = list(k_dims) + list(n_dims)
    na, nb = len(a_dims), len(b_dims)
    sig_a = sig_a or list(range(na - 1, -1, -1))
    sig_b = sig_b or list(range(nb - 1, -1, -1))
    modes_a = list(range(len(m_dims), na))
    modes_b = list(range(len(k_dims)))
    return lco.ContractPlan(a_dims, sig_a, nnz_a, b_dims, sig_b, nnz_b, modes_a, modes_b, alg)


@pytest.mark.parametrize("ma,kk,nb", [(1, 1, 1), (1, 100, 1), (100, 1, 1), (1, 1, 100), (100, 100, 100),
                                      (100, 1, 100), (1, 100, 100), (100, 100, 1), (2, 4, 8), (8, 4, 2)])
def test_dispatch_matches_oracle(ma, kk, nb):
    """The library's Table-4 choice equals the oracle's on row-major operands."""
    nnz = 1000
    m, k, n = 1000 * ma, 1000 * kk, 1000 * nb
    for nnz_a, nnz_b in [(nnz, nnz), (10 * nnz, nnz), (nnz, 10 * nnz), (100 * nnz, 100 * nnz)]:
        p = _plan([m], [k], [n], nnz_a, nnz_b)
        # row-major operands need no permutation for the row variants and two for the column ones
        assert p.info["alg"] == oracle.dispatch(m, k, n, nnz_a, nnz_b, 0, 2)
        assert p.info["m"] == m and p.info["k"] == k and p.info["n"] == n


def test_dispatch_prefers_fewer_rearrangements():
    # operands already column-major: the column variant needs no permutation
    p = _plan([50], [50], [50], 1000, 1000, sig_a=[0, 1], sig_b=[0, 1])
    assert p.info["alg"] == "CSC" and p.info["transposed"] == 1
    assert p.info["permute_a"] == 0 and p.info["permute_b"] == 0
    # C comes out column-major: B's free mode most significant
    assert p.c_sig == [0, 1]


def test_configs_branches():
    import synth
    c = synth.config_fd2d(16)
    p = lco.ContractPlan(c["A"]["dims"], c["A"]["sig"], len(c["A"]["liv"]), c["B"]["dims"], c["B"]["sig"],
                         len(c["B"]["liv"]), c["modes_a"], c["modes_b"])
    assert p.info["alg"] == "CSR" and p.c_dims == [16] * 4 and p.c_sig == [3, 2, 1, 0]
    p = _plan([1 << 20], [1 << 20, 1 << 12], [1 << 20], 10_000_000, 10_000_000)
    assert p.info["alg"] == "DCSR"
    p = _plan([1 << 14, 1 << 14], [1 << 12], [1 << 14, 1 << 14], 1 << 18, 1 << 18)
    assert p.info["alg"] == "CSRNA"


def test_forced_algorithms_plan():
    for alg in lco.ALG_NAMES:
        p = _plan([30], [40], [50], 100, 100, alg=alg)
        assert p.info["alg"] == alg
        assert p.info["transposed"] == (alg in ("CSC", "DCSC", "CSCNA"))


def test_timing_hooks_without_launches():
    lco.timing_enable(True)
    assert lco.timing_read() == []
    lco.timing_enable(False)
    assert lco.launch_count() >= 0


def test_entrywise_plan_validation():
    import paper_1802_02619_gb300 as lco
    with pytest.raises(lco.LcoError):      # a mode both contracted and entrywise
        lco.ContractPlan([3, 4], [1, 0], 5, [3, 4], [1, 0], 5, [1], [1], entry_a=[1], entry_b=[1])
    with pytest.raises(lco.LcoError):      # entrywise dims differ
        lco.ContractPlan([3, 4], [1, 0], 5, [4, 3], [1, 0], 5, [], [], entry_a=[0], entry_b=[0])
    p = lco.ContractPlan([3, 4, 5], [2, 1, 0], 30, [3, 5, 6], [2, 1, 0], 40, [2], [1], entry_a=[0], entry_b=[0])
    assert p.c_dims == [3, 4, 6] and p.c_sig == [2, 1, 0]


@pytest.mark.parametrize("order", [2, 3, 4])
def test_wide_plan_matches_the_64_bit_classification(order):
    """The wide permutation classifies indices like the 64-bit path (Sec.
    4.1) and its key is the new LIV without the resting suffix."""
    rng = np.random.default_rng(40 + order)
    dims = [int(x) for x in rng.integers(2, 9, size=order)]
    for so in itertools.permutations(range(order)):
        for sn in itertools.permutations(range(order)):
            w = lco.radix_permute_wide_info(dims, list(so), list(sn), nnz=10)
            n = lco.radix_permute_info(dims, list(so), list(sn), nnz=10)
            assert w["n_rearr"] == n["n_rearr"]
            if n["n_rearr"]:
                total = int(np.prod(dims))
                assert (1 << w["key_bits"]) >= total // n["m_low"] > (1 << w["key_bits"]) // 2
                assert w["chunks"] == 1
            else:
                assert w["key_bits"] == 0 and w["chunks"] == 0


def test_wide_limits_and_chunks():
    # 2^127 - 1 is the wide limit; past it the shape is rejected
    with pytest.raises(lco.LcoError) as e:
        lco.radix_permute_wide_info([(1 << 63) - 1, (1 << 63) - 1, 4], [2, 1, 0], [0, 1, 2])
    assert e.value.status == 2
    with pytest.raises(lco.LcoError):
        lco.radix_permute_wide_info([1 << 40, 1 << 40], [0, 0], [1, 0])       # sig not a permutation
    # a 123-bit key is sorted in three 54-bit chunks, least significant first
    info = lco.radix_permute_wide_info([15, 1 << 61, 1 << 62], [2, 1, 0], [0, 2, 1])
    assert info == {"n_rearr": 2, "key_bits": 123, "chunks": 3, "passes": info["passes"]}
    assert info["passes"] >= 3
    # the 64-bit entry points still reject such shapes
    with pytest.raises(lco.LcoError):
        lco.radix_permute_info([15, 1 << 61, 1 << 62], [2, 1, 0], [0, 2, 1])


def test_wide_key_of_unit_range_still_takes_a_chunk():
    """Two unit dims swapped above everything else: one rearrangement index
    (Sec. 4.1) whose key range is 1.  The plan keeps one 1-bit chunk, so
    the gather reads positions the radix engine wrote."""
    for dims in ([4, 1, 1], [1 << 61, 1 << 62, 1, 1]):
        order = len(dims)
        sig = list(range(order))
        new_sig = sig[:-2] + [sig[-1], sig[-2]]
        info = lco.radix_permute_wide_info(dims, sig, new_sig)
        assert info["n_rearr"] == 1 and info["key_bits"] == 1 and info["chunks"] == 1
