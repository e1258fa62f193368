"""Contractions with entrywise (shared, unsummed) mode pairs on the GPU
against the oracle, on every branch of Table 4."""
import numpy as np
import pytest

import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches, dev

pytestmark = pytest.mark.gpu

ALGS = (None, "CSR", "CSRNA", "DCSR", "SOP", "CSC", "CSCNA", "DCSC")


def _rand(dims, density, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    n = max(1, int(total * density))
    liv = np.sort(rng.choice(total, size=n, replace=False)).astype(np.int64)
    return {"dims": list(dims), "sig": list(range(len(dims) - 1, -1, -1)), "liv": liv,
            "val": rng.uniform(-1, 1, n)}


CASES = [
    ((3, 4, 5), (3, 5, 6), [2], [1], [0], [0]),
    ((4, 5, 3), (6, 3, 5), [1], [2], [2], [1]),
    ((2, 3, 4, 5), (5, 2, 3, 6), [3], [0], [0, 1], [1, 2]),
    ((3, 4), (3, 5), [], [], [0], [0]),
    ((3, 4), (4, 3), [1], [0], [0], [1]),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("alg", ALGS)
def test_entrywise_small_every_branch(case, alg):
    da, db, ma, mb, ea, eb = case
    A, B = _rand(da, 0.5, 1), _rand(db, 0.5, 2)
    C, info = lco.contract(dev(A), dev(B), ma, mb, alg=alg, return_info=True, entry_a=ea, entry_b=eb)
    assert info["status"] == 0
    assert_contract_matches(C, A, B, ma, mb, ea=ea, eb=eb)


@pytest.mark.parametrize("alg", ALGS)
def test_entrywise_batch_of_rmat_products(alg):
    """64 shared-index values, each a hyper-sparse R-MAT-like product."""
    A = synth.rmat3((6, 9, 9), 40000, seed=61)     # (h, i, k)
    B = synth.rmat3((6, 9, 9), 40000, seed=62)     # (h, k, j)
    C, info = lco.contract(dev(A), dev(B), [2], [1], alg=alg, return_info=True, entry_a=[0], entry_b=[0])
    assert info["status"] == 0
    assert C.dims[0] == 64
    assert_contract_matches(C, A, B, [2], [1], ea=[0], eb=[0])


def test_entrywise_heavy_rows():
    """Rows with thousands of products inside one shared-index value."""
    rng = np.random.default_rng(70)
    H, I, K, J = 3, 4, 64, 3000
    a_co = np.array([(h, i, k) for h in range(H) for i in range(I) for k in range(0, K, 2)])
    b_co = np.array([(h, k, j) for h in range(H) for k in range(K) for j in rng.choice(J, 200, replace=False)])
    A = {"dims": [H, I, K], "sig": [2, 1, 0], "liv": np.ravel_multi_index(tuple(a_co.T), (H, I, K)).astype(np.int64),
         "val": rng.uniform(-1, 1, len(a_co))}
    bl = np.sort(np.ravel_multi_index(tuple(b_co.T), (H, K, J))).astype(np.int64)
    B = {"dims": [H, K, J], "sig": [2, 1, 0], "liv": bl, "val": rng.uniform(-1, 1, len(bl))}
    for alg in ("CSR", "CSRNA", "DCSR", None):
        C, info = lco.contract(dev(A), dev(B), [2], [1], alg=alg, return_info=True, entry_a=[0], entry_b=[0])
        assert_contract_matches(C, A, B, [2], [1], ea=[0], eb=[0])
