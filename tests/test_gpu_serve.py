"""Served contractions: every request's result equals the same product run
alone through lco_contract (bit for bit: same plan and kernels, summation in
generation order), a sample matches the oracle, memory comes back on
release, and a request that cannot fit fails with LCO_ERR_ADMISSION."""
import pytest
import torch

import paper_1802_02619_gb300 as lco
import synth
from gpu_util import assert_contract_matches, dev

pytestmark = pytest.mark.gpu


def _host(T):
    return {"dims": list(T.dims), "sig": list(T.sig), "liv": T.liv.cpu().numpy(), "val": T.val.cpu().numpy()}


def _problems():
    probs = synth.batch_problems(count=24, seed=21, fd2d=(5, 30), fd3d=(4, 9), rmat_nnz=(200, 20000))
    out = []
    for A, B, ma, mb, kind in probs:
        Ad = lco.LcoTensor(list(A["dims"]), list(A["sig"]), A["liv"].cuda(), A["val"].cuda()) \
            if isinstance(A["liv"], torch.Tensor) else dev(A)
        Bd = lco.LcoTensor(list(B["dims"]), list(B["sig"]), B["liv"].cuda(), B["val"].cuda()) \
            if isinstance(B["liv"], torch.Tensor) else dev(B)
        out.append((Ad, Bd, ma, mb, kind))
    return out


def test_served_results_equal_single_calls():
    probs = _problems()
    srv = lco.Server(pool_bytes=1 << 30, nslots=8)
    handles = [(srv.put(A), srv.put(B)) for A, B, *_ in probs]
    reqs = []
    for rep in range(3):                               # every problem three times, interleaved
        for (ha, hb), (A, B, ma, mb, kind) in zip(handles, probs):
            reqs.append((srv.submit(ha, hb, ma, mb), A, B, ma, mb, kind))
    for i, (rid, A, B, ma, mb, kind) in enumerate(reqs):
        r = srv.wait(rid)
        assert r["done"] and r["status"] == 0, (kind, r)
        ref, info = lco.contract(A, B, ma, mb, return_info=True)
        C = r["C"]
        assert r["alg"] == info["alg"]
        assert torch.equal(C.liv, ref.liv), f"{kind}: pattern differs from the single call"
        assert torch.equal(C.val.view(torch.int64), ref.val.view(torch.int64)), f"{kind}: values differ"
        if i < len(probs) and i % 3 == 0:
            assert_contract_matches(C, _host(A), _host(B), ma, mb)
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["in_flight"] == 0
    # only the operands remain in the pool
    assert st["pool_used"] == sum(((A.nnz if A.nnz else 1) * 16 + 255) // 256 * 256 +
                                  ((B.nnz if B.nnz else 1) * 16 + 255) // 256 * 256 for A, B, *_ in probs)
    srv.close()


def test_drop_while_pending_and_admission_failure():
    cfg = synth.config_fd2d(16)
    A = dev(cfg["A"])
    srv = lco.Server(pool_bytes=4 << 20, nslots=2)
    ha = srv.put(A)
    rid = srv.submit(ha, ha, cfg["modes_a"], cfg["modes_b"])
    srv.drop(ha)                                        # the pending request keeps it alive
    r = srv.wait(rid)
    assert r["status"] == 0
    assert_contract_matches(r["C"], cfg["A"], cfg["A"], cfg["modes_a"], cfg["modes_b"])
    srv.release(rid)
    assert srv.stats()["pool_used"] == 0
    # an operand pair whose workspace can never fit the 4 MiB pool
    big = synth.laplacian((24, 24, 24))
    hb = srv.put(dev(big))
    rid = srv.submit(hb, hb, [3, 4, 5], [0, 1, 2])
    r = srv.wait(rid, timeout_us=20_000_000)
    assert r["done"] and r["status"] == 7              # LCO_ERR_ADMISSION
    srv.close()
