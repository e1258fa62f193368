"""Programmatic dependent launches change when kernels start, not what they
compute.  A kernel that follows another kernel in the contraction or radix
chain is scheduled while its predecessor drains and waits on it first thing;
with LCO_PDL=0 in the environment the same kernels are launched the ordinary
way.  The products below (a CSR plan with its output permuted high digit
first, a DCSR plan whose R operand is permuted by LSD passes, a no-accumulator
plan) are computed in a child process with LCO_PDL=0 and here with the
default, and must agree bit for bit; the first is also checked against the
oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    fd = synth.config_fd3d(24)
    dc = synth.config_rmat_dcsr(bits=(13, 13, 8), nnz=300_000)
    na = synth.config_rmat_na(bits=(10, 10, 8), nnz=40_000)
    return [(fd, fd["permute_sig"]), (dc, None), (na, None)]


def _compute():
    """Every case's result as host arrays (LIVs, values), in order."""
    import paper_1802_02619_gb300 as lco
    out = []
    for cfg, psig in _cases():
        A = lco.LcoTensor.from_host(cfg["A"], "cuda")
        B = lco.LcoTensor.from_host(cfg["B"], "cuda")
        C = lco.contract(A, B, cfg["modes_a"], cfg["modes_b"])
        if psig is not None:
            C = lco.radix_permute(C, psig)
        out += [C.liv.cpu().numpy(), C.val.cpu().numpy()]
    return out


def test_dependent_launches_match_ordinary_launches(tmp_path):
    if os.environ.get("LCO_PDL", "1").startswith("0"):
        pytest.skip("dependent launches are turned off in this process")
    here = _compute()
    out = tmp_path / "ordinary.npz"
    code = ("import sys, numpy as np; sys.path[:0] = [sys.argv[1], sys.argv[1] + '/tests']; "
            "import test_gpu_pdl as t; np.savez(sys.argv[2], *t._compute())")
    env = dict(os.environ, LCO_PDL="0")
    r = subprocess.run([sys.executable, "-c", code, ROOT, str(out)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    there = np.load(out)
    ordinary = [there["arr_%d" % i] for i in range(len(here))]
    for i, (a, b) in enumerate(zip(here, ordinary)):
        assert a.shape == b.shape, (i, a.shape, b.shape)
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), "case %d, array %d differs" % (i // 2, i % 2)
    # the first case against the oracle: contraction, then the permutation
    cfg, psig = _cases()[0]
    rl, rv, _ = oracle.contract(cfg["A"], cfg["B"], cfg["modes_a"], cfg["modes_b"])
    c_dims = [d for t, d in enumerate(cfg["A"]["dims"]) if t not in cfg["modes_a"]] + \
             [d for t, d in enumerate(cfg["B"]["dims"]) if t not in cfg["modes_b"]]
    rm = list(range(len(c_dims) - 1, -1, -1))
    pl, pv = oracle.permute(c_dims, rm, psig, rl, rv)
    assert np.array_equal(here[0], pl)
    # stencil products of the 3D Laplacian with the derivative: at most 3
    # products per output, |a||b| <= 6; 1e-13 * sum |a||b| bounds the error
    assert np.max(np.abs(here[1] - pv)) <= 1e-13 * 3 * 6
