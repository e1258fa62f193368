"""Helpers shared by the GPU parity tests: move seeded inputs to the device,
compare device results with the oracle."""
import numpy as np
import torch

import oracle
import paper_1802_02619_gb300 as lco

TOL = 1e-13   # |c - c_ref| <= TOL * sum |a||b| per entry


def dev(T):
    return lco.LcoTensor.from_host(T, "cuda")


def host(t):
    return t.liv.cpu().numpy(), t.val.cpu().numpy()


def oracle_contract_in(A, B, ma, mb, c_dims, c_sig, ea=(), eb=()):
    """Oracle result expressed in the order c_sig (the oracle produces row-major)."""
    liv, val, ab = oracle.contract(A, B, ma, mb, ea, eb)
    rm = list(range(len(c_dims) - 1, -1, -1))
    if list(c_sig) != rm and liv.shape[0] > 0:
        l2, v2 = oracle.permute(c_dims, rm, c_sig, liv, val)
        l3, a2 = oracle.permute(c_dims, rm, c_sig, liv, ab)
        assert np.array_equal(l2, l3)
        return l2, v2, a2
    return liv, val, ab


def assert_contract_matches(C, A, B, ma, mb, tol=TOL, ea=(), eb=()):
    liv, val = host(C)
    rl, rv, ra = oracle_contract_in(A, B, ma, mb, C.dims, C.sig, ea, eb)
    assert liv.shape == rl.shape, f"nnz {liv.shape[0]} vs oracle {rl.shape[0]}"
    assert np.array_equal(liv, rl), "index pattern differs from the oracle"
    err = np.abs(val - rv)
    bad = err > tol * ra
    assert not np.any(bad), f"{int(bad.sum())} values out of tolerance, worst {err[bad].max()}"
    return liv, val


def cuda_sync():
    torch.cuda.synchronize()
