"""The no-allocation radix permutation (lco_radix_permute_static).

It exists for callers that cannot allocate device memory (a plug-in whose
host application owns every allocation), so it takes no workspace and uses a
fixed scratch array inside the library.  This file is collected last so that,
run after the other tests, it also sees the array in whatever state earlier
library use left the device in; it must pass alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1802_02619_gb300 as lco

pytestmark = pytest.mark.gpu

MAX_NNZ = 65536


def _tensor(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    total = int(np.prod(dims))
    liv = np.sort(rng.choice(total, size=nnz, replace=False)).astype(np.int64)
    return lco.LcoTensor(list(dims), list(range(len(dims) - 1, -1, -1)),
                         torch.tensor(liv, device="cuda"),
                         torch.tensor(rng.standard_normal(nnz), device="cuda"))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _static_permute(t, new_sig):
    lib = lco.load()
    sh = t.shape()
    sig = (ctypes.c_int32 * lco.MAX_ORDER)(*new_sig)
    liv_out = torch.empty_like(t.liv)
    val_out = torch.empty_like(t.val)
    rc = lib.lco_radix_permute_static(ctypes.byref(sh), sig, ctypes.c_void_p(t.liv.data_ptr()),
                                      ctypes.c_void_p(t.val.data_ptr()), ctypes.c_void_p(liv_out.data_ptr()),
                                      ctypes.c_void_p(val_out.data_ptr()), _stream())
    assert rc == 0, f"lco_radix_permute_static returned {rc}"
    st = ctypes.c_int32(-1)
    assert lib.lco_radix_permute_static_status(ctypes.byref(st), _stream()) == 0
    assert st.value == 0, f"device status {st.value} after lco_radix_permute_static"
    return liv_out, val_out


def test_static_permute_matches_workspace_entry_point_twice():
    """Two calls in a row (different shapes, orders and key widths) agree
    bit-for-bit with lco_radix_permute, which uses a caller workspace, and
    with the oracle."""
    cases = [([31, 17, 63, 15], 50_000, [1, 3, 0, 2], 1),      # odd dims, 2 radix passes
             ([64, 64, 64], MAX_NNZ, [0, 2, 1], 2)]             # maximum size, different plan
    for dims, nnz, new_sig, seed in cases:
        t = _tensor(dims, nnz, seed)
        ref = lco.radix_permute(t, new_sig)
        liv, val = _static_permute(t, new_sig)
        assert torch.equal(liv, ref.liv)
        assert torch.equal(val.view(torch.int64), ref.val.view(torch.int64))
        ol, ov = oracle.permute(t.dims, t.sig, new_sig, t.liv.cpu().numpy(), t.val.cpu().numpy())
        assert np.array_equal(liv.cpu().numpy(), ol)
        assert np.array_equal(val.cpu().numpy().view(np.int64), ov.view(np.int64))


def test_static_permute_rejects_oversized_input():
    lib = lco.load()
    sh = lco.make_shape([1 << 10, 1 << 10], [1, 0], MAX_NNZ + 1)
    sig = (ctypes.c_int32 * lco.MAX_ORDER)(0, 1)
    rc = lib.lco_radix_permute_static(ctypes.byref(sh), sig, None, None, None, None, None)
    assert rc == 9   # LCO_ERR_TOO_LARGE, before any device work
    assert lib.lco_radix_permute_static_status(None, None) == 1   # LCO_ERR_INVALID
