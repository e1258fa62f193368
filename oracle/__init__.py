"""CPU oracle for the LCO hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing from the product.

The arithmetic lives in ``lco_oracle.c`` (plain C, single-threaded, built with
gcc); this module only builds it and marshals numpy arrays through ctypes.
Each wrapper names the passage of the paper that the C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lco_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "liblco_oracle.so")
_lock = threading.Lock()
_lib = None

# algorithm codes returned by dispatch (Table 4)
ALG_NAMES = ("CSR", "CSC", "DCSR", "DCSC", "CSRNA", "CSCNA", "SOP")


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: runs on x86 and Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    # -ffp-contract=off: every product and sum is rounded as written (no
    # fused multiply-add on targets that have one), the same on x86 and Arm
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
            _lib.lco_oracle_dispatch.restype = ctypes.c_int
            _lib.lco_oracle_sparsity_class.restype = ctypes.c_int
            _lib.lco_oracle_free.argtypes = [ctypes.c_void_p]
        return _lib


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def linearise(dims, sig, coords):
    """Sec. 3.1 LIV formula: coords is (nnz, order); sig[0] least significant."""
    lib = _load()
    dims, sig, coords = _i64(dims), _i32(sig), _i64(coords).reshape(-1, len(dims))
    out = np.empty(coords.shape[0], dtype=np.int64)
    _check(lib.lco_oracle_linearise(ctypes.c_int32(len(dims)), _p(dims), _p(sig),
                                    ctypes.c_int64(coords.shape[0]), _p(coords), _p(out)),
           "linearise")
    return out


def delinearise(dims, sig, liv):
    lib = _load()
    dims, sig, liv = _i64(dims), _i32(sig), _i64(liv)
    out = np.empty((liv.shape[0], len(dims)), dtype=np.int64)
    _check(lib.lco_oracle_delinearise(ctypes.c_int32(len(dims)), _p(dims), _p(sig),
                                      ctypes.c_int64(liv.shape[0]), _p(liv), _p(out)),
           "delinearise")
    return out


def relinearise(dims, sig_old, sig_new, liv):
    """Sec. 3.1 LIV shuffle."""
    lib = _load()
    dims, so, sn, liv = _i64(dims), _i32(sig_old), _i32(sig_new), _i64(liv)
    out = np.empty_like(liv)
    _check(lib.lco_oracle_relinearise(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                      ctypes.c_int64(liv.shape[0]), _p(liv), _p(out)),
           "relinearise")
    return out


def permute(dims, sig_old, sig_new, liv, val):
    """Permutation by definition (Sec. 4): relinearise then sort by the new LIV."""
    lib = _load()
    dims, so, sn, liv, val = _i64(dims), _i32(sig_old), _i32(sig_new), _i64(liv), _f64(val)
    lo, vo = np.empty_like(liv), np.empty_like(val)
    _check(lib.lco_oracle_permute(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                  ctypes.c_int64(liv.shape[0]), _p(liv), _p(val), _p(lo), _p(vo)),
           "permute")
    return lo, vo


def _u64pairs(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("wide LIVs are an (nnz, 2) uint64 array: low word, high word")
    return a


def relinearise_wide(dims, sig_old, sig_new, liv):
    """Sec. 3.1 LIV shuffle with unsigned 128-bit LIVs (Sec. 7 future work):
    liv is (nnz, 2) uint64, low word first."""
    lib = _load()
    dims, so, sn, liv = _i64(dims), _i32(sig_old), _i32(sig_new), _u64pairs(liv)
    out = np.empty_like(liv)
    _check(lib.lco_oracle_relinearise_wide(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                           ctypes.c_int64(liv.shape[0]), _p(liv), _p(out)),
           "relinearise_wide")
    return out


def permute_wide(dims, sig_old, sig_new, liv, val):
    """Permutation by definition (Sec. 4) with unsigned 128-bit LIVs."""
    lib = _load()
    dims, so, sn, liv, val = _i64(dims), _i32(sig_old), _i32(sig_new), _u64pairs(liv), _f64(val)
    lo, vo = np.empty_like(liv), np.empty_like(val)
    _check(lib.lco_oracle_permute_wide(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                       ctypes.c_int64(liv.shape[0]), _p(liv), _p(val), _p(lo), _p(vo)),
           "permute_wide")
    return lo, vo


def contract_wide(A, B, modes_a, modes_b):
    """Contraction by definition with wide (128-bit) LIVs: A and B are dicts
    with dims, sig, liv ((nnz, 2) uint64, low word first) and val.  Returns
    (liv_c (nnz_c, 2) uint64, val_c, abs_c), C row-major over (A free modes,
    B free modes)."""
    lib = _load()
    da, sa, la, va = _i64(A["dims"]), _i32(A["sig"]), _u64pairs(A["liv"]), _f64(A["val"])
    db, sb, lb, vb = _i64(B["dims"]), _i32(B["sig"]), _u64pairs(B["liv"]), _f64(B["val"])
    ma, mb = _i32(modes_a), _i32(modes_b)
    nnz_c = ctypes.c_int64()
    pl, pv, pa = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.lco_oracle_contract_wide(
        ctypes.c_int32(len(da)), _p(da), _p(sa), ctypes.c_int64(la.shape[0]), _p(la), _p(va),
        ctypes.c_int32(len(db)), _p(db), _p(sb), ctypes.c_int64(lb.shape[0]), _p(lb), _p(vb),
        ctypes.c_int32(len(ma)), _p(ma), _p(mb),
        ctypes.byref(nnz_c), ctypes.byref(pl), ctypes.byref(pv), ctypes.byref(pa))
    _check(rc, "contract_wide")
    n = nnz_c.value
    try:
        if n == 0:
            return np.empty((0, 2), np.uint64), np.empty(0, np.float64), np.empty(0, np.float64)
        liv = np.ctypeslib.as_array(ctypes.cast(pl, ctypes.POINTER(ctypes.c_uint64)), (n, 2)).copy()
        val = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_double)), (n,)).copy()
        ab = np.ctypeslib.as_array(ctypes.cast(pa, ctypes.POINTER(ctypes.c_double)), (n,)).copy()
        return liv, val, ab
    finally:
        for p in (pl, pv, pa):
            if p.value:
                lib.lco_oracle_free(p)


def rp_permute(dims, sig_old, sig_new, liv, val):
    """The RP algorithm of Sec. 4.1 (regions + stable sort on the shaved key)."""
    lib = _load()
    dims, so, sn, liv, val = _i64(dims), _i32(sig_old), _i32(sig_new), _i64(liv), _f64(val)
    lo, vo = np.empty_like(liv), np.empty_like(val)
    _check(lib.lco_oracle_rp_permute(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                     ctypes.c_int64(liv.shape[0]), _p(liv), _p(val), _p(lo), _p(vo)),
           "rp_permute")
    return lo, vo


def rp_classify(sig_old, sig_new):
    """Sec. 4.1: per-mode flag, 1 = rearrangement index, 0 = resting index."""
    lib = _load()
    so, sn = _i32(sig_old), _i32(sig_new)
    out = np.zeros(len(so), dtype=np.int32)
    _check(lib.lco_oracle_rp_classify(ctypes.c_int32(len(so)), _p(so), _p(sn), _p(out)),
           "rp_classify")
    return out


def rp_keyspec(dims, sig_old, sig_new):
    """Sec. 4.1 shaving parameters: (m_top, m_low, n_rearr)."""
    lib = _load()
    dims, so, sn = _i64(dims), _i32(sig_old), _i32(sig_new)
    mt, ml, nr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib.lco_oracle_rp_keyspec(ctypes.c_int32(len(dims)), _p(dims), _p(so), _p(sn),
                                     ctypes.byref(mt), ctypes.byref(ml), ctypes.byref(nr)),
           "rp_keyspec")
    return mt.value, ml.value, nr.value


def contract(A, B, modes_a, modes_b, entry_a=(), entry_b=()):
    """Contraction by definition.  A and B are dicts with dims, sig, liv, val.

    Returns (liv_c, val_c, abs_c) with C row-major over (entrywise pairs, A
    free modes, B free modes); abs_c is the per-entry sum of |a||b| used by
    the tolerance.  entry_a/entry_b pair up shared modes that are kept, not
    summed (Sec. 5's entrywise products).
    """
    lib = _load()
    da, sa, la, va = _i64(A["dims"]), _i32(A["sig"]), _i64(A["liv"]), _f64(A["val"])
    db, sb, lb, vb = _i64(B["dims"]), _i32(B["sig"]), _i64(B["liv"]), _f64(B["val"])
    ma, mb = _i32(modes_a), _i32(modes_b)
    ea, eb = _i32(entry_a), _i32(entry_b)
    nnz_c = ctypes.c_int64()
    pl, pv, pa = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.lco_oracle_contract_ew(
        ctypes.c_int32(len(da)), _p(da), _p(sa), ctypes.c_int64(la.shape[0]), _p(la), _p(va),
        ctypes.c_int32(len(db)), _p(db), _p(sb), ctypes.c_int64(lb.shape[0]), _p(lb), _p(vb),
        ctypes.c_int32(len(ma)), _p(ma), _p(mb), ctypes.c_int32(len(ea)), _p(ea), _p(eb),
        ctypes.byref(nnz_c), ctypes.byref(pl), ctypes.byref(pv), ctypes.byref(pa))
    _check(rc, "contract")
    n = nnz_c.value
    try:
        if n == 0:
            return (np.empty(0, np.int64), np.empty(0, np.float64), np.empty(0, np.float64))
        liv = np.ctypeslib.as_array(ctypes.cast(pl, ctypes.POINTER(ctypes.c_int64)), (n,)).copy()
        val = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_double)), (n,)).copy()
        ab = np.ctypeslib.as_array(ctypes.cast(pa, ctypes.POINTER(ctypes.c_double)), (n,)).copy()
        return liv, val, ab
    finally:
        for p in (pl, pv, pa):
            if p.value:
                lib.lco_oracle_free(p)


def flops(A, B, modes_a, modes_b):
    """Sec. 5.2: f, the number of scalar products of the contraction."""
    lib = _load()
    da, sa, la = _i64(A["dims"]), _i32(A["sig"]), _i64(A["liv"])
    db, sb, lb = _i64(B["dims"]), _i32(B["sig"]), _i64(B["liv"])
    ma, mb = _i32(modes_a), _i32(modes_b)
    f = ctypes.c_int64()
    _check(lib.lco_oracle_flops(
        ctypes.c_int32(len(da)), _p(da), _p(sa), ctypes.c_int64(la.shape[0]), _p(la),
        ctypes.c_int32(len(db)), _p(db), _p(sb), ctypes.c_int64(lb.shape[0]), _p(lb),
        ctypes.c_int32(len(ma)), _p(ma), _p(mb), ctypes.byref(f)), "flops")
    return f.value


def sparsity_class(rows, cols, nnz):
    """0 sparse, 1 row-sparse, 2 column-sparse, 3 index-sparse (ratio > 3)."""
    return _load().lco_oracle_sparsity_class(ctypes.c_int64(rows), ctypes.c_int64(cols),
                                             ctypes.c_int64(nnz))


def dispatch(m, k, n, nnz_a, nnz_b, perm_row=0, perm_col=0):
    """Table 4 choice; returns the algorithm name."""
    code = _load().lco_oracle_dispatch(ctypes.c_int64(m), ctypes.c_int64(k), ctypes.c_int64(n),
                                       ctypes.c_int64(nnz_a), ctypes.c_int64(nnz_b),
                                       ctypes.c_int32(perm_row), ctypes.c_int32(perm_col))
    return ALG_NAMES[code]


def sort(liv, val):
    """Entries in ascending LIV order (stable for equal LIVs): Sec. 3.2."""
    lib = _load()
    l, v = _i64(liv), _f64(val)
    n = l.shape[0]
    lo, vo = np.empty(n, np.int64), np.empty(n, np.float64)
    _check(lib.lco_oracle_sort(ctypes.c_int64(n), _p(l), _p(v), _p(lo), _p(vo)), "sort")
    return lo, vo


def add(alpha, A, beta, B):
    """alpha*A + beta*B for sorted LCO dicts in the same dims and order
    (union of entries, structural zeros kept): Sec. 3.2, Eq. 4's sum."""
    lib = _load()
    la, va, lb, vb = _i64(A["liv"]), _f64(A["val"]), _i64(B["liv"]), _f64(B["val"])
    n = la.shape[0] + lb.shape[0]
    lc, vc = np.empty(max(n, 1), np.int64), np.empty(max(n, 1), np.float64)
    nc = ctypes.c_int64()
    _check(lib.lco_oracle_add(ctypes.c_double(alpha), ctypes.c_int64(la.shape[0]), _p(la), _p(va),
                              ctypes.c_double(beta), ctypes.c_int64(lb.shape[0]), _p(lb), _p(vb),
                              _p(lc), _p(vc), ctypes.byref(nc)), "add")
    return lc[:nc.value].copy(), vc[:nc.value].copy()
