"""GB300 (sm_103a) sparse-tensor rearrangement and multiplication over the
linearised-coordinate (LCO) format (Harrison & Joseph, arXiv 1802.02619).

This module is a thin ctypes binding over the C ABI declared in
``include/lco.h`` (library ``_lib/liblco.so``).  It only marshals arguments:
every step of the hot path runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _build

MAX_ORDER = 16
ALG_NAMES = ("CSR", "CSC", "DCSR", "DCSC", "CSRNA", "CSCNA", "SOP")
ALG = {name: i for i, name in enumerate(ALG_NAMES)}

STATUS = {
    0: "ok", 1: "invalid argument", 2: "index space exceeds the LIV range (2^63-1; 2^127-1 for wide LIVs)", 3: "unsorted input",
    4: "workspace too small", 5: "device wait timed out", 6: "CUDA runtime error",
    7: "admission refused", 8: "output capacity too small", 9: "input exceeds the fixed scratch",
}


class LcoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} (status {status})")


class Shape(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("sig", ctypes.c_int32 * MAX_ORDER),
                ("dims", ctypes.c_int64 * MAX_ORDER), ("nnz", ctypes.c_int64)]


class RpInfo(ctypes.Structure):
    _fields_ = [("n_rearr", ctypes.c_int32), ("is_rearr", ctypes.c_int32 * MAX_ORDER),
                ("m_top", ctypes.c_int64), ("m_low", ctypes.c_int64), ("key_bits", ctypes.c_int32),
                ("digit_bits", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("segments", ctypes.c_int32)]


class RpWideInfo(ctypes.Structure):
    _fields_ = [("n_rearr", ctypes.c_int32), ("key_bits", ctypes.c_int32), ("chunks", ctypes.c_int32),
                ("passes", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int32), ("transposed", ctypes.c_int32),
                ("class_a", ctypes.c_int32), ("class_b", ctypes.c_int32),
                ("permute_a", ctypes.c_int32), ("permute_b", ctypes.c_int32),
                ("m", ctypes.c_int64), ("k", ctypes.c_int64), ("n", ctypes.c_int64),
                ("c_shape", Shape)]


class ContractResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("alg", ctypes.c_int32), ("nnz_c", ctypes.c_int64),
                ("f", ctypes.c_int64), ("nzr_b", ctypes.c_int64)]


class TimingRecord(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("ms", ctypes.c_float)]


class Tune(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int32), ("max_digit_bits", ctypes.c_int32), ("radix_order", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("a", Shape), ("b", Shape), ("ncontract", ctypes.c_int32),
                ("modes_a", ctypes.c_int32 * MAX_ORDER), ("modes_b", ctypes.c_int32 * MAX_ORDER),
                ("alg", ctypes.c_int32), ("max_digit_bits", ctypes.c_int32), ("radix_order", ctypes.c_int32)]


class Operands(ctypes.Structure):
    _fields_ = [("a_liv", ctypes.c_void_p), ("a_val", ctypes.c_void_p), ("b_liv", ctypes.c_void_p),
                ("b_val", ctypes.c_void_p), ("c_liv", ctypes.c_void_p), ("c_val", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t), ("nslots", ctypes.c_int32),
                ("device", ctypes.c_int32), ("nworkers", ctypes.c_int32)]


class ServeResult(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32), ("alg", ctypes.c_int32), ("c", Shape),
                ("c_liv", ctypes.c_void_p), ("c_val", ctypes.c_void_p), ("f", ctypes.c_int64),
                ("submit_us", ctypes.c_double), ("done_us", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("pool_used", ctypes.c_size_t),
                ("pool_peak", ctypes.c_size_t), ("pool_bytes", ctypes.c_size_t)]


_lib = None
_lock = threading.Lock()

_SIGNATURES = {
    "lco_status_str": ([ctypes.c_int32], ctypes.c_char_p),
    "lco_build_arch": ([], ctypes.c_int32),
    "lco_workspace_status": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p], ctypes.c_int32),
    "lco_timing_enable": ([ctypes.c_int32], ctypes.c_int32),
    "lco_timing_read": ([ctypes.POINTER(TimingRecord), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
                        ctypes.c_int32),
    "lco_launch_count": ([], ctypes.c_int64),
    "lco_relinearise": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p], ctypes.c_int32),
    "lco_radix_permute_info": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.POINTER(RpInfo)],
                               ctypes.c_int32),
    "lco_radix_permute_workspace": ([ctypes.POINTER(Shape), ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_radix_permute": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                           ctypes.c_void_p], ctypes.c_int32),
    "lco_radix_permute_static": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "lco_radix_permute_static_status": ([ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p], ctypes.c_int32),
    "lco_relinearise_wide": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p], ctypes.c_int32),
    "lco_radix_permute_wide_info": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.POINTER(RpWideInfo)],
                                    ctypes.c_int32),
    "lco_radix_permute_wide_workspace": ([ctypes.POINTER(Shape), ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_radix_permute_wide": ([ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_wide_plan": ([ctypes.POINTER(Shape), ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_contract_wide_plan_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_wide_info": ([ctypes.c_void_p, ctypes.POINTER(Shape), ctypes.POINTER(ctypes.c_int32)],
                               ctypes.c_int32),
    "lco_contract_wide_workspace": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)],
                                    ctypes.c_int32),
    "lco_contract_wide_symbolic": ([ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_void_p, ctypes.c_size_t,
                                                                                ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_wide_numeric": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_wide_result_get": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ContractResult),
                                      ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_plan": ([ctypes.POINTER(Shape), ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_plan_get_info": ([ctypes.c_void_p, ctypes.POINTER(PlanInfo)], ctypes.c_int32),
    "lco_plan_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_workspace": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)],
                               ctypes.c_int32),
    "lco_contract_symbolic": ([ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_void_p, ctypes.c_size_t,
                                                                          ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_numeric": ([ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_void_p,
                                                                         ctypes.c_size_t, ctypes.c_void_p],
                             ctypes.c_int32),
    "lco_contract": ([ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_void_p,
                                                                 ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_contract_result_get": ([ctypes.c_void_p, ctypes.POINTER(ContractResult), ctypes.c_void_p],
                                ctypes.c_int32),
    "lco_contract_plan_ex": ([ctypes.POINTER(Shape), ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.POINTER(Tune), ctypes.POINTER(ctypes.c_void_p)],
                             ctypes.c_int32),
    "lco_contract_plan_entrywise": ([ctypes.POINTER(Shape), ctypes.POINTER(Shape), ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(Tune), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_batch_plan": ([ctypes.c_int32, ctypes.POINTER(Problem), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
                       ctypes.c_int32),
    "lco_batch_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "lco_batch_info": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(PlanInfo)], ctypes.c_int32),
    "lco_batch_workspace": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_batch_symbolic": ([ctypes.c_void_p, ctypes.POINTER(Operands), ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_batch_numeric": ([ctypes.c_void_p, ctypes.POINTER(Operands), ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_batch_contract": ([ctypes.c_void_p, ctypes.POINTER(Operands), ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_batch_results": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ContractResult),
                          ctypes.c_void_p], ctypes.c_int32),
    "lco_selftest_wait": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p], ctypes.c_int32),
    "lco_sort_workspace": ([ctypes.POINTER(Shape), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_sort": ([ctypes.POINTER(Shape)] + [ctypes.c_void_p] * 5 + [ctypes.c_size_t, ctypes.c_void_p],
                 ctypes.c_int32),
    "lco_add_workspace": ([ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_add": ([ctypes.POINTER(Shape), ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int32),
    "lco_add_result": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                        ctypes.c_void_p], ctypes.c_int32),
    "lco_pool_create": ([ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_pool_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "lco_pool_alloc": ([ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_pool_free": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
    "lco_pool_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                        ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "lco_serve_create": ([ctypes.POINTER(ServeConfig), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
    "lco_serve_destroy": ([ctypes.c_void_p], ctypes.c_int32),
    "lco_serve_put": ([ctypes.c_void_p, ctypes.POINTER(Shape), ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.POINTER(ctypes.c_int64)], ctypes.c_int32),
    "lco_serve_drop": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int32),
    "lco_serve_submit": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int32),
    "lco_serve_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ServeResult)], ctypes.c_int32),
    "lco_serve_wait": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ServeResult)],
                       ctypes.c_int32),
    "lco_serve_release": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int32),
    "lco_serve_get_stats": ([ctypes.c_void_p, ctypes.POINTER(ServeStats)], ctypes.c_int32),
}


def lib_path() -> str:
    return _build.SO_PATH


def load(build_if_missing: bool = True):
    """Load liblco.so (building it with nvcc if it is missing or stale).

    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and _build.is_stale():
            _build.build()
        if not os.path.exists(_build.SO_PATH):
            raise RuntimeError(f"CUDA library not built: {_build.SO_PATH}")
        lib = ctypes.CDLL(_build.SO_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols():
    return sorted(_SIGNATURES)


def timing_enable(on: bool = True):
    """Bracket every library kernel launch with CUDA events (outside graph capture)."""
    _check(load().lco_timing_enable(1 if on else 0), "lco_timing_enable")


def timing_read():
    """[(kernel name, ms)] of the launches recorded since timing was enabled."""
    lib = load()
    recs = (TimingRecord * 4096)()
    n = ctypes.c_int32()
    _check(lib.lco_timing_read(recs, 4096, ctypes.byref(n)), "lco_timing_read")
    return [(recs[i].name.decode(), float(recs[i].ms)) for i in range(n.value)]


def launch_count() -> int:
    return int(load().lco_launch_count())


def _check(rc: int, what: str):
    if rc != 0:
        raise LcoError(rc, what)


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _sig_arr(sig):
    a = (ctypes.c_int32 * MAX_ORDER)()
    for i, s in enumerate(sig):
        a[i] = int(s)
    return a


def make_shape(dims: Sequence[int], sig: Sequence[int], nnz: int) -> Shape:
    if len(dims) != len(sig) or not (1 <= len(dims) <= MAX_ORDER):
        raise ValueError("dims and sig must have the same length (1..16)")
    s = Shape()
    s.order = len(dims)
    for i, (d, g) in enumerate(zip(dims, sig)):
        s.dims[i] = int(d)
        s.sig[i] = int(g)
    s.nnz = int(nnz)
    return s


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda):
            raise ValueError("LCO arrays must be CUDA tensors")


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Zero-filled device workspace of at least nbytes (256-byte aligned)."""
    n = max(256, (int(nbytes) + 255) // 256 * 256)
    return torch.zeros(n, dtype=torch.uint8, device=device or "cuda")


@dataclass
class LcoTensor:
    """An LCO tensor: int64 LIVs (strictly ascending in order `sig`) and
    float64 values, both on the GPU.  sig[0] is the least significant mode."""
    dims: list
    sig: list
    liv: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.liv.numel())

    @property
    def order(self) -> int:
        return len(self.dims)

    def shape(self) -> Shape:
        return make_shape(self.dims, self.sig, self.nnz)

    @staticmethod
    def from_host(T: dict, device="cuda") -> "LcoTensor":
        liv = torch.as_tensor(T["liv"], dtype=torch.int64).to(device)
        val = torch.as_tensor(T["val"], dtype=torch.float64).to(device)
        return LcoTensor(list(T["dims"]), list(T["sig"]), liv, val)


# ---------------------------------------------------------------------------
# Re-linearisation and permutation
# ---------------------------------------------------------------------------

def relinearise(t: LcoTensor, new_sig, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """LIV shuffle (Sec. 3.1): the LIVs of t in order new_sig (element order kept)."""
    lib = load()
    _require_cuda(t.liv)
    if out is None:
        out = torch.empty_like(t.liv)
    sh = t.shape()
    _check(lib.lco_relinearise(ctypes.byref(sh), _sig_arr(new_sig), _ptr(t.liv), _ptr(out), _stream(stream)),
           "lco_relinearise")
    return out


def radix_permute_info(dims, sig, new_sig, nnz: int = 0) -> dict:
    lib = load()
    sh = make_shape(dims, sig, nnz)
    info = RpInfo()
    _check(lib.lco_radix_permute_info(ctypes.byref(sh), _sig_arr(new_sig), ctypes.byref(info)),
           "lco_radix_permute_info")
    return {"n_rearr": info.n_rearr, "is_rearr": [info.is_rearr[i] for i in range(len(dims))],
            "m_top": info.m_top, "m_low": info.m_low, "key_bits": info.key_bits,
            "digit_bits": info.digit_bits, "passes": info.passes, "segments": info.segments}


class Permuter:
    """Reusable permutation of tensors of one shape to one new order (holds
    the workspace so repeated calls allocate nothing)."""

    def __init__(self, dims, sig, new_sig, nnz: int, device="cuda"):
        self.lib = load()
        self.dims, self.sig, self.new_sig = list(dims), list(sig), list(new_sig)
        self.nnz = int(nnz)
        self.sh = make_shape(self.dims, self.sig, self.nnz)
        self._new = _sig_arr(self.new_sig)
        nb = ctypes.c_size_t()
        _check(self.lib.lco_radix_permute_workspace(ctypes.byref(self.sh), self._new, ctypes.byref(nb)),
               "lco_radix_permute_workspace")
        self.ws = workspace(nb.value, device)

    def __call__(self, liv, val, liv_out=None, val_out=None, stream=None):
        _require_cuda(liv, val)
        if liv.numel() != self.nnz:
            raise ValueError("nnz differs from the planned size")
        liv_out = torch.empty_like(liv) if liv_out is None else liv_out
        val_out = torch.empty_like(val) if val_out is None else val_out
        _check(self.lib.lco_radix_permute(ctypes.byref(self.sh), self._new, _ptr(liv), _ptr(val), _ptr(liv_out),
                                          _ptr(val_out), _ptr(self.ws), ctypes.c_size_t(self.ws.numel()),
                                          _stream(stream)), "lco_radix_permute")
        return liv_out, val_out

    def device_status(self, stream=None) -> int:
        st = ctypes.c_int32()
        _check(self.lib.lco_workspace_status(_ptr(self.ws), ctypes.byref(st), _stream(stream)),
               "lco_workspace_status")
        return st.value


def radix_permute(t: LcoTensor, new_sig, stream=None) -> LcoTensor:
    """Rearrange t into lexicographic order new_sig (Sec. 4.1, RP)."""
    p = Permuter(t.dims, t.sig, new_sig, t.nnz, device=t.liv.device)
    liv, val = p(t.liv, t.val, stream=stream)
    st = p.device_status(stream)
    if st != 0:
        raise LcoError(st, "lco_radix_permute (device)")
    return LcoTensor(list(t.dims), list(new_sig), liv, val)


# ---------------------------------------------------------------------------
# Wide LIVs (unsigned 128-bit; dims multiplying past 2^63 - 1)
# ---------------------------------------------------------------------------

def _wide(liv: torch.Tensor):
    if liv.dtype != torch.int64 or liv.dim() != 2 or liv.shape[1] != 2 or not liv.is_contiguous():
        raise ValueError("wide LIVs are a contiguous (nnz, 2) int64 tensor: low word, high word (bit patterns)")


def relinearise_wide(dims, sig, new_sig, liv: torch.Tensor, out: Optional[torch.Tensor] = None,
                     stream=None) -> torch.Tensor:
    """LIV shuffle (Sec. 3.1) of wide LIVs; element order kept."""
    lib = load()
    _require_cuda(liv)
    _wide(liv)
    out = torch.empty_like(liv) if out is None else out
    sh = make_shape(dims, sig, liv.shape[0])
    _check(lib.lco_relinearise_wide(ctypes.byref(sh), _sig_arr(new_sig), _ptr(liv), _ptr(out), _stream(stream)),
           "lco_relinearise_wide")
    return out


def radix_permute_wide_info(dims, sig, new_sig, nnz: int = 0) -> dict:
    lib = load()
    sh = make_shape(dims, sig, nnz)
    info = RpWideInfo()
    _check(lib.lco_radix_permute_wide_info(ctypes.byref(sh), _sig_arr(new_sig), ctypes.byref(info)),
           "lco_radix_permute_wide_info")
    return {"n_rearr": info.n_rearr, "key_bits": info.key_bits, "chunks": info.chunks, "passes": info.passes}


class WidePermuter:
    """Reusable permutation of wide-LIV tensors of one shape to one order."""

    def __init__(self, dims, sig, new_sig, nnz: int, device="cuda"):
        self.lib = load()
        self.nnz = int(nnz)
        self.sh = make_shape(dims, sig, self.nnz)
        self._new = _sig_arr(new_sig)
        nb = ctypes.c_size_t()
        _check(self.lib.lco_radix_permute_wide_workspace(ctypes.byref(self.sh), self._new, ctypes.byref(nb)),
               "lco_radix_permute_wide_workspace")
        self.ws = workspace(nb.value, device)

    def __call__(self, liv, val, liv_out=None, val_out=None, stream=None):
        _require_cuda(liv, val)
        _wide(liv)
        if liv.shape[0] != self.nnz or val.numel() != self.nnz:
            raise ValueError("nnz differs from the planned size")
        liv_out = torch.empty_like(liv) if liv_out is None else liv_out
        val_out = torch.empty_like(val) if val_out is None else val_out
        _check(self.lib.lco_radix_permute_wide(ctypes.byref(self.sh), self._new, _ptr(liv), _ptr(val),
                                               _ptr(liv_out), _ptr(val_out), _ptr(self.ws),
                                               ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_radix_permute_wide")
        return liv_out, val_out

    def device_status(self, stream=None) -> int:
        st = ctypes.c_int32()
        _check(self.lib.lco_workspace_status(_ptr(self.ws), ctypes.byref(st), _stream(stream)),
               "lco_workspace_status")
        return st.value


def radix_permute_wide(dims, sig, new_sig, liv: torch.Tensor, val: torch.Tensor, stream=None):
    """Rearrange a wide-LIV tensor into order new_sig (Sec. 4.1 with 128-bit LIVs)."""
    p = WidePermuter(dims, sig, new_sig, liv.shape[0], device=liv.device)
    lo, vo = p(liv, val, stream=stream)
    st = p.device_status(stream)
    if st != 0:
        raise LcoError(st, "lco_radix_permute_wide (device)")
    return lo, vo


class WideContractPlan:
    """Plan for C = A x_modes B with wide (128-bit) LIVs (lco_contract_wide_*
    in include/lco.h): shapes as lists (dims may multiply past 2^63 - 1, up
    to 2^127 - 1), contracted mode pairs.  C is row-major over A's free
    modes then B's."""

    def __init__(self, a_dims, a_sig, a_nnz, b_dims, b_sig, b_nnz, modes_a, modes_b, device="cuda"):
        self.lib = load()
        self.device = device
        self.sa = make_shape(a_dims, a_sig, a_nnz)
        self.sb = make_shape(b_dims, b_sig, b_nnz)
        ma = (ctypes.c_int32 * MAX_ORDER)(*modes_a)
        mb = (ctypes.c_int32 * MAX_ORDER)(*modes_b)
        h = ctypes.c_void_p()
        _check(self.lib.lco_contract_wide_plan(ctypes.byref(self.sa), ctypes.byref(self.sb), len(modes_a), ma, mb,
                                               ctypes.byref(h)), "lco_contract_wide_plan")
        self.handle = h
        cs = Shape()
        alg = ctypes.c_int32()
        _check(self.lib.lco_contract_wide_info(h, ctypes.byref(cs), ctypes.byref(alg)), "lco_contract_wide_info")
        self.c_dims = [cs.dims[i] for i in range(cs.order)]
        self.c_sig = [cs.sig[i] for i in range(cs.order)]
        self.inner_alg = ALG_NAMES[alg.value]
        self.ws = None
        self.cap = -1

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.handle.value:
                self.lib.lco_contract_wide_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def ensure_workspace(self, cap: int):
        if cap > self.cap:
            nb = ctypes.c_size_t()
            _check(self.lib.lco_contract_wide_workspace(self.handle, int(cap), ctypes.byref(nb)),
                   "lco_contract_wide_workspace")
            self.ws = workspace(nb.value, self.device)
            self.cap = int(cap)

    def symbolic(self, a_liv, a_val, b_liv, b_val, stream=None):
        _check(self.lib.lco_contract_wide_symbolic(self.handle, _ptr(a_liv), _ptr(a_val), _ptr(b_liv), _ptr(b_val),
                                                   _ptr(self.ws), ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_contract_wide_symbolic")

    def numeric(self, c_liv, c_val, stream=None):
        _check(self.lib.lco_contract_wide_numeric(self.handle, _ptr(c_liv), _ptr(c_val), int(self.cap),
                                                  _ptr(self.ws), ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_contract_wide_numeric")

    def result(self, stream=None) -> dict:
        r = ContractResult()
        _check(self.lib.lco_contract_wide_result_get(self.handle, _ptr(self.ws), ctypes.byref(r), _stream(stream)),
               "lco_contract_wide_result_get")
        return {"status": r.status, "alg": ALG_NAMES[r.alg] if 0 <= r.alg < len(ALG_NAMES) else r.alg,
                "nnz_c": int(r.nnz_c), "f": int(r.f)}


def contract_wide(a_dims, a_sig, a_liv, a_val, b_dims, b_sig, b_liv, b_val, modes_a, modes_b, stream=None):
    """C = A x_modes B for wide-LIV tensors (liv: (nnz, 2) int64 device
    tensors holding uint64 words, low first).  Phase 1 sizes C by the
    product count f; returns (c_liv (nnz_c, 2), c_val, plan)."""
    for t in (a_liv, b_liv):
        _require_cuda(t)
        _wide(t)
    p = WideContractPlan(a_dims, a_sig, a_liv.shape[0], b_dims, b_sig, b_liv.shape[0], modes_a, modes_b,
                         device=a_liv.device)
    p.ensure_workspace(0)
    p.symbolic(a_liv, a_val, b_liv, b_val, stream)
    r = p.result(stream)
    if r["status"] != 0:
        raise LcoError(r["status"], "lco_contract_wide_symbolic (device)")
    f = r["f"]
    p.ensure_workspace(f)
    c_liv = torch.empty((max(f, 1), 2), dtype=torch.int64, device=a_liv.device)
    c_val = torch.empty(max(f, 1), dtype=torch.float64, device=a_liv.device)
    p.symbolic(a_liv, a_val, b_liv, b_val, stream)
    p.numeric(c_liv, c_val, stream)
    r = p.result(stream)
    if r["status"] != 0:
        raise LcoError(r["status"], "lco_contract_wide_numeric (device)")
    n = r["nnz_c"]
    return c_liv[:n], c_val[:n], p


# ---------------------------------------------------------------------------
# Contraction
# ---------------------------------------------------------------------------

def _alg_code(alg):
    return -1 if alg is None else (ALG[alg] if isinstance(alg, str) else int(alg))


class ContractPlan:
    """Plan for C = A x_modes B (Sec. 5.2 poly-algorithm, Table 4 dispatch).

    alg forces an algorithm (name or code); max_digit_bits caps the radix
    digit width of operand permutations and radix_order = 1 keeps them to
    LSD passes (0: high digit first when the device finds that two passes
    remain and every high-digit bucket fits one CTA) -- tuning hints."""

    def __init__(self, a_dims, a_sig, a_nnz, b_dims, b_sig, b_nnz, modes_a, modes_b, alg=None,
                 max_digit_bits=0, entry_a=(), entry_b=(), radix_order=0):
        self.lib = load()
        self.sa = make_shape(a_dims, a_sig, a_nnz)
        self.sb = make_shape(b_dims, b_sig, b_nnz)
        if len(modes_a) != len(modes_b) or len(entry_a) != len(entry_b):
            raise ValueError("modes_a/modes_b and entry_a/entry_b must pair up")
        nc, ne = len(modes_a), len(entry_a)
        self._ma = (ctypes.c_int32 * max(1, nc))(*[int(x) for x in modes_a])
        self._mb = (ctypes.c_int32 * max(1, nc))(*[int(x) for x in modes_b])
        self._ea = (ctypes.c_int32 * max(1, ne))(*[int(x) for x in entry_a])
        self._eb = (ctypes.c_int32 * max(1, ne))(*[int(x) for x in entry_b])
        tune = Tune(_alg_code(alg), int(max_digit_bits), int(radix_order))
        h = ctypes.c_void_p()
        _check(self.lib.lco_contract_plan_entrywise(ctypes.byref(self.sa), ctypes.byref(self.sb), nc, self._ma,
                                                    self._mb, ne, self._ea, self._eb, ctypes.byref(tune),
                                                    ctypes.byref(h)), "lco_contract_plan_entrywise")
        self.handle = h
        info = PlanInfo()
        _check(self.lib.lco_plan_get_info(h, ctypes.byref(info)), "lco_plan_get_info")
        cs = info.c_shape
        self.info = {"alg": ALG_NAMES[info.alg], "transposed": info.transposed, "class_a": info.class_a,
                     "class_b": info.class_b, "permute_a": info.permute_a, "permute_b": info.permute_b,
                     "m": info.m, "k": info.k, "n": info.n}
        self.c_dims = [cs.dims[i] for i in range(cs.order)]
        self.c_sig = [cs.sig[i] for i in range(cs.order)]
        self.ws = None
        self.cap = -1

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.handle.value:
                self.lib.lco_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def workspace_bytes(self, cap: int) -> int:
        nb = ctypes.c_size_t()
        _check(self.lib.lco_contract_workspace(self.handle, ctypes.c_int64(int(cap)), ctypes.byref(nb)),
               "lco_contract_workspace")
        return nb.value

    def ensure_workspace(self, cap: int, device="cuda"):
        if self.ws is None or cap > self.cap:
            old = self.ws
            self.ws = workspace(self.workspace_bytes(cap), device)
            if old is not None:
                # keep the header and phase-1 region (layout is independent of cap)
                n = min(old.numel(), self.workspace_bytes(0))
                self.ws[:n].copy_(old[:n])
            self.cap = cap
        return self.ws

    def result(self, stream=None) -> dict:
        r = ContractResult()
        _check(self.lib.lco_contract_result_get(_ptr(self.ws), ctypes.byref(r), _stream(stream)),
               "lco_contract_result_get")
        return {"status": r.status, "alg": ALG_NAMES[r.alg] if 0 <= r.alg < len(ALG_NAMES) else r.alg,
                "nnz_c": r.nnz_c, "f": r.f, "nzr_b": r.nzr_b}

    def symbolic(self, A: LcoTensor, B: LcoTensor, stream=None):
        _require_cuda(A.liv, A.val, B.liv, B.val)
        _check(self.lib.lco_contract_symbolic(self.handle, _ptr(A.liv), _ptr(A.val), _ptr(B.liv), _ptr(B.val),
                                              _ptr(self.ws), ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_contract_symbolic")

    def numeric(self, A: LcoTensor, B: LcoTensor, c_liv, c_val, stream=None):
        _check(self.lib.lco_contract_numeric(self.handle, _ptr(A.liv), _ptr(A.val), _ptr(B.liv), _ptr(B.val),
                                             _ptr(c_liv), _ptr(c_val), ctypes.c_int64(c_liv.numel()),
                                             _ptr(self.ws), ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_contract_numeric")

    def run(self, A: LcoTensor, B: LcoTensor, c_liv, c_val, stream=None):
        """Both phases, no host synchronisation (c_liv/c_val must hold >= f entries)."""
        _check(self.lib.lco_contract(self.handle, _ptr(A.liv), _ptr(A.val), _ptr(B.liv), _ptr(B.val),
                                     _ptr(c_liv), _ptr(c_val), ctypes.c_int64(c_liv.numel()),
                                     _ptr(self.ws), ctypes.c_size_t(self.ws.numel()), _stream(stream)),
               "lco_contract")


def contract(A: LcoTensor, B: LcoTensor, modes_a, modes_b, alg=None, stream=None, return_info=False,
             entry_a=(), entry_b=(), max_digit_bits=0, radix_order=0):
    """C = A x_modes B as an LCO tensor (Sec. 5.2).  entry_a/entry_b pair up
    shared modes kept in C (entrywise products, Sec. 5); C's modes are those
    pairs, A's free modes, B's free modes.  max_digit_bits and radix_order
    are the operand permutations' tuning hints (see ContractPlan).
    Synchronises twice: after phase 1 to size C by the product count f, and
    at the end to read nnz_C."""
    plan = ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, modes_a, modes_b, alg,
                        max_digit_bits=max_digit_bits, entry_a=entry_a, entry_b=entry_b,
                        radix_order=radix_order)
    dev = A.liv.device
    plan.ensure_workspace(0, dev)
    plan.symbolic(A, B, stream)
    r = plan.result(stream)
    if r["status"] != 0:
        raise LcoError(r["status"], "lco_contract_symbolic (device)")
    f = r["f"]
    plan.ensure_workspace(f, dev)
    c_liv = torch.empty(max(f, 1), dtype=torch.int64, device=dev)
    c_val = torch.empty(max(f, 1), dtype=torch.float64, device=dev)
    plan.numeric(A, B, c_liv[:f] if f else c_liv[:0], c_val[:f] if f else c_val[:0], stream)
    r = plan.result(stream)
    if r["status"] != 0:
        raise LcoError(r["status"], "lco_contract_numeric (device)")
    n = r["nnz_c"]
    C = LcoTensor(plan.c_dims, plan.c_sig, c_liv[:n], c_val[:n])
    if return_info:
        return C, dict(plan.info, **r)
    return C


# ---------------------------------------------------------------------------
# Batched contractions
# ---------------------------------------------------------------------------

def _problem(A: LcoTensor, B: LcoTensor, modes_a, modes_b, alg=None, max_digit_bits=0, radix_order=0) -> Problem:
    p = Problem()
    p.a = A.shape()
    p.b = B.shape()
    p.ncontract = len(modes_a)
    for i, (x, y) in enumerate(zip(modes_a, modes_b)):
        p.modes_a[i] = int(x)
        p.modes_b[i] = int(y)
    p.alg = _alg_code(alg)
    p.max_digit_bits = int(max_digit_bits or 0)
    p.radix_order = int(radix_order or 0)
    return p


class Batch:
    """Many independent contractions enqueued together (see lco_batch_* in
    include/lco.h).  items: list of (A, B, modes_a, modes_b[, alg[, max_digit_bits[, radix_order]]]).  The
    first call sizes every output by its product count f; `run()` then
    enqueues the whole batch with no host synchronisation and can be
    captured into a CUDA graph."""

    def __init__(self, items, nstreams: int = 16, device="cuda"):
        self.lib = load()
        self.items = [tuple(it) + (None,) * (7 - len(it)) for it in items]
        n = len(self.items)
        self.n = n
        self._probs = (Problem * n)(*[_problem(A, B, ma, mb, alg, bits, order)
                                      for A, B, ma, mb, alg, bits, order in self.items])
        h = ctypes.c_void_p()
        _check(self.lib.lco_batch_plan(n, self._probs, int(nstreams), ctypes.byref(h)), "lco_batch_plan")
        self.handle = h
        self.device = device
        self._ops = (Operands * n)()
        for i, (A, B, *_rest) in enumerate(self.items):
            self._ops[i].a_liv = A.liv.data_ptr() if A.nnz else None
            self._ops[i].a_val = A.val.data_ptr() if A.nnz else None
            self._ops[i].b_liv = B.liv.data_ptr() if B.nnz else None
            self._ops[i].b_val = B.val.data_ptr() if B.nnz else None
        # phase 1 once to learn every f
        nb = ctypes.c_size_t()
        _check(self.lib.lco_batch_workspace(h, None, ctypes.byref(nb)), "lco_batch_workspace")
        ws = workspace(nb.value, device)
        _check(self.lib.lco_batch_symbolic(h, self._ops, None, _ptr(ws), ctypes.c_size_t(ws.numel()),
                                           _stream(None)), "lco_batch_symbolic")
        res = (ContractResult * n)()
        _check(self.lib.lco_batch_results(h, None, _ptr(ws), res, _stream(None)), "lco_batch_results")
        for i in range(n):
            if res[i].status != 0:
                raise LcoError(res[i].status, f"batch problem {i} (symbolic)")
        self.f = [int(res[i].f) for i in range(n)]
        self._caps = (ctypes.c_int64 * n)(*self.f)
        del ws
        total = sum(self.f)
        self.c_liv_all = torch.empty(max(total, 1), dtype=torch.int64, device=device)
        self.c_val_all = torch.empty(max(total, 1), dtype=torch.float64, device=device)
        self.c_off = []
        off = 0
        for i in range(n):
            self.c_off.append(off)
            self._ops[i].c_liv = self.c_liv_all.data_ptr() + 8 * off if self.f[i] else None
            self._ops[i].c_val = self.c_val_all.data_ptr() + 8 * off if self.f[i] else None
            off += self.f[i]
        _check(self.lib.lco_batch_workspace(h, self._caps, ctypes.byref(nb)), "lco_batch_workspace")
        self.ws = workspace(nb.value, device)
        self.info = []
        for i in range(n):
            pi = PlanInfo()
            _check(self.lib.lco_batch_info(h, i, ctypes.byref(pi)), "lco_batch_info")
            cs = pi.c_shape
            self.info.append({"alg": ALG_NAMES[pi.alg], "c_dims": [cs.dims[k] for k in range(cs.order)],
                              "c_sig": [cs.sig[k] for k in range(cs.order)]})

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.handle.value:
                self.lib.lco_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def run(self, stream=None):
        """The whole batch as stacked products (lco_batch_contract)."""
        _check(self.lib.lco_batch_contract(self.handle, self._ops, self._caps, _ptr(self.ws),
                                           ctypes.c_size_t(self.ws.numel()), _stream(stream)), "lco_batch_contract")

    def run_per_problem(self, stream=None):
        """Every problem's two phases on their own over the stream pool
        (lco_batch_symbolic + lco_batch_numeric): the same results."""
        n = ctypes.c_size_t(self.ws.numel())
        _check(self.lib.lco_batch_symbolic(self.handle, self._ops, self._caps, _ptr(self.ws), n, _stream(stream)),
               "lco_batch_symbolic")
        _check(self.lib.lco_batch_numeric(self.handle, self._ops, self._caps, _ptr(self.ws), n, _stream(stream)),
               "lco_batch_numeric")

    def results(self, stream=None):
        res = (ContractResult * self.n)()
        _check(self.lib.lco_batch_results(self.handle, self._caps, _ptr(self.ws), res, _stream(stream)),
               "lco_batch_results")
        out = []
        for i in range(self.n):
            r = res[i]
            if r.status != 0:
                raise LcoError(r.status, f"batch problem {i}")
            o, nc = self.c_off[i], int(r.nnz_c)
            out.append(LcoTensor(self.info[i]["c_dims"], self.info[i]["c_sig"], self.c_liv_all[o:o + nc],
                                 self.c_val_all[o:o + nc]))
        return out


# ---------------------------------------------------------------------------
# Failure detection self-test
# ---------------------------------------------------------------------------

def selftest_wait(budget_cycles: int = 1_000_000, stream=None):
    """Make the library's bounded device waits run out on purpose (see
    lco_selftest_wait); returns (look-back status, mbarrier status)."""
    lib = load()
    scratch = workspace(512)
    lb, mb = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.lco_selftest_wait(_ptr(scratch), ctypes.c_int64(budget_cycles), ctypes.byref(lb), ctypes.byref(mb),
                                 _stream(stream)), "lco_selftest_wait")
    return lb.value, mb.value


# ---------------------------------------------------------------------------
# Sorting and addition
# ---------------------------------------------------------------------------

def sort(t: LcoTensor, stream=None) -> LcoTensor:
    """t's entries in ascending LIV order (Sec. 3.2); t.liv need not be
    sorted.  Equal LIVs keep their input order."""
    lib = load()
    _require_cuda(t.liv, t.val)
    sh = t.shape()
    nb = ctypes.c_size_t()
    _check(lib.lco_sort_workspace(ctypes.byref(sh), ctypes.byref(nb)), "lco_sort_workspace")
    ws = workspace(nb.value, t.liv.device)
    liv, val = torch.empty_like(t.liv), torch.empty_like(t.val)
    _check(lib.lco_sort(ctypes.byref(sh), _ptr(t.liv), _ptr(t.val), _ptr(liv), _ptr(val), _ptr(ws),
                        ctypes.c_size_t(ws.numel()), _stream(stream)), "lco_sort")
    st = ctypes.c_int32()
    _check(lib.lco_workspace_status(_ptr(ws), ctypes.byref(st), _stream(stream)), "lco_workspace_status")
    if st.value != 0:
        raise LcoError(st.value, "lco_sort (device)")
    return LcoTensor(list(t.dims), list(t.sig), liv, val)


def add(A: LcoTensor, B: LcoTensor, alpha: float = 1.0, beta: float = 1.0, stream=None) -> LcoTensor:
    """alpha*A + beta*B for two sorted tensors of the same dims and order
    (Sec. 3.2; Eq. 4's sum).  Cancelled sums stay as explicit zeros."""
    if list(A.dims) != list(B.dims) or list(A.sig) != list(B.sig):
        raise ValueError("A and B must have the same dims and order (permute one first)")
    lib = load()
    _require_cuda(A.liv, A.val, B.liv, B.val)
    sh = A.shape()
    nb = ctypes.c_size_t()
    _check(lib.lco_add_workspace(A.nnz, B.nnz, ctypes.byref(nb)), "lco_add_workspace")
    dev = A.liv.device
    ws = workspace(nb.value, dev)
    n = A.nnz + B.nnz
    c_liv = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    c_val = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    _check(lib.lco_add(ctypes.byref(sh), ctypes.c_double(alpha), _ptr(A.liv), _ptr(A.val), A.nnz,
                       ctypes.c_double(beta), _ptr(B.liv), _ptr(B.val), B.nnz, _ptr(c_liv), _ptr(c_val), _ptr(ws),
                       ctypes.c_size_t(ws.numel()), _stream(stream)), "lco_add")
    nc, st = ctypes.c_int64(), ctypes.c_int32()
    _check(lib.lco_add_result(_ptr(ws), ctypes.byref(nc), ctypes.byref(st), _stream(stream)), "lco_add_result")
    if st.value != 0:
        raise LcoError(st.value, "lco_add (device)")
    return LcoTensor(list(A.dims), list(A.sig), c_liv[:nc.value], c_val[:nc.value])


# ---------------------------------------------------------------------------
# Device memory pool and served contractions
# ---------------------------------------------------------------------------

class Pool:
    """First-fit bookkeeping over [base, base + nbytes) (see lco_pool_* in
    include/lco.h); the pool never touches the memory."""

    def __init__(self, base: int, nbytes: int):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.lco_pool_create(ctypes.c_void_p(base), ctypes.c_size_t(nbytes), ctypes.byref(h)),
               "lco_pool_create")
        self.handle = h

    def alloc(self, nbytes: int) -> Optional[int]:
        p = ctypes.c_void_p()
        rc = self.lib.lco_pool_alloc(self.handle, ctypes.c_size_t(nbytes), ctypes.byref(p))
        if rc == 4:          # LCO_ERR_OOM
            return None
        _check(rc, "lco_pool_alloc")
        return int(p.value)

    def free(self, ptr: int):
        _check(self.lib.lco_pool_free(self.handle, ctypes.c_void_p(ptr)), "lco_pool_free")

    def stats(self):
        u, pk, lf = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(self.lib.lco_pool_stats(self.handle, ctypes.byref(u), ctypes.byref(pk), ctypes.byref(lf)),
               "lco_pool_stats")
        return {"used": u.value, "peak": pk.value, "largest_free": lf.value}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.lco_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A device pointer exposed through the CUDA array interface, so that
    torch can view library-owned memory without copying."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _view(ptr, n, dtype, device):
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device=device)
    typestr = "<i8" if dtype == torch.int64 else "<f8"
    return torch.as_tensor(_DeviceArray(int(ptr), int(n), typestr), device=device)


class Server:
    """Served contractions (see lco_serve_* in include/lco.h): operands are
    put once and named by handle; submit() returns at once and a worker
    thread in the library runs each request on one of `nslots` streams."""

    def __init__(self, pool_bytes: int, nslots: int = 16, device=None, nworkers: int = 4):
        self.lib = load()
        dev = torch.device(device or "cuda")
        self.device = dev
        cfg = ServeConfig()
        cfg.pool = None
        cfg.pool_bytes = int(pool_bytes)
        cfg.nslots = int(nslots)
        cfg.device = dev.index if dev.index is not None else torch.cuda.current_device()
        cfg.nworkers = int(nworkers)
        h = ctypes.c_void_p()
        _check(self.lib.lco_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "lco_serve_create")
        self.handle = h

    def put(self, t: LcoTensor) -> int:
        sh = t.shape()
        hdl = ctypes.c_int64()
        torch.cuda.current_stream(t.liv.device).synchronize()
        _check(self.lib.lco_serve_put(self.handle, ctypes.byref(sh), _ptr(t.liv), _ptr(t.val), ctypes.byref(hdl)),
               "lco_serve_put")
        return int(hdl.value)

    def drop(self, handle: int):
        _check(self.lib.lco_serve_drop(self.handle, ctypes.c_int64(handle)), "lco_serve_drop")

    def submit(self, ha: int, hb: int, modes_a, modes_b) -> int:
        if len(modes_a) != len(modes_b):
            raise ValueError("modes_a and modes_b must pair up")
        ma, mb = _sig_arr(modes_a), _sig_arr(modes_b)
        rid = ctypes.c_uint64()
        _check(self.lib.lco_serve_submit(self.handle, ctypes.c_int64(ha), ctypes.c_int64(hb), len(modes_a), ma, mb,
                                         ctypes.byref(rid)), "lco_serve_submit")
        return int(rid.value)

    def _result(self, r: ServeResult) -> dict:
        out = {"done": bool(r.done), "status": int(r.status), "alg": ALG_NAMES[r.alg] if r.done else None,
               "f": int(r.f), "submit_us": r.submit_us, "done_us": r.done_us}
        if r.done and r.status == 0:
            c = r.c
            n = int(c.nnz)
            out["C"] = LcoTensor([c.dims[i] for i in range(c.order)], [c.sig[i] for i in range(c.order)],
                                 _view(r.c_liv, n, torch.int64, self.device),
                                 _view(r.c_val, n, torch.float64, self.device))
        return out

    def poll(self, req: int) -> dict:
        r = ServeResult()
        _check(self.lib.lco_serve_poll(self.handle, ctypes.c_uint64(req), ctypes.byref(r)), "lco_serve_poll")
        return self._result(r)

    def wait(self, req: int, timeout_us: int = -1) -> dict:
        r = ServeResult()
        _check(self.lib.lco_serve_wait(self.handle, ctypes.c_uint64(req), ctypes.c_int64(timeout_us),
                                       ctypes.byref(r)), "lco_serve_wait")
        return self._result(r)

    def release(self, req: int):
        _check(self.lib.lco_serve_release(self.handle, ctypes.c_uint64(req)), "lco_serve_release")

    def stats(self) -> dict:
        st = ServeStats()
        _check(self.lib.lco_serve_get_stats(self.handle, ctypes.byref(st)), "lco_serve_get_stats")
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.lco_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
