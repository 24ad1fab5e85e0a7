"""ctypes declarations of the gbspmv C ABI (include/gbspmv.h).

Loading fails loudly: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_longlong

GBS_OK = 0
GBS_EINVAL = -1
GBS_EALIGN = -2
GBS_EDTYPE = -3
GBS_ECUDA = -4
GBS_EINDEX = -5
GBS_ETIMEOUT = -6
GBS_ENOMEM = -7
GBS_EUNSUPPORTED = -8

GBS_F64 = 0
GBS_F32 = 1

VARIANT_AUTO = 0
VARIANT_ROWS = 1
VARIANT_MERGE = 2
VARIANT_ROWS_TMA = 3
VARIANT_MERGE_DIRECT = 4

PLAN_TUNE = 1
PLAN_CHECK = 2
PLAN_EMULATE = 4


class gbs_config(ctypes.Structure):
    _fields_ = [("variant", I32), ("lanes", I32), ("threads", I32), ("tile_nnz", I32), ("items", I32), ("emul", I32),
                ("relabel", I32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class gbs_stats(ctypes.Structure):
    _fields_ = [("m", I32), ("n", I32), ("nnz", I32), ("max_row", I32), ("empty_rows", I32),
                ("mean_row", ctypes.c_double), ("cv_row", ctypes.c_double),
                ("rows_over_32", I64), ("rows_over_256", I64), ("rows_over_4096", I64)]

    def as_dict(self) -> dict:
        return {f: (float(getattr(self, f)) if t is ctypes.c_double else int(getattr(self, f))) for f, t in self._fields_}


# name -> (restype, argtypes)
SIGNATURES = {
    "gbs_version": (I32, []),
    "gbs_fp64_probe": (I32, [P, I32, I32, I32, P]),
    "gbs_wait_probe": (I32, [I64, P]),
    "gbs_status_string": (ctypes.c_char_p, [I32]),
    "gbs_last_error": (ctypes.c_char_p, []),
    "gbs_validate_csr": (I32, [I32, I32, I32, P, P, P]),
    "gbs_csr_stats": (I32, [I32, I32, I32, P, ctypes.POINTER(gbs_stats), P]),
    "gbs_default_config": (I32, [ctypes.POINTER(gbs_stats), I32, I32, ctypes.POINTER(gbs_config)]),
    "spmv_csr": (I32, [I32, I32, I32, P, P, P, I32, P, P, P]),
    "spmv_csr_cfg": (I32, [I32, I32, I32, P, P, P, I32, P, P, ctypes.POINTER(gbs_config), P]),
    "spmv_csr_noalloc": (I32, [I32, I32, I32, P, P, P, I32, P, P, P]),
    "spmm_csr": (I32, [I32, I32, I32, P, P, P, I32, I32, P, I32, P, I32, P]),
    "spmm_csr_cfg": (I32, [I32, I32, I32, P, P, P, I32, I32, P, I32, P, I32, ctypes.POINTER(gbs_config), P]),
    "gbs_plan_create": (I32, [ctypes.POINTER(P), I32, I32, I32, P, P, I32, I32, I32, P]),
    "gbs_plan_destroy": (I32, [P]),
    "gbs_plan_get_config": (I32, [P, ctypes.POINTER(gbs_config)]),
    "gbs_plan_set_config": (I32, [P, ctypes.POINTER(gbs_config)]),
    "gbs_plan_get_stats": (I32, [P, ctypes.POINTER(gbs_stats)]),
    "gbs_plan_relabel_ids": (I32, [P, P, P]),
    "spmv_csr_plan": (I32, [P, P, P, P, P]),
    "gbs_plan_status": (I32, [P, ctypes.POINTER(I32), P]),
    "spmm_csr_plan": (I32, [P, P, P, I32, P, I32, P]),
    "gbs_transpose_plan": (I32, [ctypes.POINTER(P), I32, I32, I32, P, P, P]),
    "gbs_tplan_arrays": (I32, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]),
    "gbs_tplan_export": (I32, [P, P, P, P, P]),
    "gbs_tplan_destroy": (I32, [P]),
    "gbs_tplan_prepare": (I32, [P, I32, I32, I32, P]),
    "gbs_rcm": (I32, [I32, I32, P, P, P, P]),
    "gbs_permute_csr": (I32, [I32, I32, P, P, P, I32, P, P, P, P, P]),
    "gbs_bcsr_create": (I32, [ctypes.POINTER(P), I32, I32, I32, P, P, P, I32, I32, I32, P]),
    "gbs_bcsr_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(I32),
                            ctypes.POINTER(I32)]),
    "gbs_bcsr_arrays": (I32, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]),
    "spmv_bcsr": (I32, [P, P, P, P]),
    "gbs_bcsr_destroy": (I32, [P]),
    "gbs_ucld": (I32, [I32, I32, I32, P, P, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                       ctypes.POINTER(ctypes.c_longlong), P]),
    "gbs_tplan_set_config": (I32, [P, I32, I32, ctypes.POINTER(gbs_config), P]),
    "gbs_tplan_get_config": (I32, [P, I32, I32, ctypes.POINTER(gbs_config)]),
    "spmv_csr_backward": (I32, [P, P, P, P, I32, I32, P, I32, P, I32, P, I32, P, P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgbspmv.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"gbspmv CUDA library not found at {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class GbsError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        self.status = status
        msg = lib.gbs_last_error().decode(errors="replace")
        name = lib.gbs_status_string(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")


def check(status: int, where: str) -> None:
    if status != GBS_OK:
        raise GbsError(status, where)


class gbs_batch_item(ctypes.Structure):
    _fields_ = [("m", I32), ("n", I32), ("nnz", I32), ("row_ptr", P), ("col_idx", P), ("vals", P),
                ("X", P), ("ldx", I32), ("Y", P), ("ldy", I32)]


SIGNATURES.update({
    "spmv_csr_batched_plan": (I32, [ctypes.POINTER(P), I32, ctypes.POINTER(gbs_batch_item), I32, I32, I32, P]),
    "spmv_csr_batched_plan_cfg": (I32, [ctypes.POINTER(P), I32, ctypes.POINTER(gbs_batch_item), I32, I32, I32,
                                        ctypes.POINTER(gbs_config), P]),
    "spmv_csr_batched": (I32, [P, P, P, P]),
    "spmv_csr_batched_looped": (I32, [P, P]),
    "spmv_csr_batched_info": (I32, [P, ctypes.POINTER(gbs_config), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                    ctypes.POINTER(I32)]),
    "spmv_csr_batched_offsets": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                       ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "spmv_csr_batched_destroy": (I32, [P]),
})
