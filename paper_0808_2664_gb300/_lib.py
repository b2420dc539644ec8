"""ctypes loader for libtsqr_gb300.so: declares the C ABI of include/tsqr.h.

Loading fails loudly when the library has not been built; there is no other
implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsqr_gb300.so")

_lib = None
_lock = threading.Lock()

i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
pi32, pi64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)


class TsqrOpts(ctypes.Structure):
    _fields_ = [("leaf_rows", ctypes.c_int64), ("arity", ctypes.c_int32), ("flags", ctypes.c_int32)]


class TsqrBatchOpts(ctypes.Structure):
    _fields_ = [("tile_kb", ctypes.c_int32), ("arity", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# name -> (argtypes, restype); mirrors include/tsqr.h.
SIGNATURES = {
    "tsqr_factor": ([i64, i64, vp, i64, vp, i64, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "tsqr_factor_f32": ([i64, i64, vp, i64, vp, i64, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "tsqr_q_create": ([i64, i64, i32, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "tsqr_refactor": ([vp, vp, i64, vp, i64, vp], ctypes.c_int),
    "tsqr_apply_qt": ([vp, i64, vp, i64, vp], ctypes.c_int),
    "tsqr_apply_q": ([vp, i64, vp, i64, vp], ctypes.c_int),
    "tsqr_form_q": ([vp, vp, i64, vp], ctypes.c_int),
    "tsqr_form_q_mul": ([vp, i64, vp, i64, vp, i64, vp], ctypes.c_int),
    "tsqr_factor_form_host": ([vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp], ctypes.c_int),
    "tsqr_sync_status": ([vp, vp], ctypes.c_int),
    "tsqr_q_info": ([vp, pi64, pi64, pi32, pi64, pi64, pi32, pi32], ctypes.c_int),
    "tsqr_q_part": ([vp, i32, i32, i64, vp, vp], ctypes.c_int),
    "tsqr_q_chains": ([vp, pi64, pi64], ctypes.c_int),
    "tsqr_lstsq": ([vp, vp, i64, i64, vp, i64, vp, i64, vp, vp], ctypes.c_int),
    "tsqr_solve_r": ([i64, i64, i32, vp, i64, vp, i64, vp, vp], ctypes.c_int),
    "tsqr_column_norms": ([i64, i64, i32, vp, i64, vp, vp], ctypes.c_int),
    "tsqr_q_destroy": ([vp], ctypes.c_int),
    "tsqr_test_reflectors": ([i64, vp, vp, i32, vp, vp], ctypes.c_int),
    "tsqr_factor_r_noalloc": ([i64, i64, vp, i64, vp, i64, vp], ctypes.c_int),
    "caqr_factor": ([i64, i64, vp, i64, i64, i32, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "caqr_factor_f32": ([i64, i64, vp, i64, i64, i32, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "caqr_q_create": ([i64, i64, i64, i32, ctypes.POINTER(TsqrOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "caqr_refactor": ([vp, vp, i64, vp], ctypes.c_int),
    "caqr_apply_qt": ([vp, i64, vp, i64, vp], ctypes.c_int),
    "caqr_apply_q": ([vp, i64, vp, i64, vp], ctypes.c_int),
    "caqr_form_q": ([vp, vp, i64, vp], ctypes.c_int),
    "caqr_sync_status": ([vp, vp], ctypes.c_int),
    "caqr_q_destroy": ([vp], ctypes.c_int),
    "caqr_q_set_timing": ([vp, i32], ctypes.c_int),
    "caqr_q_stage_times": ([vp, ctypes.POINTER(ctypes.c_double), pi64, i32], ctypes.c_int),
    "tsqr_qr_backward": ([i64, i64, i32, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp], ctypes.c_int),
    "tsqr_batch_create": ([i32, pi64, pi64, ctypes.POINTER(vp), pi64, ctypes.POINTER(vp), pi64, i32,
                           ctypes.POINTER(TsqrBatchOpts), ctypes.POINTER(vp), vp], ctypes.c_int),
    "tsqr_batch_factor": ([vp, vp], ctypes.c_int),
    "tsqr_batch_factor_graph": ([vp, vp], ctypes.c_int),
    "tsqr_batch_info": ([vp, pi32, pi32, pi64, pi64], ctypes.c_int),
    "tsqr_batch_sync_status": ([vp, vp], ctypes.c_int),
    "tsqr_batch_destroy": ([vp], ctypes.c_int),
    "tsqr_q_set_timing": ([vp, i32], ctypes.c_int),
    "tsqr_q_stage_times": ([vp, ctypes.POINTER(ctypes.c_double), pi64, i32], ctypes.c_int),
    "tsqr_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "tsqr_version": ([], ctypes.c_int),
}


class TsqrError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().tsqr_status_string(code).decode() if _lib is not None else str(code)
        if code < 0:
            msg = f"argument {-code} is invalid"
        super().__init__(f"{where}: {msg} (code {code})")


def lib():
    """The loaded library; raises if libtsqr_gb300.so has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_0808_2664_gb300.build` "
                    "(or __graft_entry__.build()); the package has no CPU fallback")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(handle, name)
                f.argtypes = args
                f.restype = res
            _lib = handle
    return _lib


def check(rc: int, where: str) -> None:
    if rc != 0:
        raise TsqrError(rc, where)
