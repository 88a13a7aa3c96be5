"""ctypes binding of ``libdpia.so`` (declarations of include/dpia.h).

Loading fails loudly: if the shared object is missing or stale it is built with
nvcc; if that is impossible an ImportError is raised. There is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

# status codes (dpia_status)
OK, ERR_NULL, ERR_SHAPE, ERR_ALIGN, ERR_STRATEGY, ERR_WORKSPACE, ERR_ALIAS, ERR_CUDA, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(10)
STATUS_NAMES = {OK: "OK", ERR_NULL: "NULL", ERR_SHAPE: "SHAPE", ERR_ALIGN: "ALIGN",
                ERR_STRATEGY: "STRATEGY", ERR_WORKSPACE: "WORKSPACE", ERR_ALIAS: "ALIAS",
                ERR_CUDA: "CUDA", ERR_TIMEOUT: "TIMEOUT", ERR_UNSUPPORTED: "UNSUPPORTED"}

# levels (dpia_level)
LVL_GRID, LVL_BLOCK, LVL_WARP, LVL_THREAD, LVL_SEQ = range(5)
MAP_INTERLEAVED, MAP_CONTIG = 0, 1
SECOND_SEQ, SECOND_TREE = 0, 1
STAGE_PRIVATE, STAGE_LOCAL = 0, 1


class DPIAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{STATUS_NAMES.get(status, status)}] {message}")
        self.status = status


class GemmStrategyC(ctypes.Structure):
    _fields_ = [("contract", ctypes.c_int32), ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("tile_k", ctypes.c_int32), ("grid", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]


class ReduceStrategyC(ctypes.Structure):
    _fields_ = [
        ("split", ctypes.c_int64),
        ("threads", ctypes.c_int32),
        ("vec", ctypes.c_int32),
        ("map_level", ctypes.c_int32),
        ("inner_level", ctypes.c_int32),
        ("thread_map", ctypes.c_int32),
        ("second", ctypes.c_int32),
        ("threads2", ctypes.c_int32),
        ("compensated", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("stage", ctypes.c_int32),
    ]


class DotInstanceC(ctypes.Structure):
    _fields_ = [("off", ctypes.c_int64), ("n", ctypes.c_int64), ("st", ReduceStrategyC)]


class GemvInstanceC(ctypes.Structure):
    _fields_ = [("a_off", ctypes.c_int64), ("x_off", ctypes.c_int64), ("y_off", ctypes.c_int64),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("lda", ctypes.c_int64), ("st", ReduceStrategyC),
                ("row_split", ctypes.c_int64)]


class BatchOptionsC(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("schedule", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t
_SP = ctypes.POINTER(ReduceStrategyC)
_GP = ctypes.POINTER(GemmStrategyC)

# name -> (restype, argtypes); kept in the order of include/dpia.h
SIGNATURES = {
    "dpia_version": (_I32, []),
    "dpia_last_error_message": (ctypes.c_char_p, []),
    "dpia_dot_workspace_size": (_SZ, [_I64, _SP]),
    "dpia_dot_f32": (_I32, [_P, _P, _I64, _SP, _P, _P, _SZ, _P]),
    "dpia_dot_i32": (_I32, [_P, _P, _I64, _SP, _P, _P, _SZ, _P]),
    "dpia_asum_f32": (_I32, [_P, _I64, _SP, _P, _P, _SZ, _P]),
    "dpia_scal_f32": (_I32, [ctypes.c_float, _P, _P, _I64, _I32, _P]),
    "dpia_dot_bwd_f32": (_I32, [_P, _P, _P, _I64, _P, _P, _P]),
    "dpia_gemv_f32": (_I32, [_P, _I64, _I64, _I64, _P, _P, _SP, _P]),
    "dpia_gemv_bwd_workspace_size": (_SZ, [_I64, _I64, _I64]),
    "dpia_gemv_bwd_f32": (_I32, [_P, _I64, _I64, _I64, _P, _P, _P, _P, _I64, _I64, _P, _SZ, _P]),
    "dpia_gemm_f32": (_I32, [_P, _P, _P, _I64, _I64, _I64, _I64, _I64, _I64, _I32, _I32, _GP, _P]),
    "dpia_gemm_bf16": (_I32, [_P, _P, _P, _I64, _I64, _I64, _I64, _I64, _I64, _I32, _I32, _GP, _P]),
    "dpia_cast_f32_bf16": (_I32, [_P, _P, _I64, _P]),
    "dpia_poll_device_status": (_I32, [ctypes.POINTER(ctypes.c_int32)]),
    "dpia_selftest_bounded_wait": (_I32, [ctypes.c_uint32, ctypes.c_void_p]),
    "dpia_batch_plan_size": (_SZ, [_I32, ctypes.POINTER(DotInstanceC), _I32, ctypes.POINTER(GemvInstanceC),
                                   ctypes.POINTER(BatchOptionsC)]),
    "dpia_batch_plan": (_I32, [_I32, ctypes.POINTER(DotInstanceC), _I32, ctypes.POINTER(GemvInstanceC),
                               ctypes.POINTER(BatchOptionsC), _P, _SZ]),
    "dpia_batch_workspace_size": (_SZ, [_P]),
    "dpia_batch_forward_f32": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _I32, _P]),
    "dpia_batch_backward_f32": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _I32, _P]),
    "dpia_dot_f32_noalloc": (_I32, [_P, _P, _I64, _SP, _P, _P]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded library (built on first use if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            try:
                path = _build.build()
            except Exception as e:  # no silent fallback: the CUDA library is the product
                raise ImportError(f"cannot build libdpia.so: {e}") from e
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, fn: str = ""):
    if status != OK:
        msg = lib().dpia_last_error_message().decode(errors="replace")
        raise DPIAError(status, msg or fn)


def exported_symbols():
    return list(SIGNATURES)


def loaded_path() -> str | None:
    return _lib._name if _lib is not None else None


def ensure_built() -> str:
    lib()
    return os.path.abspath(_build.LIB)
