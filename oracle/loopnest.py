"""c2 loader: builds and binds ``loopnest.c`` -- TEST INFRASTRUCTURE ONLY.

The shared object is built with the system C compiler at ``-O2
-ffp-contract=off`` (no ``-ffast-math``, no ``-march``), so each float + and *
is rounded separately on both x86-64 and AArch64 hosts, and with ``-fopenmp``:
the independent units of a strategy (chunks, rows, columns, GEMM entries, map
elements) may run on several host threads, while every fold across units runs
on one thread in the strategy's order, so results do not depend on the thread
count. ``set_threads`` chooses it; the loader starts with every core this
process may run on (``os.sched_getaffinity``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "loopnest.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_loopnest.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-fopenmp"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``loopnest.c`` (if stale) and return the shared-object path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "gcc")
    subprocess.run([cc, *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
            _lib.oracle_set_threads(len(os.sched_getaffinity(0)))
    return _lib


def set_threads(n: int) -> int:
    """Use ``n`` host threads for the per-unit loops; returns the previous count."""
    L = lib()
    old = L.oracle_threads()
    if L.oracle_set_threads(int(n)) != 0:
        raise ValueError(f"set_threads: bad thread count {n}")
    return old


def threads() -> int:
    return lib().oracle_threads()


_f = ctypes.POINTER(ctypes.c_float)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_I = ctypes.c_int
_L = ctypes.c_int64


def _declare(L):
    L.oracle_dot_f32.argtypes = [_f, _f, _L, _L, _I, _I, _I, _I, _I, _I, _I, _f]
    L.oracle_asum_f32.argtypes = [_f, _L, _L, _I, _I, _I, _I, _I, _I, _I, _f]
    L.oracle_dot_f32_partials.argtypes = [_f, _f, _L, _L, _I, _I, _I, _I, _f]
    L.oracle_dot_i32.argtypes = [_i32, _i32, _L, _L, _I, _I, _I, _I, _I, _I, _i64p]
    L.oracle_scal_f32.argtypes = [ctypes.c_float, _f, _f, _L]
    L.oracle_scal_f32.restype = None
    L.oracle_dot_bwd_f32.argtypes = [_f, _f, ctypes.c_float, _L, _f, _f]
    L.oracle_dot_bwd_f32.restype = None
    L.oracle_gemv_f32.argtypes = [_f, _L, _L, _L, _f, _f, _L, _I, _I, _I, _I, _I]
    L.oracle_gemv_bwd_dx_f32.argtypes = [_f, _L, _L, _L, _f, _L, _f]
    L.oracle_gemv_bwd_dA_f32.argtypes = [_f, _f, _L, _L, _f, _L]
    L.oracle_gemv_bwd_dA_f32.restype = None
    L.oracle_gemm_f32_sample.argtypes = [_f, _f, _L, _L, _L, _L, _L, _I, _I, _I,
                                         _i64p, _L, _i64p, _L, _f]
    L.oracle_lane_partials_f32.argtypes = [_I, _f, _f, _L, _L, _I, _I, _I, _I, _f]
    L.oracle_lane_partials_f32.restype = ctypes.c_int
    L.oracle_set_threads.argtypes = [_I]
    L.oracle_set_threads.restype = ctypes.c_int
    L.oracle_threads.argtypes = []
    L.oracle_threads.restype = ctypes.c_int
    L.oracle_max_threads.argtypes = []
    L.oracle_max_threads.restype = ctypes.c_int
    for name in ("oracle_dot_f32", "oracle_asum_f32", "oracle_dot_f32_partials",
                 "oracle_dot_i32", "oracle_gemv_f32", "oracle_gemv_bwd_dx_f32",
                 "oracle_gemm_f32_sample"):
        getattr(L, name).restype = ctypes.c_int


def _fp(a):
    return a.ctypes.data_as(_f) if a is not None else None


def _c32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what}: oracle rejected the arguments (code {rc})")


def _st_args(st):
    return (int(st.s), int(st.T), int(st.V), 1 if st.thread_map == "interleaved" else 0,
            1 if st.second == "tree" else 0, int(st.T2), 1 if st.compensated else 0,
            1 if st.pad else 0)


def dot_f32(x, y, st) -> np.float32:
    """Strategy dot product (same tree as ``patterns.dot_R``)."""
    x, y = _c32(x), _c32(y)
    out = np.zeros(1, np.float32)
    _check(lib().oracle_dot_f32(_fp(x), _fp(y), x.size, *_st_args(st), _fp(out)), "dot_f32")
    return out[0]


def asum_f32(x, st) -> np.float32:
    x = _c32(x)
    out = np.zeros(1, np.float32)
    _check(lib().oracle_asum_f32(_fp(x), x.size, *_st_args(st), _fp(out)), "asum_f32")
    return out[0]


def dot_f32_partials(x, y, st) -> np.ndarray:
    x, y = _c32(x), _c32(y)
    C = -(-x.size // st.s)
    out = np.zeros(C, np.float32)
    s, T, V, inter, _, _, _, pad = _st_args(st)
    _check(lib().oracle_dot_f32_partials(_fp(x), _fp(y), x.size, s, T, V, inter, pad, _fp(out)),
           "dot_f32_partials")
    return out


def lane_partials_f32(kind, x, y, st) -> np.ndarray:
    """The un-reduced first level of Section 6's kernel: for chunk c, thread t
    and lane v (at index (c*T + t)*V + v) the fold of that lane's items from +0
    (kind "dot": x*y; "asum": |x|). st.pad pads a ragged last chunk."""
    x = _c32(x)
    y = _c32(y) if y is not None else None
    C = -(-x.size // st.s)
    out = np.zeros(C * st.T * st.V, np.float32)
    s, T, V, inter, _, _, _, pad = _st_args(st)
    _check(lib().oracle_lane_partials_f32({"dot": 0, "asum": 1}[kind], _fp(x), _fp(y), x.size, s, T, V, inter,
                                          pad, _fp(out)), "lane_partials_f32")
    return out


def dot_i32(x, y, st) -> int:
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    out = np.zeros(1, np.int64)
    s, T, V, inter, tree, T2, _, pad = _st_args(st)
    _check(lib().oracle_dot_i32(x.ctypes.data_as(_i32), y.ctypes.data_as(_i32), x.size, s, T, V,
                                inter, tree, T2, pad, out.ctypes.data_as(_i64p)), "dot_i32")
    return int(out[0])


def scal_f32(a, x) -> np.ndarray:
    x = _c32(x)
    y = np.empty_like(x)
    lib().oracle_scal_f32(ctypes.c_float(a), _fp(x), _fp(y), x.size)
    return y


def dot_bwd_f32(x, y, g):
    x, y = _c32(x), _c32(y)
    dx, dy = np.empty_like(x), np.empty_like(y)
    lib().oracle_dot_bwd_f32(_fp(x), _fp(y), ctypes.c_float(g), x.size, _fp(dx), _fp(dy))
    return dx, dy


def gemv_f32(A, x, st) -> np.ndarray:
    """Rows of A (M x N, row-major) each reduced with ``st`` (second level seq;
    with st.pad a ragged row's last chunk takes identity items)."""
    A, x = _c32(A), _c32(x)
    M, N = A.shape
    y = np.zeros(M, np.float32)
    _check(lib().oracle_gemv_f32(_fp(A), M, N, N, _fp(x), _fp(y), int(st.s), int(st.T),
                                 int(st.V), 1 if st.thread_map == "interleaved" else 0,
                                 1 if st.compensated else 0, 1 if st.pad else 0), "gemv_f32")
    return y


def gemv_bwd_dx_f32(A, dy, row_split) -> np.ndarray:
    A, dy = _c32(A), _c32(dy)
    M, N = A.shape
    dx = np.zeros(N, np.float32)
    _check(lib().oracle_gemv_bwd_dx_f32(_fp(A), M, N, N, _fp(dy), int(row_split), _fp(dx)),
           "gemv_bwd_dx_f32")
    return dx


def gemv_bwd_dA_f32(x, dy) -> np.ndarray:
    x, dy = _c32(x), _c32(dy)
    dA = np.empty((dy.size, x.size), np.float32)
    lib().oracle_gemv_bwd_dA_f32(_fp(x), _fp(dy), dy.size, x.size, _fp(dA), x.size)
    return dA


def gemm_f32_sample(A, B, transA, transB, contract_fma, rows, cols) -> np.ndarray:
    """Entries C[rows][:, cols] of the FP32 fold GEMM (A, B stored row-major)."""
    A, B = _c32(A), _c32(B)
    if transA:
        K, M = A.shape
    else:
        M, K = A.shape
    N = B.shape[0] if transB else B.shape[1]
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    out = np.zeros((rows.size, cols.size), np.float32)
    _check(lib().oracle_gemm_f32_sample(_fp(A), _fp(B), M, N, K, A.shape[1], B.shape[1],
                                        int(bool(transA)), int(bool(transB)),
                                        int(bool(contract_fma)), rows.ctypes.data_as(_i64p),
                                        rows.size, cols.ctypes.data_as(_i64p), cols.size,
                                        _fp(out)), "gemm_f32_sample")
    return out


def gemm_f32(A, B, transA=False, transB=False, contract_fma=True) -> np.ndarray:
    M = A.shape[1] if transA else A.shape[0]
    N = B.shape[0] if transB else B.shape[1]
    return gemm_f32_sample(A, B, transA, transB, contract_fma, np.arange(M), np.arange(N))
