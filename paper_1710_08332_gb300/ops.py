"""Python binding of the C ABI: one function per entry point, same names.

The ``dpia_*`` functions only marshal torch tensors (device pointers, sizes,
the current CUDA stream) into the C call and raise ``DPIAError`` on a non-OK
status; every step of the computation runs in the library's kernels. The
short names (``dot``, ``asum``, ...) additionally allocate outputs and
workspaces with torch.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _native as N
from .strategy import ReduceStrategy, default_dot_strategy


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("dpia: tensors must be CUDA tensors (device memory)")


def _st(st: ReduceStrategy):
    return ctypes.byref(st.to_c())


# ---------------------------------------------------------------------------
# entry points (same names as include/dpia.h)
# ---------------------------------------------------------------------------


def dpia_version() -> int:
    return N.lib().dpia_version()


def dpia_last_error_message() -> str:
    return N.lib().dpia_last_error_message().decode(errors="replace")


def dpia_dot_workspace_size(n: int, st: ReduceStrategy) -> int:
    return int(N.lib().dpia_dot_workspace_size(int(n), _st(st)))


def dpia_dot_f32(x, y, n, st, out, ws, stream=None):
    _need_cuda(x, y, out, ws)
    N.check(N.lib().dpia_dot_f32(_ptr(x), _ptr(y), int(n), _st(st), _ptr(out), _ptr(ws),
                                 ws.numel() * ws.element_size() if ws is not None else 0,
                                 _stream(stream)), "dpia_dot_f32")


def dpia_dot_i32(x, y, n, st, out, ws, stream=None):
    _need_cuda(x, y, out, ws)
    N.check(N.lib().dpia_dot_i32(_ptr(x), _ptr(y), int(n), _st(st), _ptr(out), _ptr(ws),
                                 ws.numel() * ws.element_size() if ws is not None else 0,
                                 _stream(stream)), "dpia_dot_i32")


def dpia_asum_f32(x, n, st, out, ws, stream=None):
    _need_cuda(x, out, ws)
    N.check(N.lib().dpia_asum_f32(_ptr(x), int(n), _st(st), _ptr(out), _ptr(ws),
                                  ws.numel() * ws.element_size() if ws is not None else 0,
                                  _stream(stream)), "dpia_asum_f32")


def dpia_scal_f32(a, x, y, n, vec=4, stream=None):
    _need_cuda(x, y)
    N.check(N.lib().dpia_scal_f32(ctypes.c_float(a), _ptr(x), _ptr(y), int(n), int(vec),
                                  _stream(stream)), "dpia_scal_f32")


def dpia_dot_bwd_f32(x, y, g, n, dx, dy, stream=None):
    _need_cuda(x, y, g, dx, dy)
    N.check(N.lib().dpia_dot_bwd_f32(_ptr(x), _ptr(y), _ptr(g), int(n), _ptr(dx), _ptr(dy),
                                     _stream(stream)), "dpia_dot_bwd_f32")


def dpia_gemv_f32(A, M, N_, lda, x, y, st, stream=None):
    _need_cuda(A, x, y)
    N.check(N.lib().dpia_gemv_f32(_ptr(A), int(M), int(N_), int(lda), _ptr(x), _ptr(y), _st(st),
                                  _stream(stream)), "dpia_gemv_f32")


def dpia_gemv_bwd_workspace_size(M, N_, row_split) -> int:
    return int(N.lib().dpia_gemv_bwd_workspace_size(int(M), int(N_), int(row_split)))


def dpia_gemv_bwd_f32(A, M, N_, lda, x, dy, dx, dA, ldda, row_split, ws, stream=None):
    _need_cuda(A, x, dy, dx, dA, ws)
    N.check(N.lib().dpia_gemv_bwd_f32(_ptr(A), int(M), int(N_), int(lda), _ptr(x), _ptr(dy),
                                      _ptr(dx), _ptr(dA), int(ldda), int(row_split), _ptr(ws),
                                      ws.numel() * ws.element_size() if ws is not None else 0,
                                      _stream(stream)), "dpia_gemv_bwd_f32")


def _gst(contract="fma", grid=0, tile_n=0, cluster=0, tile_m=0, schedule=0):
    return ctypes.byref(N.GemmStrategyC(1 if contract == "fma" else 0, int(tile_m), int(tile_n), 0, int(grid),
                                        int(cluster), int(schedule)))


def dpia_gemm_f32(A, B, C, M, N_, K, lda, ldb, ldc, transA=0, transB=0, contract="fma", schedule=0, stream=None):
    """schedule: 0 automatic, 1 one launch of 128 x 128 tiles, 2 half-height tiles
    for a last wave at most half full, 3 k-range pieces over two launches."""
    _need_cuda(A, B, C)
    N.check(N.lib().dpia_gemm_f32(_ptr(A), _ptr(B), _ptr(C), int(M), int(N_), int(K), int(lda), int(ldb),
                                  int(ldc), int(transA), int(transB), _gst(contract, schedule=schedule),
                                  _stream(stream)), "dpia_gemm_f32")


def dpia_gemm_bf16(A, B, C, M, N_, K, lda, ldb, ldc, transA=0, transB=0, grid=0, tile_n=0, cluster=0,
                   tile_m=0, stream=None):
    """A, B: torch.bfloat16 (or int16/uint16 bit patterns) device tensors; C float32."""
    _need_cuda(A, B, C)
    N.check(N.lib().dpia_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), int(M), int(N_), int(K), int(lda), int(ldb),
                                   int(ldc), int(transA), int(transB), _gst("fma", grid, tile_n, cluster, tile_m),
                                   _stream(stream)), "dpia_gemm_bf16")


def dpia_cast_f32_bf16(x, y, n, stream=None):
    _need_cuda(x, y)
    N.check(N.lib().dpia_cast_f32_bf16(_ptr(x), _ptr(y), int(n), _stream(stream)), "dpia_cast_f32_bf16")


def dpia_poll_device_status() -> int:
    v = ctypes.c_int32(-1)
    N.check(N.lib().dpia_poll_device_status(ctypes.byref(v)), "dpia_poll_device_status")
    return int(v.value)


def dpia_selftest_bounded_wait(timeout_us: int, stream=None) -> None:
    N.check(N.lib().dpia_selftest_bounded_wait(int(timeout_us), _stream(stream)), "dpia_selftest_bounded_wait")


def dpia_dot_f32_noalloc(x, y, n, st, out, stream=None):
    """dpia_dot_f32 without a workspace argument, for callers that cannot
    allocate device memory: the scratch is the library's static 1 MiB device
    array (calls that overlap on the GPU race on it)."""
    _need_cuda(x, y, out)
    N.check(N.lib().dpia_dot_f32_noalloc(_ptr(x), _ptr(y), int(n), _st(st), _ptr(out), _stream(stream)),
            "dpia_dot_f32_noalloc")


# ---------------------------------------------------------------------------
# workspaces: zero-filled once, reused (each call leaves its counters zero)
# ---------------------------------------------------------------------------

_ws_lock = threading.Lock()
_ws_cache: dict = {}


def workspace(nbytes: int, device=None, stream=None, kind="reduce") -> torch.Tensor:
    """A zero-initialised workspace of >= nbytes for calls on ``stream``.

    One buffer per (device, stream, kind) is kept and grown on demand; calls on
    one stream are ordered, so they can share it. Workspaces may only be shared
    by calls with the same counter layout: every dot / asum / int32-dot call
    keeps its counter in the first 128 bytes (kind "reduce", any shape), while a
    GEMV backward's counters depend on its shape, so its kind is the shape.
    """
    device = torch.device(device) if device is not None else torch.device("cuda")
    if device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    stream = stream or torch.cuda.current_stream(device)
    key = (device.index, stream.cuda_stream, kind)
    nbytes = max(int(nbytes), 128)
    with _ws_lock:
        buf = _ws_cache.get(key)
        if buf is None or buf.numel() < nbytes:
            size = 1 << (nbytes - 1).bit_length()
            with torch.cuda.stream(stream):
                buf = torch.zeros(size, dtype=torch.uint8, device=device)
            _ws_cache[key] = buf
    return buf


# ---------------------------------------------------------------------------
# convenience API
# ---------------------------------------------------------------------------


def dot(x, y, strategy: ReduceStrategy | None = None, out=None):
    """dot(x, y) under a reduction strategy (float32 or int32 inputs)."""
    n = x.numel()
    st = strategy or default_dot_strategy(n)
    if x.dtype == torch.int32:
        out = out if out is not None else torch.empty(1, dtype=torch.int64, device=x.device)
        ws = workspace(dpia_dot_workspace_size(n, st), x.device)
        dpia_dot_i32(x, y, n, st, out, ws)
        return out[0]
    out = out if out is not None else torch.empty(1, dtype=torch.float32, device=x.device)
    ws = workspace(dpia_dot_workspace_size(n, st), x.device)
    dpia_dot_f32(x, y, n, st, out, ws)
    return out[0]


def asum(x, strategy: ReduceStrategy | None = None, out=None):
    n = x.numel()
    st = strategy or default_dot_strategy(n)
    out = out if out is not None else torch.empty(1, dtype=torch.float32, device=x.device)
    ws = workspace(dpia_dot_workspace_size(n, st), x.device)
    dpia_asum_f32(x, n, st, out, ws)
    return out[0]


def scal(a: float, x, out=None, vec: int = 4):
    y = out if out is not None else torch.empty_like(x)
    dpia_scal_f32(a, x, y, x.numel(), vec)
    return y


def default_gemv_strategy(N_: int, lda: int | None = None, aligned16: bool = True) -> ReduceStrategy:
    """One chunk per row: a block per row for long rows, a warp per row for
    short ones; the vector width is the widest the row alignment allows."""
    lda = N_ if lda is None else lda
    V = 4 if (aligned16 and lda % 4 == 0) else 2 if lda % 2 == 0 else 1
    if N_ >= 1024:
        q = 128 * V
        s = ((N_ + q - 1) // q) * q
        return ReduceStrategy(split=s, threads=128, vec=V, pad=N_ % q != 0)
    q = 32 * V
    s = ((max(N_, 1) + q - 1) // q) * q
    return ReduceStrategy(split=s, threads=128, vec=V, map_level="warp", pad=N_ % q != 0)


def gemv(A, x, strategy: ReduceStrategy | None = None, out=None):
    M, N_ = A.shape
    st = strategy or default_gemv_strategy(N_, A.stride(0), A.data_ptr() % 16 == 0 and x.data_ptr() % 16 == 0)
    y = out if out is not None else torch.empty(M, dtype=torch.float32, device=A.device)
    dpia_gemv_f32(A, M, N_, A.stride(0), x, y, st)
    return y


def gemv_bwd(A, x, dy, need_dx=True, need_dA=True, row_split=256):
    M, N_ = A.shape
    dx = torch.empty(N_, dtype=torch.float32, device=A.device) if need_dx else None
    dA = torch.empty(M, N_, dtype=torch.float32, device=A.device) if need_dA else None
    ws = workspace(dpia_gemv_bwd_workspace_size(M, N_, row_split), A.device,
                   kind=("gemv_bwd", M, N_, row_split)) if need_dx else None
    dpia_gemv_bwd_f32(A, M, N_, A.stride(0), x, dy, dx, dA, N_, row_split, ws)
    return dx, dA


def dot_bwd(x, y, g):
    dx, dy = torch.empty_like(x), torch.empty_like(y)
    dpia_dot_bwd_f32(x, y, g, x.numel(), dx, dy)
    return dx, dy


def _op_shape(t, trans):
    r, c = t.shape
    return (c, r) if trans else (r, c)


def gemm(A, B, transA=False, transB=False, precision="f32", contract="fma", out=None):
    """C = op(A) op(B). precision "f32": the FP32 fold on CUDA cores (bit-exact
    against a sequential k loop); "bf16": A and B (float32 or bfloat16) are
    rounded to bf16 and multiplied on the tensor cores with f32 accumulation."""
    M, K = _op_shape(A, transA)
    K2, N_ = _op_shape(B, transB)
    if K != K2:
        raise ValueError(f"inner dimensions differ: {K} vs {K2}")
    C = out if out is not None else torch.empty(M, N_, dtype=torch.float32, device=A.device)
    if precision == "f32":
        dpia_gemm_f32(A, B, C, M, N_, K, A.stride(0), B.stride(0), C.stride(0), int(transA), int(transB), contract)
    elif precision == "bf16":
        Ab, Bb = to_bf16(A), to_bf16(B)
        dpia_gemm_bf16(Ab, Bb, C, M, N_, K, Ab.stride(0), Bb.stride(0), C.stride(0), int(transA), int(transB))
    else:
        raise ValueError(precision)
    return C


def to_bf16(x):
    """x as bfloat16 (round to nearest even by the library's cast kernel)."""
    if x.dtype == torch.bfloat16:
        return x
    y = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    dpia_cast_f32_bf16(x.contiguous(), y, x.numel())
    return y
