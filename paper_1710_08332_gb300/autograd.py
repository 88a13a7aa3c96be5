"""torch.autograd.Functions over the C ABI (forward and backward both run in
the library's kernels; this module only routes tensors).

Adjoints of the functional forms: the adjoint of reduce(+) is a broadcast of
the incoming gradient and the adjoint of the pointwise product map multiplies
by the other operand, so for d = dot(x, y): dx = g*y, dy = g*x; for y = A x
(a map of dot products over rows): dA = dy x^T and dx = A^T dy; for C = A B:
dA = dC B^T and dB = A^T dC (split, join and transpose are re-indexings and
become the operand layouts of the backward products).
"""
from __future__ import annotations

import torch

from . import ops
from .strategy import ReduceStrategy, default_dot_strategy


class DotFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, strategy: ReduceStrategy | None = None):
        x = x.contiguous()
        y = y.contiguous()
        ctx.save_for_backward(x, y)
        st = strategy or default_dot_strategy(x.numel())
        out = torch.empty(1, dtype=torch.float32, device=x.device)
        ws = ops.workspace(ops.dpia_dot_workspace_size(x.numel(), st), x.device)
        ops.dpia_dot_f32(x, y, x.numel(), st, out, ws)
        return out.reshape(())

    @staticmethod
    def backward(ctx, g):
        x, y = ctx.saved_tensors
        g = g.reshape(1).to(torch.float32).contiguous()
        dx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dy = torch.empty_like(y) if ctx.needs_input_grad[1] else None
        ops.dpia_dot_bwd_f32(x, y, g, x.numel(), dx, dy)
        return dx, dy, None


class GemvFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, x, strategy: ReduceStrategy | None = None, row_split: int = 256):
        A = A.contiguous()
        x = x.contiguous()
        ctx.save_for_backward(A, x)
        ctx.row_split = row_split
        return ops.gemv(A, x, strategy)

    @staticmethod
    def backward(ctx, dy):
        A, x = ctx.saved_tensors
        dy = dy.contiguous()
        M, N = A.shape
        need_dA, need_dx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dx = torch.empty(N, dtype=torch.float32, device=A.device) if need_dx else None
        dA = torch.empty(M, N, dtype=torch.float32, device=A.device) if need_dA else None
        ws = ops.workspace(ops.dpia_gemv_bwd_workspace_size(M, N, ctx.row_split), A.device,
                           kind=("gemv_bwd", M, N, ctx.row_split)) if need_dx else None
        ops.dpia_gemv_bwd_f32(A, M, N, N, x, dy, dx, dA, N, ctx.row_split, ws)
        return dA, dx, None, None


class GemmFn(torch.autograd.Function):
    """C = A B with A (M x K), B (K x N); precision "f32" (CUDA-core fold) or
    "bf16" (tensor cores, f32 accumulation). The backward products reuse the
    forward kernels with transposed operand layouts."""

    @staticmethod
    def forward(ctx, A, B, precision: str = "f32", contract: str = "fma"):
        A = A.contiguous()
        B = B.contiguous()
        ctx.save_for_backward(A, B)
        ctx.precision = precision
        ctx.contract = contract
        return ops.gemm(A, B, precision=precision, contract=contract)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous().to(torch.float32)
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = ops.gemm(dC, B, transB=True, precision=ctx.precision, contract=ctx.contract)   # dC B^T
        if ctx.needs_input_grad[1]:
            dB = ops.gemm(A, dC, transA=True, precision=ctx.precision, contract=ctx.contract)   # A^T dC
        return dA, dB, None, None


def dot(x, y, strategy: ReduceStrategy | None = None):
    return DotFn.apply(x, y, strategy)


def gemv(A, x, strategy: ReduceStrategy | None = None, row_split: int = 256):
    return GemvFn.apply(A, x, strategy, row_split)


def gemm(A, B, precision: str = "f32", contract: str = "fma"):
    return GemmFn.apply(A, B, precision, contract)
