"""Strategy-preserving map/reduce hot path for GB300 (sm_103a).

The C-ABI library ``libdpia.so`` (include/dpia.h) computes dot, asum, scal,
GEMV (forward and backward) and GEMM instances of the paper's
strategy-annotated map/reduce skeleton with hand-written CUDA kernels; this
package is its Python binding. PyTorch supplies device memory and streams.
"""
from . import _native
from ._native import DPIAError
from .ops import (asum, dot, dot_bwd, dpia_asum_f32, dpia_cast_f32_bf16, dpia_dot_bwd_f32, dpia_dot_f32,
                  dpia_dot_f32_noalloc, dpia_dot_i32, dpia_dot_workspace_size, dpia_gemm_bf16,
                  dpia_gemm_f32, dpia_gemv_bwd_f32, dpia_gemv_bwd_workspace_size, dpia_gemv_f32,
                  dpia_last_error_message, dpia_poll_device_status, dpia_scal_f32,
                  dpia_selftest_bounded_wait, dpia_version, gemm,
                  gemv, gemv_bwd, scal, to_bf16, workspace)
from .strategy import ReduceStrategy, default_dot_strategy

__all__ = [n for n in dir() if not n.startswith("_")]
