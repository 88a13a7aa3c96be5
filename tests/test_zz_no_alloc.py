"""The allocation-free dot entry point, called through the C ABI.

dpia_dot_f32_noalloc serves callers that cannot allocate device memory (for
instance a plugin whose host framework owns every device allocation): it uses
the library's static scratch array instead of a caller workspace. Its result
must equal dpia_dot_f32's with the same strategy -- bit for bit, the tolerance
the parity tests use for same-strategy FP32 -- on two calls in a row (the
second call reuses the scratch left by the first), and the oracle's evaluation
of the same strategy tree. This file is collected last
so that a failure here cannot hide earlier tests in a run that stops at the
first failure; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import loopnest
from paper_1710_08332_gb300 import _native as N
from paper_1710_08332_gb300.strategy import ReduceStrategy
from synth import workloads as W
from tests.helpers import host, oracle_strategy

pytestmark = pytest.mark.gpu


def _c_dot(x, y, st, with_workspace: bool):
    L = N.lib()
    n = x.numel()
    out = torch.full((1,), float("nan"), device=x.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if with_workspace:
        nbytes = L.dpia_dot_workspace_size(n, ctypes.byref(st.to_c()))
        ws = torch.zeros(nbytes, dtype=torch.uint8, device=x.device)
        rc = L.dpia_dot_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), n,
                            ctypes.byref(st.to_c()), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(ws.data_ptr()), nbytes, stream)
    else:
        rc = L.dpia_dot_f32_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), n,
                                    ctypes.byref(st.to_c()), ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == N.OK, L.dpia_last_error_message().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_workspace_entry_twice(cuda_device):
    st = ReduceStrategy(split=8192, threads=256, vec=4, second="tree", threads2=256, pad=True)
    for seed, n in ((0, W.DOT_N), (7, (1 << 22) + 123)):  # two calls in a row, different inputs
        x, y = W.dot_f32("cuda", n=n, seed=seed)
        want = _c_dot(x, y, st, with_workspace=True)
        got = _c_dot(x, y, st, with_workspace=False)
        assert got.tobytes() == want.tobytes(), (got, want)
        oracle = loopnest.dot_f32(host(x), host(y), oracle_strategy(st))
        assert got[0].tobytes() == oracle.tobytes(), (got, oracle)
    # the sequential second level over 128 partials (the 2^20 dot's split) as well
    st2 = ReduceStrategy(split=W.DOT_SPLIT, threads=256, vec=4)
    x, y = W.dot_f32("cuda")
    a = _c_dot(x, y, st2, with_workspace=False)
    b = _c_dot(x, y, st2, with_workspace=False)
    assert a.tobytes() == b.tobytes() == _c_dot(x, y, st2, with_workspace=True).tobytes()
    assert a[0].tobytes() == loopnest.dot_f32(host(x), host(y), oracle_strategy(st2)).tobytes()


def test_noalloc_rejects_more_chunks_than_scratch(cuda_device):
    L = N.lib()
    n = 1 << 26
    st = ReduceStrategy(split=256, threads=64, vec=4)  # 262144 chunks: 2 MiB of partials
    x = torch.zeros(n, device="cuda")
    out = torch.zeros(1, device="cuda")
    rc = L.dpia_dot_f32_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), n,
                                ctypes.byref(st.to_c()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == N.ERR_WORKSPACE
    assert "static scratch" in L.dpia_last_error_message().decode()
