"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/dpia.h declares, and rejects bad arguments on the host before
any CUDA call (null pointers, shapes, alignment, illegal level nestings,
small workspaces, aliasing). Pointers here are fake host addresses: validation
never dereferences them and fails before anything is launched."""
import ctypes
import os
import re

import pytest

import paper_1710_08332_gb300 as dpia
from paper_1710_08332_gb300 import _native as N
from paper_1710_08332_gb300.strategy import ReduceStrategy

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "dpia.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpia_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = N.lib()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), f"{name} declared in dpia.h but not exported"
    assert set(names) == set(N.SIGNATURES), "binding signatures out of sync with dpia.h"


def test_version_and_empty_error():
    assert dpia.dpia_version() == 10000
    assert isinstance(dpia.dpia_last_error_message(), str)


def _call_dot(st, n=1 << 20, x=0x10000, y=0x20000000, out=0x7000000000, ws=0x7100000000,
              ws_bytes=1 << 20):
    L = N.lib()
    return L.dpia_dot_f32(ctypes.c_void_p(x), ctypes.c_void_p(y), n, ctypes.byref(st.to_c()),
                          ctypes.c_void_p(out), ctypes.c_void_p(ws), ws_bytes, None)


BASE = ReduceStrategy(split=8192, threads=256, vec=4)


@pytest.mark.parametrize("bad,code", [
    (BASE.with_(threads=48), N.ERR_STRATEGY),
    (BASE.with_(threads=2048), N.ERR_STRATEGY),
    (BASE.with_(vec=3), N.ERR_STRATEGY),
    (BASE.with_(vec=16, threads=1024), N.ERR_STRATEGY),
    (BASE.with_(split=1000), N.ERR_STRATEGY),
    (BASE.with_(split=3 * 8192), N.ERR_SHAPE),
    (BASE.with_(map_level="thread", inner_level="seq"), N.ERR_STRATEGY),
    (BASE.with_(map_level="warp", inner_level="block"), N.ERR_STRATEGY),
    (BASE.with_(map_level="grid", inner_level="thread"), N.ERR_STRATEGY),
    (BASE.with_(map_level="block", inner_level="block"), N.ERR_STRATEGY),
    (BASE.with_(map_level="block", inner_level="seq"), N.ERR_UNSUPPORTED),
    (BASE.with_(map_level="block", inner_level="warp"), N.ERR_UNSUPPORTED),
    (BASE.with_(second="tree", threads2=512), N.ERR_STRATEGY),
    (BASE.with_(second="tree", threads2=24), N.ERR_STRATEGY),
    (BASE.with_(grid=-1), N.ERR_STRATEGY),
    (BASE.with_(stage="local", map_level="warp"), N.ERR_UNSUPPORTED),
    (BASE.with_(stage="local", map_level="grid", inner_level="seq", split=8192), N.ERR_UNSUPPORTED),
    (BASE.with_(stage="local", vec=8), N.ERR_UNSUPPORTED),
    (BASE.with_(stage="local", thread_map="contig"), N.ERR_UNSUPPORTED),
])
def test_strategy_validation(bad, code):
    assert _call_dot(bad) == code
    assert dpia.dpia_last_error_message()


def test_hierarchy_legality_message():
    _call_dot(BASE.with_(map_level="warp", inner_level="block"))
    assert "not finer" in dpia.dpia_last_error_message()


def test_pointer_shape_alias_workspace_errors():
    assert _call_dot(BASE, x=0) == N.ERR_NULL
    assert _call_dot(BASE, out=0) == N.ERR_NULL
    assert _call_dot(BASE, n=-5) == N.ERR_SHAPE
    assert _call_dot(BASE, x=0x10004) == N.ERR_ALIGN          # not 16-byte aligned for vec=4
    assert _call_dot(BASE.with_(vec=1), x=0x10004) != N.ERR_ALIGN
    assert _call_dot(BASE, out=0x10000 + 64) == N.ERR_ALIAS  # out inside x
    assert _call_dot(BASE, ws=0) == N.ERR_WORKSPACE
    need = dpia.dpia_dot_workspace_size(1 << 20, BASE)
    assert need == 128 + 128 * 8
    assert _call_dot(BASE, ws_bytes=need - 1) == N.ERR_WORKSPACE
    assert _call_dot(BASE, ws=0x20000000 + 4096) == N.ERR_ALIAS  # workspace inside y
    assert _call_dot(BASE, ws=0x7100000040) == N.ERR_ALIGN      # workspace not 128-byte aligned


def test_workspace_size_matches_chunks():
    for n, s in ((1 << 26, 1024), (1 << 26, 65536), (12345, 1024)):
        st = BASE.with_(split=s, pad=True)
        C = -(-n // s)
        assert dpia.dpia_dot_workspace_size(n, st) == 128 + -(-C * 8 // 128) * 128
    assert dpia.dpia_dot_workspace_size(100, BASE.with_(threads=7)) == 0


def test_int32_rejects_compensated():
    L = N.lib()
    st = BASE.with_(compensated=True)
    rc = L.dpia_dot_i32(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000000), 1 << 20,
                        ctypes.byref(st.to_c()), ctypes.c_void_p(0x7000000000),
                        ctypes.c_void_p(0x7100000000), 1 << 20, None)
    assert rc == N.ERR_STRATEGY


def test_scal_and_gemv_validation():
    L = N.lib()
    p = ctypes.c_void_p
    assert L.dpia_scal_f32(1.5, p(0x10000), p(0x10000 + 8), 1000, 4, None) in (N.ERR_ALIAS, N.ERR_ALIGN)
    assert L.dpia_scal_f32(1.5, p(0x10000), p(0x10000 + 16), 1000, 4, None) == N.ERR_ALIAS
    assert L.dpia_scal_f32(1.5, p(0x10000), p(0x20000), 1000, 5, None) == N.ERR_STRATEGY
    assert L.dpia_scal_f32(1.5, p(0x10000), p(0x20000), -1, 4, None) == N.ERR_SHAPE
    st = ReduceStrategy(split=8192, threads=256, vec=4, second="tree", threads2=256)
    assert L.dpia_gemv_f32(p(0x10000000), 64, 8192, 8192, p(0x20000), p(0x30000), ctypes.byref(st.to_c()),
                           None) == N.ERR_UNSUPPORTED
    st = ReduceStrategy(split=8192, threads=256, vec=4)
    assert L.dpia_gemv_f32(p(0x10000000), 64, 8192, 100, p(0x20000), p(0x30000), ctypes.byref(st.to_c()),
                           None) == N.ERR_SHAPE
    assert L.dpia_gemv_f32(p(0x10000000), 64, 8192, 8193, p(0x20000), p(0x30000), ctypes.byref(st.to_c()),
                           None) == N.ERR_ALIGN
    assert L.dpia_gemv_bwd_f32(p(0x10000000), 1 << 20, 64, 64, p(0x20000), p(0x30000), p(0x40000), None, 64, 8,
                               p(0x50000000), 1 << 30, None) == N.ERR_STRATEGY  # > 65535 row chunks
    assert dpia.dpia_gemv_bwd_workspace_size(8192, 8192, 64) == 128 + 1024 + 128 * 8192 * 4


def test_stage_values():
    """stage is PRIVATE (0) or LOCAL (1); LOCAL passes validation for the
    implemented shape (the fake pointers then fail only on alignment), and is
    not implemented for GEMV rows or batched instances."""
    L = N.lib()
    p = ctypes.c_void_p
    c = BASE.to_c()
    c.stage = 7
    rc = L.dpia_dot_f32(p(0x10000), p(0x20000000), 1 << 20, ctypes.byref(c), p(0x7000000000), p(0x7100000000),
                        1 << 20, None)
    assert rc == N.ERR_STRATEGY and "stage" in dpia.dpia_last_error_message()
    assert _call_dot(BASE.with_(stage="local"), x=0x10004) == N.ERR_ALIGN
    assert dpia.dpia_dot_workspace_size(1 << 20, BASE.with_(stage="local")) == 128 + 128 * 8
    st = ReduceStrategy(split=8192, threads=256, vec=4, stage="local")
    assert L.dpia_gemv_f32(p(0x10000000), 64, 8192, 8192, p(0x20000), p(0x30000), ctypes.byref(st.to_c()),
                           None) == N.ERR_UNSUPPORTED
    from paper_1710_08332_gb300.batch import BatchPolicy
    d = (N.DotInstanceC * 1)()
    d[0] = N.DotInstanceC(0, 4096, BatchPolicy().dot_strategy(4096).with_(stage="local").to_c())
    g = (N.GemvInstanceC * 1)()
    opt = ctypes.byref(N.BatchOptionsC(256, 0))
    assert L.dpia_batch_plan_size(1, d, 0, g, opt) == 0
    assert "stage" in dpia.dpia_last_error_message()


def test_selftest_bounded_wait_range():
    L = N.lib()
    assert L.dpia_selftest_bounded_wait(0, None) == N.ERR_SHAPE
    assert L.dpia_selftest_bounded_wait(2000001, None) == N.ERR_SHAPE
    assert "timeout_us" in dpia.dpia_last_error_message()


def test_gemm_strategy_validation():
    """The BF16 GEMM's tiles are 256 (or, on CTA pairs, 512) x tile_n x 64,
    computed by one CTA or a CTA pair (cluster 1 or 2; 0 = one CTA); anything
    else is refused before any CUDA call."""
    L = N.lib()
    p = ctypes.c_void_p

    def call(**kw):
        st = N.GemmStrategyC(1, kw.get("tile_m", 0), kw.get("tile_n", 0), kw.get("tile_k", 0), kw.get("grid", 0),
                             kw.get("cluster", 0), kw.get("schedule", 0))
        return L.dpia_gemm_bf16(p(0x10000), p(0x20000), p(0x30000), 512, 512, 512, 512, 512, 512, 0, 0,
                                ctypes.byref(st), None)

    assert ctypes.sizeof(N.GemmStrategyC) == 7 * 4
    for c in (3, 4, 8, -1):
        assert call(cluster=c) == N.ERR_STRATEGY
        assert "cluster" in dpia.dpia_last_error_message()
    assert call(grid=-1) == N.ERR_STRATEGY
    assert call(tile_n=96) == N.ERR_UNSUPPORTED
    assert call(tile_n=240) == N.ERR_UNSUPPORTED
    assert call(tile_m=128) == N.ERR_UNSUPPORTED
    assert call(tile_m=512, cluster=1) == N.ERR_UNSUPPORTED  # 512-row tiles only on CTA pairs
    assert call(tile_m=512) == N.ERR_UNSUPPORTED
    assert L.dpia_gemm_bf16(p(0x10000), p(0x20000), p(0x30000), 512, 512, 512, 512, 512, 512, 0, 0, None,
                            None) == N.ERR_NULL


def test_gemm_f32_schedule_values():
    """The FP32 fold's schedules are 0..3; any other value is refused before any
    CUDA call (schedule 3 that does not fit the device is refused on a GPU)."""
    L = N.lib()
    p = ctypes.c_void_p
    for sched, want in ((-1, N.ERR_STRATEGY), (4, N.ERR_STRATEGY), (7, N.ERR_STRATEGY)):
        st = N.GemmStrategyC(1, 0, 0, 0, 0, 0, sched)
        assert L.dpia_gemm_f32(p(0x10000), p(0x20000), p(0x30000), 512, 512, 512, 512, 512, 512, 0, 0,
                               ctypes.byref(st), None) == want
        assert "schedule" in dpia.dpia_last_error_message()


def test_batch_row_alignment_is_checked():
    """The packer's row alignment is a positive multiple of 4 floats (the vector
    loads need 16-byte rows); it is checked before anything is planned."""
    from paper_1710_08332_gb300.batch import Batch

    for bad in (0, 3, 6, -4):
        with pytest.raises(ValueError):
            Batch([16], [(4, 8)], "cpu", row_align=bad)


def test_batch_schedule_values():
    """Schedules 0 (longest first, round robin), 1 (equal-cost runs) and 2
    (longest first, taken from a counter) plan; anything else is refused."""
    from paper_1710_08332_gb300.batch import BatchPolicy

    L = N.lib()
    d = (N.DotInstanceC * 1)()
    d[0] = N.DotInstanceC(0, 4096, BatchPolicy().dot_strategy(4096).to_c())
    g = (N.GemvInstanceC * 1)()
    for sched in (0, 1, 2):
        assert L.dpia_batch_plan_size(1, d, 0, g, ctypes.byref(N.BatchOptionsC(256, sched))) > 0
    for sched in (-1, 3):
        assert L.dpia_batch_plan_size(1, d, 0, g, ctypes.byref(N.BatchOptionsC(256, sched))) == 0
        assert "schedule" in dpia.dpia_last_error_message()
