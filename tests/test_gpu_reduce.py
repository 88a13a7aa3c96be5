"""GPU parity of the strategy reductions and maps against the CPU oracle.

Same-strategy FP32 and int32 results must be bit-identical to the oracle's
loop-nest evaluation of the same tree; FP32 results must also lie within the
normwise bound |r - r64| <= 1e-5 * sum|x_i y_i| of the exact value.
"""
import numpy as np
import pytest
import torch

import paper_1710_08332_gb300 as dpia
from oracle import loopnest, naive64
from synth import workloads as W
from tests.helpers import assert_bits_equal, host, oracle_strategy

pytestmark = pytest.mark.gpu

RS = dpia.ReduceStrategy


def _run(op, x, y, st):
    n = x.numel()
    ws = torch.zeros(dpia.dpia_dot_workspace_size(n, st), dtype=torch.uint8, device=x.device)
    if op == "dot":
        out = torch.full((1,), float("nan"), device=x.device)
        dpia.dpia_dot_f32(x, y, n, st, out, ws)
    elif op == "asum":
        out = torch.full((1,), float("nan"), device=x.device)
        dpia.dpia_asum_f32(x, n, st, out, ws)
    else:
        out = torch.full((1,), -1, dtype=torch.int64, device=x.device)
        dpia.dpia_dot_i32(x, y, n, st, out, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0, "workspace counter not left at zero"
    return host(out)[0]


def _oracle(op, x, y, st):
    o = oracle_strategy(st)
    if op == "dot":
        return loopnest.dot_f32(host(x), host(y), o)
    if op == "asum":
        return loopnest.asum_f32(host(x), o)
    return loopnest.dot_i32(host(x), host(y), o)


# --------------------------------------------------------------------------
# the dot workload: n = 2^20, split 8192, 128 partials, seq second level
# --------------------------------------------------------------------------

CFG1 = RS(split=W.DOT_SPLIT, threads=256, vec=4, map_level="block", inner_level="thread",
          second="seq")


def test_dot_f32_n2e20_split8192(cuda_device):
    x, y = W.dot_f32("cuda")
    got = _run("dot", x, y, CFG1)
    want = loopnest.dot_f32(host(x), host(y), oracle_strategy(CFG1))
    assert_bits_equal(np.float32(got), np.float32(want), "dot f32 config")
    exact = naive64.dot_exact(host(x), host(y))
    assert abs(float(got) - exact) <= 1e-5 * naive64.abs_dot_f64(host(x), host(y))


def test_dot_i32_n2e20_split8192(cuda_device):
    x, y = W.dot_i32("cuda")
    got = _run("i32", x, y, CFG1)
    want = int(np.dot(host(x).astype(np.int64), host(y).astype(np.int64)))
    assert int(got) == want


# --------------------------------------------------------------------------
# strategy sweep at sizes spanning several chunks and a ragged tail
# --------------------------------------------------------------------------

SWEEP = [
    RS(split=8192, threads=256, vec=4),
    RS(split=8192, threads=256, vec=4, thread_map="contig"),
    RS(split=4096, threads=1024, vec=4, second="tree", threads2=1024),
    RS(split=1024, threads=32, vec=1, second="tree", threads2=8),
    RS(split=2048, threads=64, vec=2, second="tree", threads2=64, thread_map="contig"),
    RS(split=16384, threads=512, vec=8),
    RS(split=16384, threads=256, vec=16, second="tree", threads2=1),
    RS(split=4096, threads=128, vec=4, map_level="warp"),
    RS(split=512, threads=256, vec=16, map_level="warp", second="tree", threads2=256),
    RS(split=256, threads=128, vec=4, map_level="grid", inner_level="seq"),
    RS(split=64, threads=256, vec=1, map_level="grid", inner_level="seq", second="tree", threads2=128),
    RS(split=8192, threads=256, vec=4, grid=3),
    RS(split=8192, threads=256, vec=4, compensated=True),
    RS(split=2048, threads=128, vec=8, compensated=True, second="tree", threads2=64, map_level="warp"),
    RS(split=512, threads=64, vec=2, compensated=True, map_level="grid", inner_level="seq"),
]


def _sid(st):
    return (f"{st.map_level[0]}s{st.split}T{st.threads}V{st.vec}{st.thread_map[0]}"
            f"{st.second}{st.threads2 if st.second == 'tree' else ''}{'K' if st.compensated else ''}"
            f"{'g' + str(st.grid) if st.grid else ''}")


@pytest.mark.parametrize("st", SWEEP, ids=_sid)
@pytest.mark.parametrize("op", ["dot", "asum", "i32"])
def test_strategy_sweep_bits(cuda_device, st, op):
    if op == "i32" and st.compensated:
        pytest.skip("compensated is f32 only")
    n_exact = st.split * 37
    for n, pad in ((n_exact, False), (n_exact - 3 * st.vec - 5 if n_exact > 64 else n_exact, True)):
        s = st.with_(pad=pad)
        if op == "i32":
            x, y = W.dot_i32("cpu", n=n, seed=21)
        else:
            x, y = W.dot_f32("cpu", n=n, seed=21)
            x[::13] *= 1e-3
        x, y = x.cuda(), y.cuda()
        got = _run(op, x, y, s)
        want = _oracle(op, x, y, s)
        if op == "i32":
            assert int(got) == int(want)
        else:
            assert_bits_equal(np.float32(got), np.float32(want), f"{op} n={n}")


# toLocal: chunks staged through shared memory by bulk asynchronous copies.
# Same items, same order: bit-identical to the oracle and to the direct loads.
SWEEP_LOCAL = [
    RS(split=8192, threads=256, vec=4, stage="local"),
    RS(split=4096, threads=1024, vec=4, second="tree", threads2=1024, stage="local"),
    RS(split=2048, threads=32, vec=4, second="tree", threads2=8, stage="local"),
    RS(split=3072, threads=256, vec=4, stage="local"),              # 3 rows: tiles of 2 + 1
    RS(split=3072, threads=128, vec=4, second="tree", threads2=128, stage="local"),  # 6 rows: 4 + 2
    RS(split=65536, threads=512, vec=4, stage="local"),
    RS(split=8192, threads=256, vec=4, grid=3, stage="local"),
    RS(split=8192, threads=256, vec=4, compensated=True, stage="local"),
]


@pytest.mark.parametrize("st", SWEEP_LOCAL, ids=lambda st: "local-" + _sid(st))
@pytest.mark.parametrize("op", ["dot", "asum", "i32"])
def test_staged_local_bits(cuda_device, st, op):
    if op == "i32" and st.compensated:
        pytest.skip("compensated is f32 only")
    n_exact = st.split * 41
    for n, pad in ((n_exact, False), (n_exact - 9, True), (st.split // 2 + 4, True), (st.split, False)):
        s = st.with_(pad=pad)
        if op == "i32":
            x, y = W.dot_i32("cpu", n=n, seed=22)
        else:
            x, y = W.dot_f32("cpu", n=n, seed=22)
            x[::11] *= 1e-3
        x, y = x.cuda(), y.cuda()
        got = _run(op, x, y, s)
        want = _oracle(op, x, y, s)
        direct = _run(op, x, y, s.with_(stage="private"))
        if op == "i32":
            assert int(got) == int(want) == int(direct)
        else:
            assert_bits_equal(np.float32(got), np.float32(want), f"{op} n={n}")
            assert_bits_equal(np.float32(got), np.float32(direct), f"{op} n={n} vs direct")
    assert dpia.dpia_poll_device_status() == 0  # no bounded wait ran out


def test_repeat_and_stream_determinism(cuda_device):
    x, y = W.dot_f32("cuda", n=(1 << 22) + 77, seed=5)
    st = RS(split=4096, threads=256, vec=4, second="tree", threads2=256, pad=True)
    a = _run("dot", x, y, st)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ws = torch.zeros(dpia.dpia_dot_workspace_size(x.numel(), st), dtype=torch.uint8, device="cuda")
        out = torch.empty(1, device="cuda")
        for _ in range(3):
            dpia.dpia_dot_f32(x, y, x.numel(), st, out, ws, stream=s)
    s.synchronize()
    assert_bits_equal(host(out), np.array([a], np.float32), "stream repeat")


def test_edge_cases(cuda_device):
    st = RS(split=1024, threads=256, vec=4, pad=True)
    e = torch.empty(0, device="cuda")
    assert float(dpia.dot(e, e, st)) == 0.0
    for n in (1, 3, 4, 5, 1023, 1025):
        x, y = W.dot_f32("cpu", n=n, seed=n)
        got = _run("dot", x.cuda(), y.cuda(), st)
        assert_bits_equal(np.float32(got), loopnest.dot_f32(x.numpy(), y.numpy(), oracle_strategy(st)), f"n={n}")
    # -0 products and subnormals are kept (no flush to zero)
    x = torch.tensor([-0.0, 1e-38, 1e-39, -1e-40] * 256, device="cuda")
    y = torch.tensor([1.0, 0.5, 3.0, 2.0] * 256, device="cuda")
    got = _run("dot", x, y, RS(split=1024, threads=256, vec=4))
    want = loopnest.dot_f32(host(x), host(y), oracle_strategy(RS(split=1024, threads=256, vec=4)))
    assert_bits_equal(np.float32(got), np.float32(want), "subnormals")
    assert got != 0.0


def test_rejects_misaligned_and_small_workspace(cuda_device):
    x, y = W.dot_f32("cuda", n=8192 + 4, seed=3)
    out = torch.empty(1, device="cuda")
    st = RS(split=8192, threads=256, vec=4)
    ws = torch.zeros(dpia.dpia_dot_workspace_size(8192, st), dtype=torch.uint8, device="cuda")
    with pytest.raises(dpia.DPIAError, match="ALIGN"):
        dpia.dpia_dot_f32(x[1:8193], y[1:8193], 8192, st, out, ws)
    with pytest.raises(dpia.DPIAError, match="WORKSPACE"):
        dpia.dpia_dot_f32(x, y, 8192, st, out, ws[:64])
    with pytest.raises(dpia.DPIAError, match="ALIAS"):
        dpia.dpia_dot_f32(x, y, 8192, st, x[100:101], ws)


# --------------------------------------------------------------------------
# bandwidth workload: n = 2^26, split swept 1024 .. 65536
# --------------------------------------------------------------------------


@pytest.fixture(scope="module")
def bw_inputs():
    x, y = W.bandwidth("cuda")
    return x, y, host(x), host(y)


@pytest.mark.parametrize("split", [1024, 4096, 8192, 16384, 65536])
def test_bandwidth_dot_asum_bits(cuda_device, bw_inputs, split):
    x, y, hx, hy = bw_inputs
    for st in (RS(split=split, threads=256, vec=4, second="tree", threads2=256),
               RS(split=split, threads=min(1024, split // 4), vec=4, second="seq"),
               RS(split=split, threads=256, vec=4, second="tree", threads2=256, stage="local")):
        got = _run("dot", x, y, st)
        assert_bits_equal(np.float32(got), loopnest.dot_f32(hx, hy, oracle_strategy(st)), f"dot s={split}")
        got = _run("asum", x, None, st)
        assert_bits_equal(np.float32(got), loopnest.asum_f32(hx, oracle_strategy(st)), f"asum s={split}")
    exact = naive64.dot_f64(hx, hy)
    assert abs(float(got) - naive64.asum_exact(hx)) <= 1e-5 * naive64.asum_exact(hx)
    got = _run("dot", x, y, RS(split=split, threads=256, vec=4, second="tree", threads2=256))
    assert abs(float(got) - exact) <= 1e-5 * naive64.abs_dot_f64(hx, hy)


def test_bandwidth_scal_exact(cuda_device, bw_inputs):
    x, _, hx, _ = bw_inputs
    y = torch.empty_like(x)
    dpia.dpia_scal_f32(W.SCAL_A, x, y, x.numel(), 4)
    assert_bits_equal(host(y), loopnest.scal_f32(W.SCAL_A, hx), "scal")
    # in place, ragged length, other vector widths
    for vec, n in ((1, 1001), (2, 4099), (8, 65541), (16, 65555)):
        z = x[:n].clone()
        dpia.dpia_scal_f32(-0.75, z, z, n, vec)
        assert_bits_equal(host(z), loopnest.scal_f32(-0.75, hx[:n]), f"scal vec={vec}")


# --------------------------------------------------------------------------
# GEMV 8192 x 8192 forward and backward
# --------------------------------------------------------------------------


@pytest.fixture(scope="module")
def gemv_inputs():
    A, x, dy = W.gemv("cuda")
    return A, x, dy, host(A), host(x), host(dy)


@pytest.mark.parametrize("st", [
    RS(split=8192, threads=256, vec=4),
    RS(split=2048, threads=256, vec=4, thread_map="contig"),
    RS(split=8192, threads=128, vec=4, map_level="warp"),
    RS(split=8192, threads=512, vec=8, compensated=True),
], ids=_sid)
def test_gemv_fwd_bits(cuda_device, gemv_inputs, st):
    A, x, _, hA, hx, _ = gemv_inputs
    y = torch.empty(A.shape[0], device="cuda")
    dpia.dpia_gemv_f32(A, A.shape[0], A.shape[1], A.stride(0), x, y, st)
    want = loopnest.gemv_f32(hA, hx, oracle_strategy(st))
    assert_bits_equal(host(y), want, "gemv")
    ref = naive64.gemv_f64(hA, hx)
    assert np.all(np.abs(host(y) - ref) <= 1e-5 * naive64.gemv_abs_f64(hA, hx))


@pytest.mark.parametrize("row_split", [64, 256, 8192])
def test_gemv_bwd_bits(cuda_device, gemv_inputs, row_split):
    A, x, dy, hA, hx, hdy = gemv_inputs
    dx, dA = dpia.gemv_bwd(A, x, dy, row_split=row_split)
    assert_bits_equal(host(dx), loopnest.gemv_bwd_dx_f32(hA, hdy, row_split), "dx")
    if row_split == 64:
        hdA = host(dA)
        want = loopnest.gemv_bwd_dA_f32(hx, hdy)
        assert_bits_equal(hdA, want, "dA")
    ref = hA.astype(np.float64).T @ hdy.astype(np.float64)
    assert np.all(np.abs(host(dx) - ref) <= 1e-5 * (np.abs(hA).T @ np.abs(hdy)))


def test_gemv_ragged_shapes(cuda_device):
    for (M, N_) in ((37, 1000), (300, 4097), (1, 129), (513, 256)):
        A, x, dy = W.gemv("cpu", M=M, N=N_, seed=M)
        Ad = torch.zeros(M, (N_ + 3) // 4 * 4, device="cuda")
        Ad[:, :N_] = A.cuda()
        st = dpia.ops.default_gemv_strategy(N_)
        y = torch.empty(M, device="cuda")
        xd = torch.zeros((N_ + 3) // 4 * 4, device="cuda")
        xd[:N_] = x.cuda()
        dpia.dpia_gemv_f32(Ad, M, N_, Ad.stride(0), xd, y, st)
        want = np.array([loopnest.dot_f32(A[i].numpy(), x.numpy(), oracle_strategy(st)) for i in range(M)],
                        np.float32)
        assert_bits_equal(host(y), want, f"gemv {M}x{N_}")
        dx = torch.empty(N_, device="cuda")
        dA = torch.empty(M, (N_ + 3) // 4 * 4, device="cuda")
        ws = torch.zeros(dpia.dpia_gemv_bwd_workspace_size(M, N_, 32), dtype=torch.uint8, device="cuda")
        dpia.dpia_gemv_bwd_f32(Ad, M, N_, Ad.stride(0), xd, dy.cuda(), dx, dA, dA.stride(0), 32, ws)
        assert_bits_equal(host(dx), loopnest.gemv_bwd_dx_f32(A.numpy(), dy.numpy(), 32), f"dx {M}x{N_}")
        assert_bits_equal(host(dA)[:, :N_], loopnest.gemv_bwd_dA_f32(x.numpy(), dy.numpy()), f"dA {M}x{N_}")


@pytest.mark.parametrize("st", [
    RS(split=256, threads=128, vec=4, map_level="warp", pad=True),
    RS(split=1024, threads=256, vec=4, map_level="warp", pad=True),
    RS(split=512, threads=128, vec=4, map_level="warp", thread_map="contig", pad=True),
    RS(split=1024, threads=128, vec=4, map_level="warp", compensated=True, pad=True),
    RS(split=1024, threads=256, vec=4, pad=True),
    RS(split=2048, threads=128, vec=8, pad=True),
], ids=_sid)
def test_gemv_padded_row_chunks(cuda_device, st):
    """Rows whose last chunk reaches past N (identity items), at block and warp
    level: the whole vectors below N take the batched loads, the rest is the
    straddling vector and identity items."""
    for (M, N_) in ((67, 1000), (33, 4097), (9, 129), (130, 3000)):
        A, x, _ = W.gemv("cpu", M=M, N=N_, seed=N_)
        ld = (N_ + 7) // 8 * 8
        Ad = torch.zeros(M, ld, device="cuda")
        Ad[:, :N_] = A.cuda()
        xd = torch.zeros(ld, device="cuda")
        xd[:N_] = x.cuda()
        y = torch.full((M,), float("nan"), device="cuda")
        dpia.dpia_gemv_f32(Ad, M, N_, ld, xd, y, st)
        assert_bits_equal(host(y), loopnest.gemv_f32(A.numpy(), x.numpy(), oracle_strategy(st)), f"{M}x{N_}")


def test_dot_bwd_exact(cuda_device):
    x, y = W.dot_f32("cuda", n=(1 << 20) + 3, seed=9)
    g = torch.tensor([0.37], device="cuda")
    dx, dy = dpia.dot_bwd(x, y, g)
    wx, wy = loopnest.dot_bwd_f32(host(x), host(y), 0.37)
    assert_bits_equal(host(dx), wx, "dx")
    assert_bits_equal(host(dy), wy, "dy")


@pytest.mark.slow
def test_beyond_int32_indexing(cuda_device):
    """n > 2^31: 64-bit index arithmetic in the fold and in the chunk map.

    All ones: every chunk sum is 2^20, the last (padded) chunk holds 2048, and
    each tree node 2^k + 2048 (k <= 31) is exact in binary32, so the result is
    exactly n."""
    n = (1 << 31) + 2048
    x = torch.ones(n, device="cuda")
    st = RS(split=1 << 20, threads=1024, vec=4, second="tree", threads2=1024, pad=True)
    got = _run("asum", x, None, st)
    assert float(got) == float(n)
    del x
    torch.cuda.empty_cache()
