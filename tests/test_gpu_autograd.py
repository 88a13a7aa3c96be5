"""Gradients through the autograd Functions (forward and backward in the
library's kernels), checked against the oracle's kernels bit for bit where the
backward is a fixed strategy, and against FP64 adjoints and FP64 central
finite differences of the FP64 forward."""
import numpy as np
import pytest
import torch

from oracle import grads, loopnest, naive64
from paper_1710_08332_gb300 import autograd as AG
from paper_1710_08332_gb300.strategy import ReduceStrategy
from tests.helpers import assert_bits_equal, host

pytestmark = pytest.mark.gpu


def _leaf(t):
    return t.detach().clone().cuda().requires_grad_(True)


def test_dot_grad(cuda_device):
    g = torch.Generator().manual_seed(1)
    x = torch.rand(4099, generator=g) * 2 - 1
    y = torch.rand(4099, generator=g) * 2 - 1
    xd, yd = _leaf(x), _leaf(y)
    out = AG.dot(xd, yd, ReduceStrategy(split=1024, threads=256, vec=4, pad=True))
    out.backward(torch.tensor(0.7, device="cuda"))
    wx, wy = loopnest.dot_bwd_f32(x.numpy(), y.numpy(), np.float32(0.7))
    assert_bits_equal(host(xd.grad), wx, "dx")
    assert_bits_equal(host(yd.grad), wy, "dy")
    ax, ay = grads.dot_adjoint(x.numpy(), y.numpy(), 0.7)
    assert np.allclose(host(xd.grad), ax, rtol=1e-6, atol=1e-9)
    assert np.allclose(host(yd.grad), ay, rtol=1e-6, atol=1e-9)
    # finite differences on a small prefix
    xs, ys = x.numpy()[:9].astype(np.float64), y.numpy()[:9].astype(np.float64)
    xs_d, ys_d = _leaf(torch.from_numpy(xs.astype(np.float32))), _leaf(torch.from_numpy(ys.astype(np.float32)))
    AG.dot(xs_d, ys_d, ReduceStrategy(split=1024, threads=256, vec=1, pad=True)).backward(
        torch.tensor(1.3, device="cuda"))
    fd = grads.central_fd(grads.dot_fwd, [xs, ys], 0, 1.3)
    assert np.allclose(host(xs_d.grad), fd, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("M,N", [(33, 70), (300, 1024)])
def test_gemv_grad(cuda_device, M, N):
    g = torch.Generator().manual_seed(M + N)
    A = torch.randn(M, N, generator=g) / np.sqrt(N)
    x = torch.rand(N, generator=g) * 2 - 1
    dy = torch.rand(M, generator=g) * 2 - 1
    Ad, xd = _leaf(A), _leaf(x)
    y = AG.gemv(Ad, xd, row_split=16)
    y.backward(dy.cuda())
    assert_bits_equal(host(xd.grad), loopnest.gemv_bwd_dx_f32(A.numpy(), dy.numpy(), 16), "dx")
    assert_bits_equal(host(Ad.grad), loopnest.gemv_bwd_dA_f32(x.numpy(), dy.numpy()), "dA")
    adA, adx = grads.gemv_adjoint(A.numpy(), x.numpy(), dy.numpy())
    assert np.all(np.abs(host(xd.grad) - adx) <= 1e-5 * (np.abs(A.numpy()).T @ np.abs(dy.numpy())) + 1e-12)
    assert np.allclose(host(Ad.grad), adA, rtol=1e-6, atol=1e-12)
    if M * N <= 4000:
        fd = grads.central_fd(grads.gemv_fwd, [A.numpy().astype(np.float64), x.numpy().astype(np.float64)], 1,
                              dy.numpy())
        assert np.allclose(host(xd.grad), fd, rtol=1e-4, atol=1e-6)


def test_gemm_f32_grad(cuda_device):
    g = torch.Generator().manual_seed(5)
    A = torch.randn(40, 36, generator=g)
    B = torch.randn(36, 28, generator=g)
    dC = torch.randn(40, 28, generator=g)
    Ad, Bd = _leaf(A), _leaf(B)
    C = AG.gemm(Ad, Bd, "f32", "fma")
    assert_bits_equal(host(C), loopnest.gemm_f32(A.numpy(), B.numpy(), False, False, True), "C")
    C.backward(dC.cuda())
    # dA = dC B^T and dB = A^T dC through the same fold kernel with transposed layouts
    assert_bits_equal(host(Ad.grad), loopnest.gemm_f32(dC.numpy(), B.numpy(), False, True, True), "dA")
    assert_bits_equal(host(Bd.grad), loopnest.gemm_f32(A.numpy(), dC.numpy(), True, False, True), "dB")
    gA, gB = grads.gemm_adjoint(A.numpy(), B.numpy(), dC.numpy())
    assert np.allclose(host(Ad.grad), gA, rtol=1e-5, atol=1e-4)
    assert np.allclose(host(Bd.grad), gB, rtol=1e-5, atol=1e-4)
    a, b = A.numpy()[:5, :4].astype(np.float64), B.numpy()[:4, :3].astype(np.float64)
    dc = dC.numpy()[:5, :3].astype(np.float64)
    a_d, b_d = _leaf(torch.from_numpy(a.astype(np.float32))), _leaf(torch.from_numpy(b.astype(np.float32)))
    AG.gemm(a_d, b_d, "f32").backward(torch.from_numpy(dc.astype(np.float32)).cuda())
    assert np.allclose(host(a_d.grad), grads.central_fd(grads.gemm_fwd, [a, b], 0, dc), rtol=1e-4, atol=1e-5)
    assert np.allclose(host(b_d.grad), grads.central_fd(grads.gemm_fwd, [a, b], 1, dc), rtol=1e-4, atol=1e-5)


def test_gemm_bf16_grad(cuda_device):
    g = torch.Generator().manual_seed(6)
    A = torch.randn(512, 256, generator=g)
    B = torch.randn(256, 384, generator=g)
    dC = torch.randn(512, 384, generator=g)
    Ad, Bd = _leaf(A), _leaf(B)
    AG.gemm(Ad, Bd, "bf16").backward(dC.cuda())
    a16, b16, c16 = (naive64.bf16_round(t.numpy()) for t in (A, B, dC))
    for got, ref16, ref in ((host(Ad.grad), c16 @ b16.T, dC.numpy().astype(np.float64) @ B.numpy().T),
                            (host(Bd.grad), a16.T @ c16, A.numpy().T.astype(np.float64) @ dC.numpy())):
        assert np.linalg.norm(got - ref16) / np.linalg.norm(ref16) <= 1e-4
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-2


def test_composite_chain(cuda_device):
    """loss = dot(gemv(A, x), w): gradients flow through both Functions."""
    g = torch.Generator().manual_seed(7)
    A = torch.randn(64, 256, generator=g) / 16
    x = torch.rand(256, generator=g) * 2 - 1
    w = torch.rand(64, generator=g) * 2 - 1
    Ad, xd, wd = _leaf(A), _leaf(x), _leaf(w)
    loss = AG.dot(AG.gemv(Ad, xd), wd, ReduceStrategy(split=1024, threads=256, vec=4, pad=True))
    loss.backward()
    A64, x64, w64 = (t.numpy().astype(np.float64) for t in (A, x, w))
    assert np.allclose(host(wd.grad), A64 @ x64, rtol=1e-5, atol=1e-6)
    assert np.allclose(host(xd.grad), A64.T @ w64, rtol=1e-4, atol=1e-6)
    assert np.allclose(host(Ad.grad), np.outer(w64, x64), rtol=1e-6, atol=1e-9)


def test_workspace_kinds_do_not_collide(cuda_device):
    """A dot (which leaves partials after its counter) followed by a GEMV
    backward on the same stream through the convenience API: each kind keeps
    its own workspace, so the backward's per-tile counters start at zero."""
    import paper_1710_08332_gb300 as dpia

    g = torch.Generator().manual_seed(8)
    A = torch.randn(96, 2048, generator=g)
    x = torch.rand(2048, generator=g) * 2 - 1
    dy = torch.rand(96, generator=g) * 2 - 1
    v = torch.rand(1 << 20, generator=g).cuda()
    for _ in range(2):
        dpia.dot(v, v)
        dx, _ = dpia.gemv_bwd(A.cuda(), x.cuda(), dy.cuda(), need_dA=False, row_split=32)
        assert_bits_equal(host(dx), loopnest.gemv_bwd_dx_f32(A.numpy(), dy.numpy(), 32), "dx after dot")
