"""Batched uneven instances: one persistent launch per direction.

Every instance's result must be bit-identical to the oracle's evaluation of
that instance's own strategy, forward and backward -- on small batches under
several policies and on the full batched workload -- and the per-launch
baseline (one single-instance call per instance with the same strategy) and a
CUDA-graph replay must reproduce the same bits.
"""
import math

import numpy as np
import pytest
import torch

from oracle import loopnest
from paper_1710_08332_gb300.batch import Batch, BatchPolicy
from synth import generator
from synth import workloads as W
from tests.helpers import assert_bits_equal, host, oracle_strategy

pytestmark = pytest.mark.gpu


def _inputs(b: Batch, seed: int):
    """Packed inputs drawn from one generator (padding slots are drawn too and unused)."""
    g = generator(seed, b.device)
    xs = torch.rand(b.xs_len, generator=g, device=b.device).mul_(2).sub_(1)
    ys = torch.rand(b.xs_len, generator=g, device=b.device).mul_(2).sub_(1)
    As = torch.randn(b.as_len, generator=g, device=b.device)
    for i, (_, n) in enumerate(b.gemv_shapes):
        b.a_view(As, i).mul_(1.0 / math.sqrt(n))
    gx = torch.rand(b.gx_len, generator=g, device=b.device).mul_(2).sub_(1)
    dot_g = torch.rand(len(b.dot_lengths), generator=g, device=b.device).mul_(2).sub_(1)
    gdy = torch.rand(b.gy_len, generator=g, device=b.device).mul_(2).sub_(1)
    return xs, ys, As, gx, dot_g, gdy


def _outputs(b: Batch):
    dev = b.device
    return (torch.full((max(len(b.dot_lengths), 1),), float("nan"), device=dev),
            torch.full((b.gy_len,), float("nan"), device=dev))


def _bwd_outputs(b: Batch):
    dev = b.device
    return (torch.zeros(b.xs_len, device=dev), torch.zeros(b.xs_len, device=dev),
            torch.zeros(b.as_len, device=dev), torch.zeros(b.gx_len, device=dev))


def _check_against_oracle(b, xs, ys, As, gx, dot_g, gdy, dot_out, gy, dxs, dys, dAs, dgx, dots=None, gemvs=None):
    hx, hy, hA, hgx, hg, hdy = (host(t) for t in (xs, ys, As, gx, dot_g, gdy))
    hdot, hgy, hdxs, hdys, hdAs, hdgx = (host(t) for t in (dot_out, gy, dxs, dys, dAs, dgx))
    for i in (range(len(b.dot_lengths)) if dots is None else dots):
        o, n = b.dot_offs[i], b.dot_lengths[i]
        st = oracle_strategy(b.dot_st[i])
        assert_bits_equal(np.float32(hdot[i]), loopnest.dot_f32(hx[o:o + n], hy[o:o + n], st), f"dot {i} n={n}")
        wx, wy = loopnest.dot_bwd_f32(hx[o:o + n], hy[o:o + n], hg[i])
        assert_bits_equal(hdxs[o:o + n], wx, f"dot {i} dx")
        assert_bits_equal(hdys[o:o + n], wy, f"dot {i} dy")
    for i in (range(len(b.gemv_shapes)) if gemvs is None else gemvs):
        M, N_ = b.gemv_shapes[i]
        lda, ao, xo, yo = b.ldas[i], b.a_offs[i], b.gx_offs[i], b.gy_offs[i]
        A = np.ascontiguousarray(hA[ao:ao + M * lda].reshape(M, lda)[:, :N_])
        x, dy = hgx[xo:xo + N_], hdy[yo:yo + M]
        assert_bits_equal(hgy[yo:yo + M], loopnest.gemv_f32(A, x, oracle_strategy(b.gemv_st[i])), f"gemv {i} y")
        assert_bits_equal(np.ascontiguousarray(hdAs[ao:ao + M * lda].reshape(M, lda)[:, :N_]),
                          loopnest.gemv_bwd_dA_f32(x, dy), f"gemv {i} dA")
        assert_bits_equal(hdgx[xo:xo + N_], loopnest.gemv_bwd_dx_f32(A, dy, b.policy.row_split), f"gemv {i} dx")


SMALL_DOTS = [0, 1, 3, 100, 1023, 1024, 1025, 5000, 8192, 8193, 20000, 70001]
# (64, 256), (17, 384), (33, 511), (5, 129): two, three and four vectors a lane, whole and ragged,
# on the forward path that takes narrow rows two at a time; (9, 640), (3, 513), (12, 1024):
# five to eight vectors a lane, loaded at once
SMALL_GEMVS = [(1, 1), (3, 5), (100, 257), (300, 1000), (50, 4096), (2000, 128), (0, 64), (257, 4100),
               (64, 256), (17, 384), (33, 511), (5, 129), (9, 640), (3, 513), (12, 1024)]


@pytest.mark.parametrize("policy", [BatchPolicy(), BatchPolicy(threads=128, dot_split_cap=2048, dot_second="seq",
                                                                gemv_split_cap=256, row_split=100),
                                    BatchPolicy(schedule=1),
                                    BatchPolicy(threads=64, schedule=1, row_split=37),
                                    BatchPolicy(schedule=2), BatchPolicy(threads=64, schedule=2, row_split=37)],
                         ids=["default", "small-splits", "contiguous", "contiguous-64", "dynamic", "dynamic-64"])
def test_batch_bits_against_oracle(cuda_device, policy):
    rng = np.random.default_rng(11)
    dots = SMALL_DOTS + [int(v) for v in np.exp(rng.uniform(np.log(256), np.log(20000), 150))]
    gemvs = SMALL_GEMVS + [(int(m), int(n)) for m, n in zip(np.exp(rng.uniform(np.log(16), np.log(3000), 12)),
                                                           np.exp(rng.uniform(np.log(32), np.log(2048), 12)))]
    b = Batch(dots, gemvs, "cuda", policy)
    xs, ys, As, gx, dot_g, gdy = _inputs(b, 3)
    dot_out, gy = _outputs(b)
    b.forward(xs, ys, dot_out, As, gx, gy)
    dxs, dys, dAs, dgx = _bwd_outputs(b)
    b.backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx)
    torch.cuda.synchronize()
    _check_against_oracle(b, xs, ys, As, gx, dot_g, gdy, dot_out, gy, dxs, dys, dAs, dgx)
    # the per-instance counters (and the dynamic schedule's) are back at zero, so a
    # second launch gives the same bits
    assert not host(b.ws)[:128 + 4 * len(dots)].view(np.uint32).any()
    dot2, gy2 = _outputs(b)
    b.forward(xs, ys, dot2, As, gx, gy2)
    dxs2, dys2, dAs2, dgx2 = _bwd_outputs(b)
    b.backward(xs, ys, dot_g, dxs2, dys2, As, gx, gdy, dAs2, dgx2)
    torch.cuda.synchronize()
    assert host(dot2).tobytes() == host(dot_out).tobytes() and host(gy2).tobytes() == host(gy).tobytes()
    assert host(dgx2).tobytes() == host(dgx).tobytes() and host(dAs2).tobytes() == host(dAs).tobytes()
    assert not host(b.ws)[:128].view(np.uint32).any()


def test_batch_equals_per_launch_and_graph(cuda_device):
    rng = np.random.default_rng(12)
    dots = [int(v) for v in np.exp(rng.uniform(np.log(256), np.log(65536), 300))]
    gemvs = [(int(m), int(n)) for m, n in zip(np.exp(rng.uniform(np.log(256), np.log(8192), 24)),
                                             np.exp(rng.uniform(np.log(256), np.log(4096), 24)))]
    b = Batch(dots, gemvs, "cuda")
    xs, ys, As, gx, dot_g, gdy = _inputs(b, 4)
    d1, y1 = _outputs(b)
    b.forward(xs, ys, d1, As, gx, y1)
    d2, y2 = _outputs(b)
    b.per_launch_forward(xs, ys, d2, As, gx, y2)
    bw1 = _bwd_outputs(b)
    b.backward(xs, ys, dot_g, *bw1[:2], As, gx, gdy, *bw1[2:])
    bw2 = _bwd_outputs(b)
    b.per_launch_backward(xs, ys, dot_g, *bw2[:2], As, gx, gdy, *bw2[2:])
    torch.cuda.synchronize()
    assert host(d1).tobytes() == host(d2).tobytes()
    for i in range(len(gemvs)):
        assert host(b.gy_view(y1, i)).tobytes() == host(b.gy_view(y2, i)).tobytes()
    for t1, t2 in zip(bw1, bw2):
        assert host(t1).tobytes() == host(t2).tobytes()
    # one launch captured in a CUDA graph, replayed twice
    d3, y3 = _outputs(b)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.forward(xs, ys, d3, As, gx, y3)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.forward(xs, ys, d3, As, gx, y3)
    for _ in range(2):
        d3.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert host(d3).tobytes() == host(d1).tobytes()


def _candidate_policies():
    from paper_1710_08332_gb300 import tune

    return tune.batch_candidates()


@pytest.mark.slow
@pytest.mark.parametrize("policy", _candidate_policies(),
                         ids=lambda p: f"T{p.threads}-cap{p.dot_split_cap}-rs{p.row_split}-sched{p.schedule}")
def test_batched_workload_full(cuda_device, policy):
    """The batched workload at full size -- 4096 dots and 512 GEMVs, lengths and
    rows log-uniform in [256, 65536], columns in [256, 4096], seed 3 -- under
    every policy the autotuner chooses from (the bench times the one it picks),
    every instance against the oracle, forward and backward: each dot's result,
    dx and dy, and each GEMV's y, dx and dA, element by element. The packed
    matrices are tens of GB, so each GEMV's matrix and dA are copied to the
    host one instance at a time."""
    dl, rows, cols = W.batched_shapes()
    b = Batch(dl.tolist(), list(zip(rows.tolist(), cols.tolist())), "cuda", policy)
    xs, ys, As, gx, dot_g, gdy = _inputs(b, 3)
    d1, y1 = _outputs(b)
    b.forward(xs, ys, d1, As, gx, y1)
    dxs, dys, dAs, dgx = _bwd_outputs(b)
    b.backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx)
    torch.cuda.synchronize()
    _check_streamed(b, xs, ys, As, gx, dot_g, gdy, d1, y1, dxs, dys, dAs, dgx)
    del As, dAs
    torch.cuda.empty_cache()


def _check_streamed(b, xs, ys, As, gx, dot_g, gdy, dot_out, gy, dxs, dys, dAs, dgx):
    hx, hy, hg, hgx, hdy = host(xs), host(ys), host(dot_g), host(gx), host(gdy)
    hdot, hgy, hdxs, hdys, hdgx = host(dot_out), host(gy), host(dxs), host(dys), host(dgx)
    for i in range(len(b.dot_lengths)):
        o, n = b.dot_offs[i], b.dot_lengths[i]
        assert_bits_equal(np.float32(hdot[i]), loopnest.dot_f32(hx[o:o + n], hy[o:o + n],
                                                                 oracle_strategy(b.dot_st[i])), f"dot {i}")
        wx, wy = loopnest.dot_bwd_f32(hx[o:o + n], hy[o:o + n], hg[i])
        assert_bits_equal(hdxs[o:o + n], wx, f"dot {i} dx")
        assert_bits_equal(hdys[o:o + n], wy, f"dot {i} dy")
    for i in range(len(b.gemv_shapes)):
        M, N_ = b.gemv_shapes[i]
        A = host(b.a_view(As, i)).copy()
        x, dy = hgx[b.gx_offs[i]:b.gx_offs[i] + N_], hdy[b.gy_offs[i]:b.gy_offs[i] + M]
        assert_bits_equal(hgy[b.gy_offs[i]:b.gy_offs[i] + M], loopnest.gemv_f32(A, x, oracle_strategy(b.gemv_st[i])),
                          f"gemv {i}")
        assert_bits_equal(hdgx[b.gx_offs[i]:b.gx_offs[i] + N_], loopnest.gemv_bwd_dx_f32(A, dy, b.policy.row_split),
                          f"gemv {i} dx")
        del A
        assert_bits_equal(host(b.a_view(dAs, i)).copy(), loopnest.gemv_bwd_dA_f32(x, dy), f"gemv {i} dA")
