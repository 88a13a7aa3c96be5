"""The autotuner picks a strategy it timed, from legal candidates, and caches it."""
import json

import pytest
import torch

import paper_1710_08332_gb300 as dpia
from paper_1710_08332_gb300 import tune

pytestmark = pytest.mark.gpu


def test_tune_reduce_and_cache(cuda_device, tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "tune.json"))
    x = torch.rand(1 << 22, device="cuda")
    y = torch.rand(1 << 22, device="cuda")
    cands = tune.reduce_candidates(x.numel(), splits=(4096, 16384))
    best, timings = tune.tune_reduce("dot", x, y, candidates=cands, reps=3)
    assert best in cands and len(timings) == len(cands)
    assert all(v > 0 for v in timings.values())
    cached = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("dot/4194304/") for k in cached)
    again, _ = tune.tune_reduce("dot", x, y, candidates=cands, reps=3)
    assert again == best
    # the tuned strategy computes the same bits as any evaluation of its own tree
    got = dpia.dot(x, y, best)
    assert torch.isfinite(got)


def test_tune_gemm_bf16_and_cache(cuda_device, tmp_path, monkeypatch):
    """The GEMM tuner times every tile choice on the shape, keeps one of them,
    caches it per shape and layout, and the choice computes C like the default."""
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "tune.json"))
    M, N, K = 1024, 768, 512
    cands = tune.gemm_bf16_candidates(M)
    assert (1, 0, 0) in cands and (2, 512, 224) in cands
    best, timings = tune.tune_gemm_bf16(M, N, K, transB=1, reps=2)
    assert best in [tuple(c) for c in cands] and len(timings) == len(cands)
    assert all(v > 0 for v in timings.values())
    cached = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("gemm_bf16/1024x768x512/t01/") for k in cached)
    again, _ = tune.tune_gemm_bf16(M, N, K, transB=1, reps=2)
    assert again == best
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    C0 = torch.empty(M, N, device="cuda")
    C1 = torch.empty(M, N, device="cuda")
    dpia.dpia_gemm_bf16(A, B, C0, M, N, K, K, K, N, 0, 1)
    cl, tm, tn = best
    dpia.dpia_gemm_bf16(A, B, C1, M, N, K, K, K, N, 0, 1, cluster=cl, tile_m=tm, tile_n=tn)
    torch.cuda.synchronize()
    ref = (A.float() @ B.float().T)
    for C in (C0, C1):
        assert ((C - ref).norm() / ref.norm()).item() <= 1e-4
