"""Autotuner: choose split sizes and levels by timing candidate strategies.

This stands in for the paper's strategy search (Section 2.1 cites a
rewrite-based exploration of strategies): here the search space is the
strategy descriptor itself (split, threads, vec, levels, second level), every
candidate is run through the C ABI on the caller's data, timed with CUDA events
on the launching stream, and the fastest is kept. Results are cached in a JSON
file keyed by (op, size, device name).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import ops
from .strategy import ReduceStrategy

CACHE_PATH = os.environ.get("DPIA_TUNE_CACHE",
                            os.path.join(os.path.expanduser("~"), ".cache", "dpia_tune.json"))
_lock = threading.Lock()


def reduce_candidates(n: int, splits=(1024, 2048, 4096, 8192, 16384, 32768, 65536)):
    """Block-per-chunk strategies over a split sweep, plus warp-per-chunk ones."""
    out = []
    for s in splits:
        for T in (256, 512, 1024):
            if s % (T * 4) != 0:
                continue
            for second, T2 in (("tree", min(T, 1024)),):
                out.append(ReduceStrategy(split=s, threads=T, vec=4, second=second, threads2=T2,
                                          pad=n % s != 0))
        if s % 128 == 0 and s <= 8192:
            out.append(ReduceStrategy(split=s, threads=256, vec=4, map_level="warp", second="tree",
                                      threads2=256, pad=n % s != 0))
    return out


def time_call(fn, reps: int = 20, warmup: int = 3, stream=None) -> float:
    """Median milliseconds of fn() over reps, CUDA events on the stream."""
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def _load():
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    try:
        os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)
    except OSError:
        pass


def tune_reduce(op: str, x, y=None, candidates=None, reps: int = 10, use_cache: bool = True):
    """Fastest strategy for ``op`` in {"dot", "asum"} on these inputs.

    Returns (strategy, {repr(strategy): ms}).
    """
    n = x.numel()
    key = f"{op}/{n}/{torch.cuda.get_device_name(x.device)}"
    if use_cache:
        with _lock:
            hit = _load().get(key)
        if hit:
            return ReduceStrategy(**hit["strategy"]), hit.get("timings", {})
    cands = candidates or reduce_candidates(n)
    out = torch.empty(1, dtype=torch.float32, device=x.device)
    timings = {}
    best, best_ms = None, float("inf")
    for st in cands:
        ws = ops.workspace(ops.dpia_dot_workspace_size(n, st), x.device)
        if op == "dot":
            fn = lambda: ops.dpia_dot_f32(x, y, n, st, out, ws)
        else:
            fn = lambda: ops.dpia_asum_f32(x, n, st, out, ws)
        ms = time_call(fn, reps=reps)
        timings[_label(st)] = ms
        if ms < best_ms:
            best, best_ms = st, ms
    if use_cache:
        with _lock:
            d = _load()
            d[key] = {"strategy": best.as_dict(), "timings": timings}
            _save(d)
    return best, timings


def _label(st: ReduceStrategy) -> str:
    return (f"{st.map_level}:s{st.split}:T{st.threads}:V{st.vec}:{st.second}"
            f"{st.threads2 if st.second == 'tree' else ''}")
