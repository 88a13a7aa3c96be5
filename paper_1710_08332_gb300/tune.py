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
    """Block-per-chunk strategies over a split sweep (direct loads, and chunks
    staged through shared memory), plus warp-per-chunk ones."""
    out = []
    for s in splits:
        for T in (256, 512, 1024):
            if s % (T * 4) != 0:
                continue
            for second, T2 in (("tree", min(T, 1024)),):
                out.append(ReduceStrategy(split=s, threads=T, vec=4, second=second, threads2=T2,
                                          pad=n % s != 0))
                if T <= 512:  # the same chunks staged through shared memory (toLocal)
                    out.append(ReduceStrategy(split=s, threads=T, vec=4, second=second, threads2=T2,
                                              pad=n % s != 0, stage="local"))
        if s % 128 == 0 and s <= 8192:
            out.append(ReduceStrategy(split=s, threads=256, vec=4, map_level="warp", second="tree",
                                      threads2=256, pad=n % s != 0))
    return out


def hold_device(stream, us: float) -> None:
    """Queue a device-side delay of about ``us`` microseconds on the stream, so
    that the host can enqueue the calls that follow before the device reaches
    them (an event pair then times the kernel, not the host's launch latency)."""
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(us * 2500))  # cycles; >= us at clocks up to 2.5 GHz


def time_call(fn, reps: int = 20, warmup: int = 3, stream=None, inner: int | None = None) -> float:
    """Median milliseconds of one fn() call, CUDA events on the stream.

    Each of the reps samples times ``inner`` back-to-back calls (chosen so that
    a sample spans about 0.3 ms: the event clock ticks in steps of about 2 us)
    and divides; all samples are enqueued behind a device-side delay, so the
    host's launch latency is not timed, then synchronised once."""
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    stream.synchronize()
    if inner is None:
        hold_device(stream, 200.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(4):
            fn()
        b.record(stream)
        b.synchronize()
        est = max(a.elapsed_time(b) / 4, 1e-4)
        inner = int(min(64, max(1, round(0.3 / est))))
    hold_device(stream, min(50.0 * reps * inner, 200000.0))
    ev = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(inner):
            fn()
        b.record(stream)
        ev.append((a, b))
    stream.synchronize()
    times = sorted(a.elapsed_time(b) / inner for a, b in ev)
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


def gemm_bf16_candidates(M: int):
    """(cluster, tile_m, tile_n) choices of the BF16 GEMM: one CTA per 256-row
    tile or a CTA pair per 256- or 512-row tile, each with the width picked
    per shape (tile_n 0) or a fixed width."""
    widths = (0, 128, 192, 224, 256)
    cands = [(1, 0, w) for w in widths] + [(2, 256, w) for w in widths]
    if M > 256:
        cands += [(2, 512, w) for w in widths]
    return cands


def tune_gemm_bf16(M: int, N: int, K: int, transA: int = 0, transB: int = 0, candidates=None,
                   reps: int = 5, use_cache: bool = True, device="cuda"):
    """Fastest (cluster, tile_m, tile_n) of dpia_gemm_bf16 for this shape and
    operand layout, timed on random bf16 operands (L2 warm; the choice only
    moves work between SMs, never the value of C).

    Returns ((cluster, tile_m, tile_n), {label: ms}); pass the first as the
    keyword arguments cluster=, tile_m=, tile_n= of ops.dpia_gemm_bf16.
    """
    dev = torch.device(device)
    key = f"gemm_bf16/{M}x{N}x{K}/t{transA}{transB}/{torch.cuda.get_device_name(dev)}"
    if use_cache:
        with _lock:
            hit = _load().get(key)
        if hit:
            return tuple(hit["choice"]), hit.get("timings", {})
    g = torch.Generator(device=dev).manual_seed(0)
    pad8 = lambda v: (v + 7) // 8 * 8  # TMA wants rows 16 bytes apart
    ra, ca = (K, M) if transA else (M, K)
    rb, cb = (N, K) if transB else (K, N)
    A = torch.randn(ra, pad8(ca), generator=g, device=dev).to(torch.bfloat16)
    B = torch.randn(rb, pad8(cb), generator=g, device=dev).to(torch.bfloat16)
    C = torch.empty(M, N, device=dev)
    lda, ldb = A.shape[1], B.shape[1]
    timings = {}
    best, best_ms = None, float("inf")
    for cl, tm, tn in candidates or gemm_bf16_candidates(M):
        fn = lambda: ops.dpia_gemm_bf16(A, B, C, M, N, K, lda, ldb, N, transA, transB, tile_n=tn, cluster=cl,
                                        tile_m=tm)
        ms = time_call(fn, reps=reps)
        timings[f"cluster{cl}:m{tm or 256}:n{tn or 'auto'}"] = ms
        if ms < best_ms:
            best, best_ms = (cl, tm, tn), ms
    if use_cache:
        with _lock:
            d = _load()
            d[key] = {"choice": list(best), "timings": timings}
            _save(d)
    return best, timings


def _label(st: ReduceStrategy) -> str:
    return (f"{st.map_level}:s{st.split}:T{st.threads}:V{st.vec}:{st.second}"
            f"{st.threads2 if st.second == 'tree' else ''}{':local' if st.stage == 'local' else ''}")


def batch_candidates():
    """Policies the batch autotuner tries (block size, dot split cap, GEMV row
    split cap, backward row split)."""
    from .batch import BatchPolicy

    out = [BatchPolicy(threads=256, dot_split_cap=8192, row_split=128, schedule=1)]
    for T, cap, rs in ((256, 8192, 128), (128, 8192, 128), (256, 16384, 256), (256, 4096, 64), (256, 8192, 512)):
        out.append(BatchPolicy(threads=T, dot_split_cap=cap, row_split=rs))
    for rs in (256, 512):  # items taken from a counter by whichever block or warp is free
        out.append(BatchPolicy(threads=256, dot_split_cap=8192, row_split=rs, schedule=2))
    return out


def tune_batch(dot_lengths, gemv_shapes, make_inputs, candidates=None, reps: int = 3):
    """Fastest policy for a batch: each candidate is planned and its forward and
    backward launches are timed on the data make_inputs(batch) returns
    (xs, ys, As, gx, dot_g, gdy). Returns (Batch, {label: ms})."""
    from .batch import Batch

    timings, best, best_ms = {}, None, float("inf")
    for pol in candidates or batch_candidates():
        b = Batch(dot_lengths, gemv_shapes, policy=pol)
        xs, ys, As, gx, dot_g, gdy = make_inputs(b)
        dot_out = torch.empty(max(len(dot_lengths), 1), device=b.device)
        gy = torch.empty(b.gy_len, device=b.device)
        dxs, dys = torch.empty_like(xs), torch.empty_like(ys)
        dAs, dgx = torch.empty_like(As), torch.empty_like(gx)
        ms = time_call(lambda: (b.forward(xs, ys, dot_out, As, gx, gy),
                                b.backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx)), reps=reps, warmup=1)
        label = f"T{pol.threads}:dotcap{pol.dot_split_cap}:rs{pol.row_split}:sched{pol.schedule}"
        timings[label] = ms
        del xs, ys, As, gx, dot_g, gdy, dxs, dys, dAs, dgx
        if ms < best_ms:
            best, best_ms = pol, ms
        torch.cuda.empty_cache()
    return Batch(dot_lengths, gemv_shapes, policy=best), timings
