"""Benchmark of the strategy-preserving map/reduce hot path on GB300.

Default workload (one step): the bandwidth set at n = 2^26 float32 (256 MiB
per vector), inputs x, y ~ U[-1, 1) from seed 1:
    asum(x)  -- one strategy reduction, 256 MiB read
    scal(1.5, x) -> y'  -- a map, 256 MiB read + 256 MiB write
    dot(x, y)  -- one strategy reduction, 512 MiB read
Split sizes are chosen per op by the autotuner from the sweep 1024..65536
(untimed, before warm-up); the sweep table is printed in the JSON line.

Prints ONE JSON line: value = algorithmic bytes of the step / device time of
the step (GB/s), whole job over all ranks. Other workloads (``--workload
dot|gemv|gemm|batched``) print their own line with their own metric.

``--impl reference`` times the CPU oracle (the paper has no runnable
reference; the oracle is the plain CPU evaluation of the same strategy trees)
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILES = os.path.join(ROOT, "profiles")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
METRIC = "HBM GB/s (dot/asum/GEMV) and TFLOP/s (GEMM) vs GB300 roofline; batched vs per-launch"


# ---------------------------------------------------------------------------
# process group (one rank per GPU; replicas of the workload)
# ---------------------------------------------------------------------------


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend: str):
    import torch.distributed as dist

    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def reduce_max(dist, value: float, device=None) -> float:
    """Max of a float over ranks (identity with one rank)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# peaks, clocks, profiles
# ---------------------------------------------------------------------------


def max_sm_mhz(clk=None) -> float:
    """The maximum SM clock: from the sampled clocks, else MEASURED_PEAKS.json, else 2070 MHz."""
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"])
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f).get("sm_max_mhz") or 2070.0)
    except (OSError, ValueError):
        return 2070.0


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return d.get("hbm_gbs", FALLBACK_HBM_GBS), d.get("bf16_tflops", FALLBACK_BF16_TFLOPS), \
            d.get("bf16_tflops_sustained"), "measured"
    except (OSError, ValueError):
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile

        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()  # nvidia-smi takes a moment to start: wait for its first sample (at most 3 s)
        while self.count() < 1 and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.02)

    def count(self) -> int:
        """Samples written so far."""
        if self.proc is None or not self.path:
            return 0
        try:
            with open(self.path) as f:
                return sum(1 for line in f if line.count(",") >= 8)
        except OSError:
            return 0

    def warm(self, step, min_samples: int = 3, max_s: float = 2.0):
        """Run more untimed warm-up steps until min_samples samples were taken
        since now (at most max_s seconds), so the clock record covers the GPU
        under this workload's load and not only its idle start."""
        if self.proc is None:
            return
        import torch

        target, t0 = self.count() + min_samples, time.time()
        while self.count() < target and time.time() - t0 < max_s:
            step()
            torch.cuda.synchronize()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        load = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "window": "warm-up (extended until three samples were taken under load) + timed steps"}


def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(summary: str, sources, key="traffic_bytes_per_launch"):
    """Per-launch DRAM bytes (or another figure named by key) recorded in a
    profiles/ summary, if it was taken on the current kernel sources (its
    'source_digest' matches); else None."""
    path = os.path.join(PROFILES, summary)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.eE+]+)", text)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    want = sources if isinstance(sources, str) else source_digest(sources)
    if not m or not d or d.group(1) != want:
        return None
    return float(m.group(1))


REDUCE_SOURCES = ["paper_1710_08332_gb300/csrc/k_reduce.cu", "paper_1710_08332_gb300/csrc/device_common.cuh"]
GEMV_SOURCES = ["paper_1710_08332_gb300/csrc/k_gemv.cu", "paper_1710_08332_gb300/csrc/device_common.cuh",
                "paper_1710_08332_gb300/csrc/k_maps.cu"]
GEMM_SOURCES = ["paper_1710_08332_gb300/csrc/k_gemm_bf16.cu"]
BATCH_SOURCES = ["paper_1710_08332_gb300/csrc/k_batched.cu", "paper_1710_08332_gb300/csrc/device_common.cuh",
                 "paper_1710_08332_gb300/batch.py"]  # the kernels and the packer's layout


def generated_dot_R_digest() -> str:
    """Digest of the generated one-kernel dot as profiled (n = 2^25, split 16384,
    256 threads, float4, tree 256, unrolled 4): the emitted kernel source
    without the shared helper prelude, so that only a change to this kernel's
    own code makes the recorded counters stale."""
    from paper_1710_08332_gb300.codegen import emit as E
    from paper_1710_08332_gb300.codegen import programs as PR

    n = 1 << 25
    g = E.generate(f"gen_dot_R_s16384_T256_n{n}", *PR.dot_R(n, 16384, 256, 4, "interleaved", "tree", 256), "cuda",
                   unroll=4)
    return hashlib.sha256(g["source"].replace(E.CUDA_PRELUDE, "").encode()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# timing helpers
# ---------------------------------------------------------------------------


class Timeline:
    """CUDA events around each kernel call of each step, on the launch stream."""

    def __init__(self, names, stream):
        import torch

        self.torch = torch
        self.stream = stream
        self.names = names
        self.events = {n: [] for n in names}

    def call(self, name, fn):
        E = self.torch.cuda.Event
        a, b = E(enable_timing=True), E(enable_timing=True)
        a.record(self.stream)
        fn()
        b.record(self.stream)
        self.events[name].append((a, b))

    def avg_ms(self, name):
        ev = self.events[name]
        return sum(a.elapsed_time(b) for a, b in ev) / max(len(ev), 1)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------


def _default_bw_strategy():
    from paper_1710_08332_gb300.strategy import ReduceStrategy

    return ReduceStrategy(split=16384, threads=256, vec=4, second="tree", threads2=256)


DEFAULT_BW_STRATEGY = None  # set in main() after the package is importable


def profile_case(args):
    """A small case of one kernel, launched args.reps times after one warm-up."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from synth import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = _default_bw_strategy()
    n = args.n
    if args.profile in ("dot", "asum", "scal", "dot_local", "asum_local"):
        x, y = W.bandwidth(dev, n=n)
        out = torch.empty(1, device=dev)
        st = st.with_(pad=n % st.split != 0,
                      stage="local" if args.profile.endswith("_local") else "private")
        ws = torch.zeros(dpia.dpia_dot_workspace_size(n, st), dtype=torch.uint8, device=dev)
        ys = torch.empty_like(x)
        fn = {"dot": lambda: dpia.dpia_dot_f32(x, y, n, st, out, ws),
              "asum": lambda: dpia.dpia_asum_f32(x, n, st, out, ws),
              "scal": lambda: dpia.dpia_scal_f32(W.SCAL_A, x, ys, n, 4)}[args.profile.split("_")[0]]
    elif args.profile == "dot1m":  # the n = 2^20 dot: split 8192, 128 chunks, sequential second level
        x, y = W.dot_f32(dev)
        n = x.numel()
        st = dpia.ReduceStrategy(split=W.DOT_SPLIT, threads=256, vec=4)
        out = torch.empty(1, device=dev)
        ws = torch.zeros(dpia.dpia_dot_workspace_size(n, st), dtype=torch.uint8, device=dev)

        def fn():
            dpia.dpia_dot_f32(x, y, n, st, out, ws)
    elif args.profile == "gemv":  # GEMV 8192 x 8192 forward, dx, dA
        A, xv, dy = W.gemv(dev)
        M, N_ = A.shape
        st = dpia.ReduceStrategy(split=N_, threads=128, vec=4)
        yv = torch.empty(M, device=dev)
        dx = torch.empty(N_, device=dev)
        dA = torch.empty(M, N_, device=dev)
        ws = torch.zeros(dpia.dpia_gemv_bwd_workspace_size(M, N_, 256), dtype=torch.uint8, device=dev)

        def fn():
            dpia.dpia_gemv_f32(A, M, N_, N_, xv, yv, st)
            dpia.dpia_gemv_bwd_f32(A, M, N_, N_, xv, dy, dx, None, N_, 256, ws)
            dpia.dpia_gemv_bwd_f32(A, M, N_, N_, xv, dy, None, dA, N_, 256, ws)
    elif args.profile == "gemm":
        m = args.n
        A, B, _ = W.gemm(dev, M=m, N=m, K=m)
        Ab, Bb = dpia.to_bf16(A), dpia.to_bf16(B)
        C = torch.empty(m, m, device=dev)

        def fn():
            dpia.dpia_gemm_bf16(Ab, Bb, C, m, m, m, m, m, m, 0, 0, cluster=args.cluster, tile_m=args.tile_m)
            dpia.dpia_gemm_f32(A, B, C, m, m, m, m, m, m, 0, 0, "fma", schedule=args.schedule)
    elif args.profile == "batched":  # the first 512 dots and 16 GEMVs of the batched workload
        import math

        from paper_1710_08332_gb300.batch import Batch

        dl, rows, cols = W.batched_shapes()
        from paper_1710_08332_gb300.batch import BatchPolicy

        # the policy the autotuner picks on the whole batch: backward items taken by free warps
        b = Batch(dl.tolist()[:512], list(zip(rows.tolist()[:16], cols.tolist()[:16])), dev,
                  policy=BatchPolicy(row_split=256, schedule=2))
        xs = torch.rand(b.xs_len, device=dev)
        ys = torch.rand(b.xs_len, device=dev)
        As = torch.randn(b.as_len, device=dev)
        gx = torch.rand(b.gx_len, device=dev)
        dot_g = torch.rand(len(b.dot_lengths), device=dev)
        gdy = torch.rand(b.gy_len, device=dev)
        dot_out, gy = torch.empty(len(b.dot_lengths), device=dev), torch.empty(b.gy_len, device=dev)
        dxs, dys, dAs, dgx = torch.empty_like(xs), torch.empty_like(ys), torch.empty_like(As), torch.empty_like(gx)

        def fn():
            b.forward(xs, ys, dot_out, As, gx, gy)
            b.backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx)
        n_dot = int(sum(b.dot_lengths))
        mn = int(sum(m * k for m, k in zip(rows.tolist()[:16], cols.tolist()[:16])))
        print(f"algorithmic bytes: forward {8 * n_dot + 4 * mn}, backward {16 * n_dot + 8 * mn}", flush=True)
    elif args.profile == "gen_dot":  # the generated dot partials kernel (asVector 4, split 2^15, 256 threads)
        from paper_1710_08332_gb300 import codegen as G
        from paper_1710_08332_gb300.codegen import programs as PR

        x, y = W.bandwidth(dev, n=n)
        k = G.compile_cuda("gen_dot_partials", *PR.dot_partials(n, 1 << 15, 256, V=4), unroll=4)
        part = torch.empty(n // (1 << 15) * 256 * 4, device=dev)

        def fn():
            k.run(x, y, part)
    elif args.profile == "gen_dot_R":  # the generated one-kernel dot (split 16384, 256 threads, float4, tree 256)
        from paper_1710_08332_gb300 import codegen as G
        from paper_1710_08332_gb300.codegen import programs as PR

        x, y = W.bandwidth(dev, n=n)
        k = G.compile_cuda(f"gen_dot_R_s16384_T256_n{n}", *PR.dot_R(n, 16384, 256, 4, "interleaved", "tree",
                                                                   min(256, n // 16384)), unroll=4)
        out1 = torch.empty(1, device=dev)
        temps = k.temps_like(dev)

        def fn():
            k.run(x, y, out1, *temps)
    else:
        raise SystemExit(f"unknown profile case {args.profile}")
    for _ in range(1 + args.reps):
        fn()
    torch.cuda.synchronize()
    print(f"profile case {args.profile} n={n} reps={args.reps} done", flush=True)
    return 0


PROFILE_CASES = {"dot", "asum", "scal", "dot_local", "asum_local", "gemm", "batched", "dot1m", "gemv", "gen_dot",
                 "gen_dot_R"}


def bandwidth_workload(args, device, dist):
    import torch

    import paper_1710_08332_gb300 as dpia
    from paper_1710_08332_gb300 import tune
    from synth import workloads as W

    n = W.BW_N
    x, y = W.bandwidth(device)
    ys = torch.empty_like(x)
    out_a = torch.empty(1, device=device)
    out_d = torch.empty(1, device=device)
    stream = torch.cuda.current_stream(device)

    # autotune split sizes (untimed)
    if args.no_tune:
        st_dot = st_asum = DEFAULT_BW_STRATEGY
        sweep_dot = sweep_asum = {}
    else:
        st_dot, sweep_dot = tune.tune_reduce("dot", x, y, reps=5, use_cache=False)
        st_asum, sweep_asum = tune.tune_reduce("asum", x, reps=5, use_cache=False)
    ws_d = dpia.workspace(dpia.dpia_dot_workspace_size(n, st_dot), device)
    ws_a = torch.zeros(dpia.dpia_dot_workspace_size(n, st_asum), dtype=torch.uint8, device=device)

    B_ASUM, B_SCAL, B_DOT = 4 * n, 8 * n, 8 * n
    step_bytes = B_ASUM + B_SCAL + B_DOT

    def step(tl=None):
        calls = (("scal", lambda: dpia.dpia_scal_f32(W.SCAL_A, x, ys, n, 4)),
                 ("asum", lambda: dpia.dpia_asum_f32(x, n, st_asum, out_a, ws_a)),
                 ("dot", lambda: dpia.dpia_dot_f32(x, y, n, st_dot, out_d, ws_d)))
        for name, fn in calls:
            if tl is None:
                fn()
            else:
                tl.call(name, fn)

    clocks = ClockSampler(device.index)
    clocks.start()
    for _ in range(args.warmup):
        step()
    clocks.warm(step)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    tl = Timeline(["scal", "asum", "dot"], stream)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    tune.hold_device(stream, 200.0 * args.steps)  # the host enqueues ahead of the device
    t0.record(stream)
    for _ in range(args.steps):
        step(tl)
    t1.record(stream)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    ms_total = t0.elapsed_time(t1)
    ms_total_max = reduce_max(dist, ms_total, device if dist and dist.get_backend() == "nccl" else None)
    ms_step = ms_total_max / args.steps

    kern = {}
    for name, b in (("asum", B_ASUM), ("scal", B_SCAL), ("dot", B_DOT)):
        ms = tl.avg_ms(name)
        kern[name] = {"avg_us": round(ms * 1e3, 2), "algorithmic_bytes": b, "GB_s": round(b / ms / 1e6, 1)}

    # the compensated (Kahan) variants of the two reductions, same strategies,
    # timed after the step (not part of it)
    variants = {}
    for name, b, fn in (
            ("dot_compensated", B_DOT, lambda st: dpia.dpia_dot_f32(x, y, n, st, out_d, ws_d)),
            ("asum_compensated", B_ASUM, lambda st: dpia.dpia_asum_f32(x, n, st, out_a, ws_a))):
        base = st_dot if name.startswith("dot") else st_asum
        stk = base.with_(compensated=True)
        need = dpia.dpia_dot_workspace_size(n, stk)
        if need > (ws_d.numel() if name.startswith("dot") else ws_a.numel()):
            continue
        ms = tune.time_call(lambda: fn(stk), reps=20, warmup=3)
        ms0 = tune.time_call(lambda: fn(base), reps=20, warmup=3)
        variants[name] = {"avg_us": round(ms * 1e3, 2), "GB_s": round(b / ms / 1e6, 1),
                          "plain_avg_us": round(ms0 * 1e3, 2), "time_ratio": round(ms / ms0, 3)}

    alone = standalone_us({"scal": lambda: dpia.dpia_scal_f32(W.SCAL_A, x, ys, n, 4),
                           "asum": lambda: dpia.dpia_asum_f32(x, n, st_asum, out_a, ws_a),
                           "dot": lambda: dpia.dpia_dot_f32(x, y, n, st_dot, out_d, ws_d)},
                          {"scal": B_SCAL, "asum": B_ASUM, "dot": B_DOT})

    # end to end: pinned host inputs -> device, the three calls, results -> host
    e2e = e2e_bandwidth(args, device, dist, st_dot, st_asum, x.cpu(), y.cpu(), step_bytes)

    hbm, _, _, src = peaks()
    dot_ms = tl.avg_ms("dot")
    achieved = B_DOT / dot_ms / 1e6
    traffic = profile_traffic("reduce_dot_bandwidth_n2e26.md", REDUCE_SOURCES)
    world = dist.get_world_size() if dist else 1
    line = {
        "metric": METRIC,
        "value": round(world * step_bytes / (ms_step / 1e3) / 1e9, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "bandwidth set: asum + scal(a=1.5) + dot, n=2^26 f32 (256 MiB per vector), "
                               "U[-1,1) seed 1, autotuned split (sweep 1024..65536)",
                   "n": n, "split_dot": st_dot.split, "split_asum": st_asum.split,
                   "strategy_dot": st_dot.as_dict(), "strategy_asum": st_asum.as_dict(),
                   "l2": "inputs larger than L2 (256 MiB per vector > 129 MB)",
                   "parallelism": f"replicas x{world}"},
        "kernels": kern,
        "kernels_alone": alone,
        "kernels_note": "in a step, asum follows scal and pays for writing back the dirty lines of scal's "
                        "256 MiB of stores still in L2; kernels_alone times each kernel by itself",
        "variants": variants,
        "split_sweep_dot_ms": sweep_dot,
        "split_sweep_asum_ms": sweep_asum,
        "roofline": {"bound": "hbm", "kernel": "reduce_kernel<DotF32,SumF32,V=4,Block> (dpia_dot_f32)",
                     "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": traffic,
                     "peak_source": f"{src} hbm_gbs (copy, burst)",
                     "algorithmic_bytes_per_launch": B_DOT},
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    return line


class L2Flush:
    """Reads a buffer larger than L2 (256 MiB) between timed steps, leaving L2
    full of clean lines (a write would leave dirty lines for the next kernel
    to write back)."""

    def __init__(self, device):
        import torch

        self.buf = torch.ones(64 << 20, dtype=torch.float32, device=device)

    def __call__(self):
        self.buf.sum()


def timed_steps(args, device, dist, names, step, flush=None):
    """W warm-up steps, then K timed steps with CUDA events around every kernel
    call (flush, if given, runs before each step outside the events). Returns
    (per-kernel avg ms, per-step kernel ms max over ranks, clocks)."""
    import torch

    from paper_1710_08332_gb300 import tune

    stream = torch.cuda.current_stream(device)
    clocks = ClockSampler(device.index)
    clocks.start()
    for _ in range(args.warmup):
        if flush:
            flush()
        step(None)
    clocks.warm(lambda: (flush() if flush else None, step(None)))
    torch.cuda.synchronize(device)
    barrier(dist, device)
    tl = Timeline(names, stream)
    # a device-side delay lets the host enqueue the steps ahead of the device,
    # so each event pair times its kernel and not the host's launch latency
    tune.hold_device(stream, 200.0 * args.steps)
    for _ in range(args.steps):
        if flush:
            flush()
        step(tl)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    clk = clocks.stop()
    per = {n: tl.avg_ms(n) for n in names}
    step_ms = reduce_max(dist, sum(per.values()), device if dist and dist.get_backend() == "nccl" else None)
    return per, step_ms, clk


def standalone_us(calls, bytes_, flush=None, reps: int = 20):
    """Each call timed alone (median over reps of back-to-back launches of the
    same kernel, events on the launch stream, the host enqueuing ahead of the
    device; with a flush, one launch per event pair and the flush before it,
    outside the events). In a step
    a kernel also pays for write-backs of the dirty lines its predecessor left
    in L2; alone it does not."""
    import torch

    from paper_1710_08332_gb300 import tune

    stream = torch.cuda.current_stream()
    out = {}
    for name, fn in calls.items():
        if flush is None:  # back-to-back launches, several per event pair
            t = tune.time_call(fn, reps=reps, stream=stream)
        else:
            for _ in range(3):
                fn()
            stream.synchronize()
            tune.hold_device(stream, 200.0 * reps)
            ev = []
            for _ in range(reps):
                flush()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                ev.append((a, b))
            stream.synchronize()
            t = sorted(a.elapsed_time(b) for a, b in ev)[reps // 2]
        out[name] = {"median_us": round(t * 1e3, 2)}
        if bytes_.get(name):
            out[name]["GB_s"] = round(bytes_[name] / t / 1e6, 1)
    return out


def _line(args, dist, metric_value, unit, step_ms, dtype, config, kernels, roofline, clk, launches, extra=None):
    world = dist.get_world_size() if dist else 1
    d = {"metric": METRIC, "value": metric_value, "unit": unit, "n_gpus": world, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config, "kernels": kernels,
         "roofline": roofline, "gpu_launches": launches, "clocks": clk}
    if extra:
        d.update(extra)
    return d


def dot_workload(args, device, dist):
    """n = 2^20 dot, split 8192 (128 chunks), block per chunk, sequential second
    level over the 128 partials; f32 and int32. The inputs (8 MiB) fit in L2,
    so L2 is flushed before every step, outside the kernel events."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from synth import workloads as W

    from paper_1710_08332_gb300 import tune

    x, y = W.dot_f32(device)
    xi, yi = W.dot_i32(device)
    n = x.numel()
    # the workload fixes split 8192 (128 chunks), a block per chunk and the
    # sequential second level; the block size and vector width are tuned under
    # the timed conditions (L2 flushed before every launch)
    flush = L2Flush(device)
    cands = [dpia.ReduceStrategy(split=W.DOT_SPLIT, threads=T, vec=V)
             for T in (256, 512, 1024) for V in (4, 8) if T * V <= W.DOT_SPLIT and not (V == 8 and T > 512)]
    out = torch.empty(1, device=device)
    sweep = {}
    for c in cands:
        wsc = torch.zeros(dpia.dpia_dot_workspace_size(n, c), dtype=torch.uint8, device=device)
        t = standalone_us({"c": lambda: dpia.dpia_dot_f32(x, y, n, c, out, wsc)}, {}, flush=flush, reps=15)
        sweep[tune._label(c)] = t["c"]["median_us"]
    st = cands[min(range(len(cands)), key=lambda i: sweep[tune._label(cands[i])])]
    ws = torch.zeros(dpia.dpia_dot_workspace_size(n, st), dtype=torch.uint8, device=device)
    wsi = torch.zeros_like(ws)
    outi = torch.empty(1, dtype=torch.int64, device=device)

    def step(tl):
        calls = (("dot_f32", lambda: dpia.dpia_dot_f32(x, y, n, st, out, ws)),
                 ("dot_i32", lambda: dpia.dpia_dot_i32(xi, yi, n, st, outi, wsi)))
        for name, fn in calls:
            fn() if tl is None else tl.call(name, fn)

    per, step_ms, clk = timed_steps(args, device, dist, ["dot_f32", "dot_i32"], step, flush)
    hbm = peaks()[0]
    b = 8 * n
    # context on the same flushed inputs: the library dot (cuBLAS through
    # torch.dot) and the event-to-event time of a launch that does no work
    tiny = torch.zeros(4, device=device)
    context = standalone_us({"dpia_dot_f32": lambda: dpia.dpia_dot_f32(x, y, n, st, out, ws),
                             "torch_dot_cublas": lambda: torch.dot(x, y),
                             "empty_launch_floor": lambda: dpia.dpia_scal_f32(1.0, tiny, tiny, 4)},
                            {"dpia_dot_f32": b, "torch_dot_cublas": b}, flush=flush)
    kern = {k: {"avg_us": round(v * 1e3, 2), "algorithmic_bytes": b, "GB_s": round(b / v / 1e6, 1)}
            for k, v in per.items()}
    achieved = b / per["dot_f32"] / 1e6
    world = dist.get_world_size() if dist else 1
    roof = {"bound": "hbm", "kernel": "reduce_kernel<DotF32,SumF32,V=4,Block> (dpia_dot_f32)",
            "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": None, "peak_source": "measured hbm_gbs (copy, burst)", "algorithmic_bytes_per_launch": b,
            "note": "8 MiB per launch (2^20 f32 pairs): the event-to-event time of an empty launch "
                    "(context.empty_launch_floor) is most of it"}
    cfg = {"workload": "dot f32 and int32, n=2^20, U[-1,1) / U{-100..100} seed 0, split 8192 (128 chunks), "
                       "block per chunk, sequential second level", "n": n, "strategy": st.as_dict(),
           "tuned_us_flushed": sweep,
           "l2": "flushed before every step (256 MiB read), outside the kernel events"}
    return _line(args, dist, round(world * 2 * b / (step_ms / 1e3) / 1e9, 1), "GB/s", step_ms, "f32",
                 cfg, kern, roof, clk, 2 * args.steps, {"context": context})


def gemv_workload(args, device, dist):
    """GEMV 8192 x 8192: forward y = A x, backward dx = A^T dy and dA = dy x^T."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from synth import workloads as W

    A, x, dy = W.gemv(device)
    M, N = A.shape
    st = dpia.ReduceStrategy(split=N, threads=128, vec=4)  # a block of 128 per row (best of the GEMV sweep)
    rs = 256
    y = torch.empty(M, device=device)
    dx = torch.empty(N, device=device)
    dA = torch.empty(M, N, device=device)
    ws = torch.zeros(dpia.dpia_gemv_bwd_workspace_size(M, N, rs), dtype=torch.uint8, device=device)

    def step(tl):
        calls = (("gemv_fwd", lambda: dpia.dpia_gemv_f32(A, M, N, N, x, y, st)),
                 ("gemv_bwd_dx", lambda: dpia.dpia_gemv_bwd_f32(A, M, N, N, x, dy, dx, None, N, rs, ws)),
                 ("gemv_bwd_dA", lambda: dpia.dpia_gemv_bwd_f32(A, M, N, N, x, dy, None, dA, N, rs, ws)))
        for name, fn in calls:
            fn() if tl is None else tl.call(name, fn)

    per, step_ms, clk = timed_steps(args, device, dist, ["gemv_fwd", "gemv_bwd_dx", "gemv_bwd_dA"], step)
    hbm = peaks()[0]
    bytes_ = {"gemv_fwd": 4 * M * N + 4 * N + 4 * M,
              "gemv_bwd_dx": 4 * M * N + 4 * M + 4 * N,
              "gemv_bwd_dA": 4 * M * N + 4 * M + 4 * N}
    alone = standalone_us({"gemv_fwd": lambda: dpia.dpia_gemv_f32(A, M, N, N, x, y, st),
                           "gemv_bwd_dx": lambda: dpia.dpia_gemv_bwd_f32(A, M, N, N, x, dy, dx, None, N, rs, ws),
                           "gemv_bwd_dA": lambda: dpia.dpia_gemv_bwd_f32(A, M, N, N, x, dy, None, dA, N, rs, ws)},
                          bytes_)
    kern = {k: {"avg_us": round(v * 1e3, 2), "algorithmic_bytes": bytes_[k], "GB_s": round(bytes_[k] / v / 1e6, 1)}
            for k, v in per.items()}
    achieved = bytes_["gemv_fwd"] / per["gemv_fwd"] / 1e6
    world = dist.get_world_size() if dist else 1
    roof = {"bound": "hbm", "kernel": "gemv_kernel<SumF32,V=4,Block> (dpia_gemv_f32)", "achieved": round(achieved, 1),
            "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": profile_traffic("gemv_8192.md", GEMV_SOURCES),
            "peak_source": "measured hbm_gbs (copy, burst)", "algorithmic_bytes_per_launch": bytes_["gemv_fwd"],
            "frac_alone": round(alone["gemv_fwd"]["GB_s"] / hbm, 4),
            "note": "achieved is the in-step time, which includes writing back the dirty lines of the previous "
                    "step's dA (256 MiB of stores) still in L2; frac_alone times the kernel by itself"}
    cfg = {"workload": "GEMV 8192x8192 f32, A ~ N(0,1/8192), x, dy ~ U[-1,1) seed 2: forward + backward (dx, dA)",
           "M": M, "N": N, "strategy": st.as_dict(), "row_split": rs,
           "l2": "inputs larger than L2 (A is 256 MiB)"}
    total = sum(bytes_.values())
    return _line(args, dist, round(world * total / (step_ms / 1e3) / 1e9, 1), "GB/s", step_ms, "f32", cfg, kern,
                 roof, clk, 3 * args.steps, {"kernels_alone": alone})


def gemm_workload(args, device, dist):
    """GEMM 4096^3: BF16 tensor-core forward C = A B and backward dA = dC B^T,
    dB = A^T dC (f32 accumulate), plus the FP32 CUDA-core fold forward."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from synth import workloads as W

    A, B, dC = W.gemm(device)
    n = A.shape[0]
    Ab, Bb, dCb = dpia.to_bf16(A), dpia.to_bf16(B), dpia.to_bf16(dC)
    C = torch.empty(n, n, device=device)
    gA = torch.empty(n, n, device=device)
    gB = torch.empty(n, n, device=device)
    Cf = torch.empty(n, n, device=device)

    def step(tl):
        calls = (("bf16_fwd", lambda: dpia.dpia_gemm_bf16(Ab, Bb, C, n, n, n, n, n, n, 0, 0)),
                 ("bf16_bwd_dA", lambda: dpia.dpia_gemm_bf16(dCb, Bb, gA, n, n, n, n, n, n, 0, 1)),
                 ("bf16_bwd_dB", lambda: dpia.dpia_gemm_bf16(Ab, dCb, gB, n, n, n, n, n, n, 1, 0)))
        for name, fn in calls:
            fn() if tl is None else tl.call(name, fn)

    per, step_ms, clk = timed_steps(args, device, dist, ["bf16_fwd", "bf16_bwd_dA", "bf16_bwd_dB"], step,
                                    L2Flush(device))
    fl = 2 * n ** 3
    _, bf16_peak, bf16_sust, src = peaks()
    kern = {k: {"avg_us": round(v * 1e3, 2), "flops": fl, "TFLOP_s": round(fl / v / 1e9, 1)} for k, v in per.items()}
    # FP32 fold forward, a few launches of each schedule, L2 flushed before each
    # (it runs on the FMA pipes, not the tensor cores)
    fl2 = L2Flush(device)

    def f32_median(schedule):
        ms = []
        for _ in range(5):
            fl2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dpia.dpia_gemm_f32(A, B, Cf, n, n, n, n, n, n, 0, 0, "fma", schedule=schedule)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]

    f32 = f32_median(0)
    f32_sched = {name: round(f32_median(sc) * 1e3, 1) for name, sc in
                 (("one_launch", 1), ("half_height_tail_tiles", 2), ("k_range_pieces", 3))}
    sm_max = max_sm_mhz(clk)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    fma_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    kern["f32_fold_fwd"] = {"median_us": round(f32 * 1e3, 1), "flops": fl, "TFLOP_s": round(fl / f32 / 1e9, 2),
                            "bound": "alu", "peak_TFLOP_s": round(fma_peak, 1),
                            "peak_source": f"{sms} SMs x 128 FP32 FMA lanes x 2 flops x {sm_max:.0f} MHz (the "
                                           "maximum SM clock)", "frac": round(fl / f32 / 1e9 / fma_peak, 4),
                            "schedules_median_us": f32_sched}
    # each launch alone (L2 flushed before it): one CTA per 256-row tile (cta_group::1), CTA pairs
    # (cta_group::2) on 256-row and 512-row tiles, and cuBLAS (torch.matmul, bf16 out) on the same shape
    flush = L2Flush(device)
    by_cluster = {}
    Cb = torch.empty(n, n, device=device, dtype=torch.bfloat16)
    for label, cl, tm in (("1", 1, 0), ("2", 2, 256), ("2x512", 2, 512)):
        calls = {"bf16_fwd": lambda cl=cl, tm=tm: dpia.dpia_gemm_bf16(Ab, Bb, C, n, n, n, n, n, n, 0, 0,
                                                                      cluster=cl, tile_m=tm),
                 "bf16_bwd_dA": lambda cl=cl, tm=tm: dpia.dpia_gemm_bf16(dCb, Bb, gA, n, n, n, n, n, n, 0, 1,
                                                                         cluster=cl, tile_m=tm),
                 "bf16_bwd_dB": lambda cl=cl, tm=tm: dpia.dpia_gemm_bf16(Ab, dCb, gB, n, n, n, n, n, n, 1, 0,
                                                                         cluster=cl, tile_m=tm)}
        alone = standalone_us(calls, {}, flush=flush, reps=10)
        by_cluster[label] = {k: {"median_us": v["median_us"], "TFLOP_s": round(fl / v["median_us"] / 1e6, 1),
                                   "frac": round(fl / v["median_us"] / 1e6 / bf16_peak, 4)}
                               for k, v in alone.items()}
    kern["alone_by_cluster"] = by_cluster
    cub = standalone_us({"bf16_fwd": lambda: torch.matmul(Ab, Bb, out=Cb)}, {}, flush=flush, reps=10)["bf16_fwd"]
    kern["cublas_same_shape"] = {"what": "torch.matmul(A, B) in bf16 (bf16 output), each launch alone, L2 flushed",
                                 "median_us": cub["median_us"], "TFLOP_s": round(fl / cub["median_us"] / 1e6, 1)}
    prec = torch.get_float32_matmul_precision()
    torch.set_float32_matmul_precision("highest")  # FP32 on the CUDA cores, no TF32
    try:
        cuf = standalone_us({"f32": lambda: torch.matmul(A, B, out=Cf)}, {}, flush=flush, reps=5)["f32"]
    finally:
        torch.set_float32_matmul_precision(prec)
    kern["f32_fold_fwd"]["cublas_same_shape"] = {
        "what": "torch.matmul(A, B) in FP32 with TF32 off (no fixed fold order), each launch alone, L2 flushed",
        "median_us": cuf["median_us"], "TFLOP_s": round(fl / cuf["median_us"] / 1e6, 2)}
    if args.gemm_ksweep:
        # the forward over K at M = N = 4096: the slope is the mainloop's rate, the intercept the
        # per-launch cost (writing C, filling the pipeline, the launch itself)
        sweep = {}
        for K in (512, 1024, 2048, 4096, 8192):
            Ak = torch.randn(n, K, device=device, generator=torch.Generator(device=device).manual_seed(4))
            Bk = torch.randn(K, n, device=device, generator=torch.Generator(device=device).manual_seed(5))
            Akb, Bkb = dpia.to_bf16(Ak), dpia.to_bf16(Bk)
            del Ak, Bk
            calls = {"one_sm": lambda: dpia.dpia_gemm_bf16(Akb, Bkb, C, n, n, K, K, n, n, 0, 0, cluster=1),
                     "pair_512": lambda: dpia.dpia_gemm_bf16(Akb, Bkb, C, n, n, K, K, n, n, 0, 0, cluster=2,
                                                             tile_m=512),
                     "cublas_bf16_out": lambda: torch.matmul(Akb, Bkb, out=Cb)}
            sweep[str(K)] = {k: v["median_us"] for k, v in standalone_us(calls, {}, flush=flush, reps=15).items()}
        kern["k_sweep_us"] = sweep
    dominant = max(per, key=per.get)  # the launch with the largest time share
    achieved = fl / per[dominant] / 1e9
    world = dist.get_world_size() if dist else 1
    total = 3 * fl
    layouts = {"bf16_fwd": "C = A B, B MN-major", "bf16_bwd_dA": "dA = dC B^T, both K-major",
               "bf16_bwd_dB": "dB = A^T dC, both MN-major"}
    roof = {"bound": "tensor",
            "kernel": f"gemm_bf16_pair_kernel<2>, 512-row tiles on CTA pairs ({dominant}: {layouts[dominant]})",
            "achieved": round(achieved, 1), "peak": bf16_peak, "unit": "TFLOP/s", "frac": round(achieved / bf16_peak, 4),
            "traffic": profile_traffic("gemm_bf16_4096.md", GEMM_SOURCES),
            "traffic_note": "DRAM bytes of one forward launch of the same kernel (ncu)",
            "peak_source": f"{src} bf16_tflops (cuBLAS burst)",
            "frac_per_launch": {k: round(fl / v / 1e9 / bf16_peak, 4) for k, v in per.items()}}
    cfg = {"workload": "GEMM 4096^3, A, B, dC ~ N(0,1) seed 4, BF16 inputs (RNE cast outside the timed kernels), "
                       "f32 accumulate: forward and backward; FP32 fold forward timed separately",
           "M": n, "N": n, "K": n, "l2": "flushed before every step (256 MiB read), outside the kernel events"}
    return _line(args, dist, round(world * total / (step_ms / 1e3) / 1e12, 1), "TFLOP/s", step_ms, "bf16", cfg,
                 kern, roof, clk, 3 * args.steps)


def batched_workload(args, device, dist):
    """4096 dots + 512 GEMVs, uneven sizes (seed 3), forward and backward: the
    batched persistent launch against one launch per instance (eager and under
    a CUDA graph). value = the fastest per-launch graph time over the policies
    the tuner tried / the batched graph time."""
    import math

    import torch

    from paper_1710_08332_gb300 import tune
    from synth import generator
    from synth import workloads as W

    dl, rows, cols = W.batched_shapes()
    dots, gemvs = dl.tolist(), list(zip(rows.tolist(), cols.tolist()))

    def make_inputs(b):
        g = generator(3, device)
        xs = torch.rand(b.xs_len, generator=g, device=device).mul_(2).sub_(1)
        ys = torch.rand(b.xs_len, generator=g, device=device).mul_(2).sub_(1)
        As = torch.randn(b.as_len, generator=g, device=device)
        for i, (_, n) in enumerate(b.gemv_shapes):
            b.a_view(As, i).mul_(1.0 / math.sqrt(n))
        gx = torch.rand(b.gx_len, generator=g, device=device).mul_(2).sub_(1)
        dot_g = torch.rand(len(b.dot_lengths), generator=g, device=device).mul_(2).sub_(1)
        gdy = torch.rand(b.gy_len, generator=g, device=device).mul_(2).sub_(1)
        return xs, ys, As, gx, dot_g, gdy

    b, tune_ms = tune.tune_batch(dots, gemvs, make_inputs)
    xs, ys, As, gx, dot_g, gdy = make_inputs(b)
    dot_out = torch.empty(len(dots), device=device)
    gy = torch.empty(b.gy_len, device=device)
    dxs, dys, dAs, dgx = torch.empty_like(xs), torch.empty_like(ys), torch.empty_like(As), torch.empty_like(gx)
    pl_ws = b.per_launch_workspace()
    pl_bws = b.per_launch_bwd_workspaces()
    stream = torch.cuda.current_stream(device)

    def graph_of(fn):
        s = torch.cuda.Stream(device)
        s.wait_stream(stream)
        with torch.cuda.stream(s):
            fn()
        stream.wait_stream(s)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            fn()
        return gr

    fwd_b = lambda: b.forward(xs, ys, dot_out, As, gx, gy)
    bwd_b = lambda: b.backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx)
    fwd_p = lambda: b.per_launch_forward(xs, ys, dot_out, As, gx, gy, pl_ws)
    bwd_p = lambda: b.per_launch_backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx, pl_bws)
    g_fwd_b, g_bwd_b, g_fwd_p, g_bwd_p = graph_of(fwd_b), graph_of(bwd_b), graph_of(fwd_p), graph_of(bwd_p)

    names = ["batched_fwd", "batched_bwd", "graph_batched_fwd", "graph_batched_bwd",
             "per_launch_fwd", "per_launch_bwd", "graph_per_launch_fwd", "graph_per_launch_bwd"]
    fns = [fwd_b, bwd_b, g_fwd_b.replay, g_bwd_b.replay, fwd_p, bwd_p, g_fwd_p.replay, g_bwd_p.replay]

    def step(tl):
        for name, fn in zip(names, fns):
            fn() if tl is None else tl.call(name, fn)

    per, _, clk = timed_steps(args, device, dist, names, step)
    # the conservative baseline: one launch per instance under each policy the tuner
    # tried (the packed layout does not depend on the policy), the fastest of them
    from paper_1710_08332_gb300.batch import Batch

    per_launch_by_policy = {}
    for pol in tune.batch_candidates():
        bb = Batch(dots, gemvs, policy=pol)
        ws1, bws1 = bb.per_launch_workspace(), bb.per_launch_bwd_workspaces()
        gr = graph_of(lambda: (bb.per_launch_forward(xs, ys, dot_out, As, gx, gy, ws1),
                               bb.per_launch_backward(xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx, bws1)))
        label = f"T{pol.threads}:dotcap{pol.dot_split_cap}:rs{pol.row_split}:sched{pol.schedule}"
        per_launch_by_policy[label] = round(tune.time_call(gr.replay, reps=3, warmup=1), 3)
        del gr, ws1, bws1, bb
    best_per_launch = min(per_launch_by_policy.values())
    # subsets (forward, batched launch each): dots only and GEMVs only
    bd = Batch(dots, [], policy=b.policy)
    bg = Batch([], gemvs, policy=b.policy)
    sub = {}
    for label, bb, f in (("dots", bd, lambda bb: bb.forward(xs, ys, dot_out, None, None, None)),
                         ("gemvs", bg, lambda bb: bb.forward(None, None, None, As, gx, gy))):
        sub[label + "_batched_fwd_us"] = round(tune.time_call(lambda: f(bb), reps=5) * 1e3, 1)
    for label, bb, f in (("dots", bd, lambda bb: bb.per_launch_forward(xs, ys, dot_out, None, None, None, pl_ws)),
                         ("gemvs", bg, lambda bb: bb.per_launch_forward(None, None, None, As, gx, gy, pl_ws))):
        gr = graph_of(lambda: f(bb))
        sub[label + "_graph_per_launch_fwd_us"] = round(tune.time_call(gr.replay, reps=5) * 1e3, 1)

    n_dot = int(sum(dots))
    mn = int(sum(m * n for m, n in gemvs))
    fwd_bytes = 8 * n_dot + 4 * mn
    bwd_bytes = 16 * n_dot + 8 * mn
    hbm = peaks()[0]
    kern = {k: {"avg_ms": round(v, 4)} for k, v in per.items()}
    kern["batched_fwd"]["GB_s"] = round(fwd_bytes / per["batched_fwd"] / 1e6, 1)
    kern["batched_bwd"]["GB_s"] = round(bwd_bytes / per["batched_bwd"] / 1e6, 1)
    speed_eager = (per["per_launch_fwd"] + per["per_launch_bwd"]) / (per["batched_fwd"] + per["batched_bwd"])
    speed_graph = (per["graph_per_launch_fwd"] + per["graph_per_launch_bwd"]) / \
        (per["graph_batched_fwd"] + per["graph_batched_bwd"])
    achieved = fwd_bytes / per["batched_fwd"] / 1e6
    ratio = profile_traffic("batch_kernels_4096dots_512gemvs.md", BATCH_SOURCES,
                            key="traffic_bytes_per_algorithmic_byte")
    traffic = round(ratio * fwd_bytes) if ratio is not None else None
    roof = {"bound": "hbm", "kernel": "batch_fwd_kernel (dpia_batch_forward_f32)", "achieved": round(achieved, 1),
            "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
            "traffic_note": "DRAM bytes per algorithmic byte of the forward kernel on a small case of the same "
                            "batch (ncu), times this launch's algorithmic bytes",
            "peak_source": "measured hbm_gbs (copy, burst)", "algorithmic_bytes_per_launch": fwd_bytes,
            "bwd_frac": round(bwd_bytes / per["batched_bwd"] / 1e6 / hbm, 4)}
    cfg = {"workload": "batched uneven instances: 4096 f32 dots (lengths log-uniform [256, 65536]) + 512 GEMVs "
                       "(rows log-uniform [256, 65536], cols [256, 4096]), seed 3, packed with offsets (matrix rows padded to 128-byte lines), forward + "
                       "backward; one persistent launch per direction vs one launch per instance",
           "dots": len(dots), "gemvs": len(gemvs), "dot_elements": n_dot, "gemv_elements": mn,
           "policy": b.policy.__dict__, "tuned_ms": tune_ms,
           "l2": "inputs larger than L2 (tens of GB)"}
    world = dist.get_world_size() if dist else 1
    speed_best = best_per_launch / (per["graph_batched_fwd"] + per["graph_batched_bwd"])
    extra = {"speedup_eager": round(speed_eager, 2), "speedup_graph_same_strategies": round(speed_graph, 2),
             "per_launch_graph_ms_by_policy": per_launch_by_policy, "subsets": sub}
    line = _line(args, dist, round(speed_best, 2),
                 "x (fastest per-launch time over the tuned policies / batched time, forward + backward, "
                 "both as CUDA graphs)",
                 per["batched_fwd"] + per["batched_bwd"], "f32", cfg, kern, roof, clk,
                 (2 + 2 + 2 * (len(dots) + len(gemvs)) * 2) * args.steps, extra)
    line["higher_is_better"] = True
    return line


def generated_single_launch(device, x, y, A, xv, sms: int, reps: int = 20):
    """The generated one-kernel reductions (thread folds, lane trees, the second
    level in the last block) on the bandwidth inputs and the GEMV matrix, each
    beside the library's kernel with the same strategy, timed alone (back to
    back launches). The dot takes the faster of two splits."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from paper_1710_08332_gb300 import codegen as G
    from paper_1710_08332_gb300 import tune
    from paper_1710_08332_gb300.codegen import programs as PR

    n = x.numel()
    M, N = A.shape
    out = torch.empty(1, device=device)
    yv = torch.empty(M, device=device)
    res, best = {}, None
    for s_, T, V, T2 in ((16384, 256, 4, 256), (32768, 256, 4, 256)):
        C = n // s_
        kd = G.compile_cuda(f"gen_dot_R_s{s_}_T{T}", *PR.dot_R(n, s_, T, V, "interleaved", "tree", min(T2, C)),
                            unroll=4)
        td = kd.temps_like(device)
        st = dpia.ReduceStrategy(split=s_, threads=T, vec=V, second="tree", threads2=min(T2, C))
        ws = dpia.workspace(dpia.dpia_dot_workspace_size(n, st), device)
        g_ms = tune.time_call(lambda: kd.run(x, y, out, *td), reps=reps)
        l_ms = tune.time_call(lambda: dpia.dpia_dot_f32(x, y, n, st, out, ws), reps=reps)
        label = f"dot_R s={s_} T={T} V={V} tree {min(T2, C)}"
        res[label] = {"generated_us": round(g_ms * 1e3, 2), "library_us": round(l_ms * 1e3, 2),
                      "generated_GB_s": round(8 * n / g_ms / 1e6, 1), "library_GB_s": round(8 * n / l_ms / 1e6, 1),
                      "generated_over_library_time": round(l_ms / g_ms, 3)}
        if best is None or g_ms < best[1]:
            best = (label, g_ms, l_ms, kd, td, st)
    label, g_ms, l_ms, kd, td, st = best
    # one operand: twice the unroll of the dot, the same bytes of loads in flight per thread
    ka = G.compile_cuda("gen_asum_R", *PR.asum_R(n, st.split, st.threads, st.vec, "interleaved", "tree",
                                                 st.threads2), unroll=8)
    ta = ka.temps_like(device)
    ws = dpia.workspace(dpia.dpia_dot_workspace_size(n, st), device)
    ga = tune.time_call(lambda: ka.run(x, out, *ta), reps=reps)
    la = tune.time_call(lambda: dpia.dpia_asum_f32(x, n, st, out, ws), reps=reps)
    res["asum_R (the dot's strategy)"] = {"generated_us": round(ga * 1e3, 2), "library_us": round(la * 1e3, 2),
                                          "generated_GB_s": round(4 * n / ga / 1e6, 1),
                                          "generated_over_library_time": round(la / ga, 3)}
    # compensated (Kahan at every level): lane pairs, trees over (s, c) by shuffles; the
    # faster of two splits (the folds not unrolled: measured fastest for this chain)
    kbest = None
    for s_ in (16384, 32768):
        C = n // s_
        kk = G.compile_cuda(f"gen_dot_R_kahan_s{s_}", *PR.dot_R_kahan(n, s_, 256, 4, "interleaved", "tree",
                                                                     min(256, C)), unroll=1)
        tk = kk.temps_like(device)
        stk = dpia.ReduceStrategy(split=s_, threads=256, vec=4, second="tree", threads2=min(256, C),
                                  compensated=True)
        wsk = dpia.workspace(dpia.dpia_dot_workspace_size(n, stk), device)
        gk = tune.time_call(lambda: kk.run(x, y, out, *tk), reps=reps)
        lk = tune.time_call(lambda: dpia.dpia_dot_f32(x, y, n, stk, out, wsk), reps=reps)
        if kbest is None or gk < kbest[1]:
            kbest = (s_, gk, lk)
    s_, gk, lk = kbest
    res[f"dot_R compensated (Kahan) s={s_} T=256 V=4 tree"] = {
        "generated_us": round(gk * 1e3, 2), "library_us": round(lk * 1e3, 2),
        "generated_GB_s": round(8 * n / gk / 1e6, 1), "generated_over_library_time": round(lk / gk, 3)}
    kg = G.compile_cuda("gen_gemv_R", *PR.gemv_R(M, N, 128, 4), unroll=4)
    stg = dpia.ReduceStrategy(split=N, threads=128, vec=4)
    gg = tune.time_call(lambda: kg.run(A, xv, yv), reps=reps)
    lg = tune.time_call(lambda: dpia.dpia_gemv_f32(A, M, N, N, xv, yv, stg), reps=reps)
    gb = 4 * M * N + 4 * (M + N)
    res["gemv_R (a block of 128 per row, float4)"] = {
        "generated_us": round(gg * 1e3, 2), "library_us": round(lg * 1e3, 2),
        "generated_GB_s": round(gb / gg / 1e6, 1), "generated_over_library_time": round(lg / gg, 3)}
    res["gemm (4096^3 FP32)"] = generated_gemm(device, reps=max(3, reps // 4))
    return res, best


def generated_gemm(device, reps: int = 5):
    """The generated FP32 GEMM at 4096^3 in two forms of the same map of maps of
    a fold over k: a workgroup per row with four adjacent columns per thread as
    one float4 fold, and the register-tiled form (a workgroup per 8 rows, each
    thread an 8 x 8 block of C accumulated in a private array, A read along k
    as float4); beside them the library's register-tiled FP32 fold with
    contraction off (the same fold of every element), all on the GEMM inputs,
    L2 flushed before every launch (A and B fit in it). Each form takes the
    fastest of its block sizes."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from paper_1710_08332_gb300 import codegen as G
    from paper_1710_08332_gb300.codegen import programs as PR
    from synth import workloads as W

    n = W.GEMM_MNK
    A, B, _ = W.gemm(device)
    C = torch.empty(n, n, device=device)
    flush = torch.empty(64 << 20, device=device)

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    fl = 2.0 * n ** 3
    lib = {c: timed(lambda: dpia.dpia_gemm_f32(A, B, C, n, n, n, n, n, n, 0, 0, c)) for c in ("off", "fma")}
    out = {"library_fold_off_ms": round(lib["off"], 3), "library_TFLOP_s": round(fl / lib["off"] / 1e9, 2),
           "library_fold_fma_ms": round(lib["fma"], 3), "library_fma_TFLOP_s": round(fl / lib["fma"] / 1e9, 2)}
    forms = {"columns (a workgroup per row, float4 columns)":
             (G.compile_cuda("gen_gemm_4096_v4", *PR.gemm(n, n, n, 4), unroll=4), (256, 512, 1024), "off"),
             "tiled (8 x 8 per thread in a private array, A along k as float4)":
             (G.compile_cuda("gen_gemm_4096_tiled", *PR.gemm_tiled(n, n, n, 8, 8, 4, 4)), (128, 256), "off"),
             "tiled, contraction fma (16 x 8 per thread)":
             (G.compile_cuda("gen_gemm_4096_tiled_fma", *PR.gemm_tiled(n, n, n, 16, 8, 4, 4, contract="fma")),
              (128, 256), "fma")}
    for label, (k, blocks, contract) in forms.items():
        by_block = {b: timed(lambda: k.run(A, B, C, block=b)) for b in blocks}
        blk = min(by_block, key=by_block.get)
        out[label] = {"ms": round(by_block[blk], 3), "TFLOP_s": round(fl / by_block[blk] / 1e9, 2), "block": blk,
                      "by_block_ms": {str(b): round(v, 3) for b, v in by_block.items()}, "contract": contract,
                      "over_library_time": round(lib[contract] / by_block[blk], 3)}
    out["note"] = ("every element of each form equal to the library's fold with the same contraction (tests); "
                   "no form stages tiles in shared memory")
    return out


def codegen_workload(args, device, dist):
    """Kernels produced by the code generator from the paper's phrases, on the
    bandwidth inputs (n = 2^26) and the GEMV 8192^2 inputs. The line's value is
    the dot generated as ONE kernel with the canonical strategy (per-thread
    folds on asVector 4, lane trees within warps and over the warp sums, the
    second level in the last block), beside the library's hand-written dot with
    the same strategy. Also timed: the same phrases in the paper's own form
    (per-thread lane partials, then folding kernels), asum, scal, GEMV (one
    kernel, and partials + row folds) and the GEMV backward, the rewrite
    exploration, and the host C build of the dot partials (OpenMP)."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from paper_1710_08332_gb300 import codegen as G
    from paper_1710_08332_gb300.codegen import programs as PR
    from synth import workloads as W

    n = W.BW_N
    x, y = W.bandwidth(device)
    A, xv, _ = W.gemv(device)
    M, N_ = A.shape
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    single, best = generated_single_launch(device, x, y, A, xv, sms)
    best_label, _, _, kdR, tdR, st_best = best
    out1 = torch.empty(1, device=device)
    # the paper's form: lane partials over 2048 chunks of 2^15 with 256 threads,
    # then the folding stages of the rewrite lowering's fold plan
    s, Tn, V = 1 << 15, 256, 4
    m1 = n // s * Tn * V
    k1 = G.compile_cuda("gen_dot_partials", *PR.dot_partials(n, s, Tn, V=V), unroll=4)
    from paper_1710_08332_gb300.codegen import rewrite as RW

    folds, left = [], m1
    for grp in RW.fold_plan(m1):
        ph = PR.fold_all(left) if grp == left else PR.fold_cols(left // grp, grp)
        folds.append((G.compile_cuda(f"gen_dot_fold_{left}_{grp}", *ph, unroll=64), left // grp))
        left //= grp
    fold_bufs = [torch.empty(max(cnt, 1), device=device) for _, cnt in folds]

    def dot_folds():
        src = part
        for (k, cnt), dst in zip(folds, fold_bufs):
            k.run(src, dst, grid=max(1, cnt // 64), block=min(64, cnt) if cnt > 1 else 1)
            src = dst
    ks = G.compile_cuda("gen_scal", *PR.scal(n, W.SCAL_A, V=V))
    kg = G.compile_cuda("gen_gemv_partials", *PR.gemv_partials(M, N_, 128))
    kr = G.compile_cuda("gen_gemv_rows", *PR.fold_rows(M, 128), unroll=64)
    R = 32  # dx: row chunks of 32 (256 workgroups), then the fold over the chunks
    kdx = G.compile_cuda("gen_gemv_dx_partials", *PR.gemv_bwd_dx_partials(M, N_, R), unroll=8)
    kdf = G.compile_cuda("gen_gemv_dx_fold", *PR.gemv_bwd_dx_fold(M // R, N_), unroll=64)
    kda = G.compile_cuda("gen_gemv_dA", *PR.gemv_bwd_dA(M, N_))
    dyv = torch.rand(M, device=device)
    dxpart = torch.empty(M // R * N_, device=device)
    dxv = torch.empty(N_, device=device)
    dAm = torch.empty(M * N_, device=device)
    part = torch.empty(m1, device=device)
    ys = torch.empty_like(x)
    gpart = torch.empty(M * 128, device=device)
    yv = torch.empty(M, device=device)
    ws = dpia.workspace(dpia.dpia_dot_workspace_size(n, st_best), device)
    # step order: each of the two compared dots follows a kernel that leaves no
    # dirty lines in L2 (the kernels after scal and dA pay for writing theirs back)
    calls = {
        "gen_gemv_dA": lambda: kda.run(dyv, xv, dAm),
        "gen_gemv_partials": lambda: kg.run(A, xv, gpart),
        "gen_gemv_rows": lambda: kr.run(gpart, yv, grid=M // 64, block=64),  # a thread per row over 128 SMs
        "gen_dot_R": lambda: kdR.run(x, y, out1, *tdR),
        "library_dot": lambda: dpia.dpia_dot_f32(x, y, n, st_best, out1, ws),
        "gen_dot_partials": lambda: k1.run(x, y, part),
        "gen_dot_folds": dot_folds,
        "gen_scal": lambda: ks.run(x, ys, grid=sms * 8, block=256),
        "gen_gemv_dx_partials": lambda: kdx.run(A, dyv, dxpart),
        "gen_gemv_dx_fold": lambda: kdf.run(dxpart, dxv, grid=N_ // 64, block=64),  # a thread per column
    }
    bytes_ = {"gen_dot_R": 8 * n, "library_dot": 8 * n, "gen_dot_partials": 8 * n, "gen_scal": 8 * n,
              "gen_gemv_partials": 4 * M * N_ + 4 * N_, "gen_gemv_dx_partials": 4 * M * N_ + 4 * M,
              "gen_gemv_dA": 4 * M * N_ + 4 * (M + N_)}
    names = list(calls)

    def step(tl):
        for name in names:
            calls[name]() if tl is None else tl.call(name, calls[name])

    per, step_ms, clk = timed_steps(args, device, dist, names, step)
    alone = standalone_us({k: calls[k] for k in ("gen_dot_R", "library_dot", "gen_dot_partials", "gen_scal",
                                                  "gen_gemv_partials", "gen_gemv_dx_partials", "gen_gemv_dA")},
                          bytes_)
    # rewrite-based exploration, every pipeline timed whole: the dot (split 2^14..2^16, 256
    # threads, both thread maps, widths 1 and 4, the paper's form and the one-kernel form),
    # sum |1.5 x_i| (with and without fusing scal's map into the reduction) and GEMV rows
    def summary(ranked, lib_us=None):
        d = {"candidates": len(ranked),
             "best": {"derivation": str(ranked[0][1]), "pipeline_us": round(ranked[0][0] * 1e3, 1)},
             "worst": {"derivation": str(ranked[-1][1]), "pipeline_us": round(ranked[-1][0] * 1e3, 1)},
             "all_us": {str(dd): round(ms * 1e3, 1) for ms, dd in ranked}}
        if lib_us is not None:
            d["library_us"] = lib_us
        return d

    explored = {"dot": summary(RW.explore("dot", [x, y], n, RW.derivations(
        n, threads=(256,), forms=("paper", "single")), reps=5), alone["library_dot"]["median_us"])}
    explored["asum_scal"] = summary(RW.explore("asum_scal", [x], n, RW.derivations(
        n, splits=(1 << 15,), threads=(256,), maps=("interleaved",), widths=(4,), forms=("paper", "single"),
        kind="asum_scal"), reps=5))
    explored["gemv"] = summary(RW.explore("gemv", [A, xv], N_, RW.gemv_derivations(M, N_, threads=(128, 256),
                                                                                  widths=(4,)), reps=5, M=M))
    explored["gemv_dx"] = summary(RW.explore("gemv_dx", [A, dyv], N_, RW.gemv_dx_derivations(M, N_), reps=5, M=M))
    # GEMM 4096^3: the plain map of maps and the register tiles (every derivation the same bits)
    gA, gB, _ = W.gemm(device)
    gk = W.GEMM_MNK
    ranked_g = RW.explore_gemm(gA, gB, gk, gk, gk, reps=3)
    explored["gemm"] = {"candidates": len(ranked_g),
                        "best": {"derivation": str(ranked_g[0][1]) or "plain", "block": ranked_g[0][2],
                                 "ms": round(ranked_g[0][0], 3),
                                 "TFLOP_s": round(2 * gk ** 3 / ranked_g[0][0] / 1e9, 2)},
                        "worst": {"derivation": str(ranked_g[-1][1]) or "plain", "block": ranked_g[-1][2],
                                  "ms": round(ranked_g[-1][0], 3)},
                        "all_ms": {f"{str(d) or 'plain'} @ {blk}": round(ms, 3) for ms, d, blk in ranked_g}}
    del gA, gB
    # the same phrases on the host (the paper's multicore target): C with the
    # outermost parallel loop (the work-group map) on OpenMP threads, the whole
    # dot (first level, trees, second level) on the full n = 2^26 inputs
    import numpy as np

    hx, hy = x.cpu().numpy(), y.cpu().numpy()
    hc = G.compile_c("host_dot_R", *PR.dot_R(n, st_best.split, st_best.threads, st_best.vec, "interleaved",
                                             "tree", st_best.threads2), openmp=True)
    hout = np.zeros(1, np.float32)
    htemps = hc.temps_like()
    hc.run(hx, hy, hout, *htemps)
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 3.0:
        hc.run(hx, hy, hout, *htemps)
        reps += 1
    host_s = (time.perf_counter() - t0) / reps
    host_line = {"kernel": f"generated C of the one-kernel dot ({best_label}), work-group loop on OpenMP threads",
                 "GB_s": round(8 * n / host_s / 1e9, 2), "ms": round(host_s * 1e3, 2), "n": n,
                 "threads": host_cores(), "reps": reps,
                 "same_bits_as_gpu": bool(hout.tobytes() == out1.cpu().numpy().tobytes())}
    hbm = peaks()[0]
    kern = {k: {"avg_us": round(v * 1e3, 2)} for k, v in per.items()}
    for k, b in bytes_.items():
        kern[k]["GB_s"] = round(b / per[k] / 1e6, 1)
    dot_ms = per["gen_dot_R"]
    achieved = 8 * n / dot_ms / 1e6
    roof = {"bound": "hbm", "kernel": f"gen_dot_R (generated, one kernel: {best_label})",
            "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": profile_traffic("codegen_dot_R_n2e25.md", generated_dot_R_digest()) if st_best.split == 16384 else None,
            "peak_source": "measured hbm_gbs (copy, burst)", "algorithmic_bytes_per_launch": 8 * n,
            "frac_alone": round(alone["gen_dot_R"]["GB_s"] / hbm, 4)}
    cfg = {"workload": "generated kernels: dot n=2^26 as one kernel (canonical strategy) and in the paper's "
                       "two-kernel form, scal (a=1.5), GEMV 8192^2 (one kernel; partials + row folds) and its "
                       "backward, bandwidth inputs seed 1 / GEMV seed 2; beside them the library's kernels with "
                       "the same strategies", "n": n, "strategy": st_best.as_dict(),
           "l2": "inputs larger than L2"}
    world = dist.get_world_size() if dist else 1
    return _line(args, dist, round(world * 8 * n / (dot_ms / 1e3) / 1e9, 1), "GB/s", dot_ms, "f32", cfg, kern,
                 roof, clk, len(names) * args.steps,
                 {"kernels_alone": alone, "single_launch": single, "explored_dot": explored,
                  "host_generated_dot": host_line,
                  "generated_dot_vs_library_dot": round(per["library_dot"] / per["gen_dot_R"], 3),
                  "paper_form_dot_vs_library_dot": round(per["library_dot"] /
                                                         (per["gen_dot_partials"] + per["gen_dot_folds"]), 3)})


def cpu_baseline_for(workload):
    """Oracle timings for the secondary workloads (bounded samples, the oracle's
    units on every host core)."""
    import numpy as np

    from oracle import loopnest
    from oracle import patterns as P
    from synth import workloads as W

    cores = host_cores()
    loopnest.set_threads(cores)

    t0 = time.perf_counter()
    if workload == "dot":
        x, y = W.dot_f32("cpu")
        reps = 0
        while time.perf_counter() - t0 < 5.0:
            loopnest.dot_f32(x.numpy(), y.numpy(), P.Strategy(s=8192, T=256, V=4))
            reps += 1
        dt = time.perf_counter() - t0
        return {"value": round(reps * 8 * x.numel() / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle dot (same strategy) on the full n=2^20 input, {reps} reps, {dt:.1f} s"}
    if workload == "gemv":
        A, x, dy = W.gemv("cpu", M=1024)
        hA, hx, hdy = A.numpy(), x.numpy(), dy.numpy()
        reps = 0
        while time.perf_counter() - t0 < 10.0:
            loopnest.gemv_f32(hA, hx, P.Strategy(s=8192, T=256, V=4))
            loopnest.gemv_bwd_dx_f32(hA, hdy, 64)
            loopnest.gemv_bwd_dA_f32(hx, hdy)
            reps += 1
        dt = time.perf_counter() - t0
        b = 3 * 4 * hA.size
        return {"value": round(reps * b / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle GEMV forward + dx + dA on 1024 of the 8192 rows, {reps} reps, {dt:.1f} s"}
    if workload == "batched":
        import torch

        dl, _, _ = W.batched_shapes()
        lens = dl.tolist()[:64]
        xs = [torch.rand(n).numpy() for n in lens]
        st = P.Strategy(s=8192, T=256, V=4, second="tree", T2=256, pad=True)
        reps = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0:
            for x in xs:
                loopnest.dot_f32(x, x, st)
            reps += 1
        dt = time.perf_counter() - t0
        return {"value": round(reps * 8 * sum(lens) / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle dots of the first 64 batch instances ({sum(lens)} elements), {reps} passes, "
                          f"{dt:.1f} s"}
    if workload == "gemm":
        A, B, _ = W.gemm("cpu", M=64)
        rows = np.arange(64)
        cols = np.arange(4096)
        loopnest.gemm_f32_sample(A.numpy(), B.numpy(), False, False, True, rows, cols)
        dt = time.perf_counter() - t0
        return {"value": round(2 * 64 * 4096 * 4096 / dt / 1e12, 5), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle FP32 fold (FMA) for 64 of the 4096 rows of C = A B, {dt:.1f} s"}
    return None


def e2e_bandwidth(args, device, dist, st_dot, st_asum, hx, hy, step_bytes):
    """The same step through the public API with pinned host inputs and a host
    read of the results, copies inside the timed region. Steps are pipelined
    over two device buffer sets: the host-to-device copies run on one stream,
    the kernels on a second and the device-to-host copies on a third, so one
    step's copies overlap the previous step's kernels and read-back."""
    import torch

    import paper_1710_08332_gb300 as dpia
    from synth import workloads as W

    n = hx.numel()
    px, py = hx.pin_memory(), hy.pin_memory()
    host_scal = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    host_res = [torch.empty(2, dtype=torch.float32).pin_memory() for _ in range(2)]
    E = lambda: torch.cuda.Event()
    sets = []
    for _ in range(2):
        sets.append({"x": torch.empty(n, device=device), "y": torch.empty(n, device=device),
                     "ys": torch.empty(n, device=device), "res": torch.empty(2, device=device),
                     "ws_d": dpia.workspace(dpia.dpia_dot_workspace_size(n, st_dot), device),
                     "ws_a": torch.zeros(dpia.dpia_dot_workspace_size(n, st_asum), dtype=torch.uint8,
                                         device=device),
                     "ev_x": E(), "ev_y": E(), "ev_s": E(), "done_comp": E(), "done_out": E()})
    s_in, s_comp, s_out = (torch.cuda.Stream(device) for _ in range(3))
    K = max(3, min(args.steps, 20))

    def one(i):
        b = sets[i % 2]
        s_in.wait_event(b["done_comp"])  # the set's previous kernels have read x and y
        s_in.wait_event(b["done_out"])   # and its previous scal output has been read back
        with torch.cuda.stream(s_in):
            b["x"].copy_(px, non_blocking=True)
            b["ev_x"].record(s_in)
            b["y"].copy_(py, non_blocking=True)
            b["ev_y"].record(s_in)
        s_comp.wait_event(b["ev_x"])
        s_comp.wait_event(b["done_out"])
        with torch.cuda.stream(s_comp):
            dpia.dpia_asum_f32(b["x"], n, st_asum, b["res"][0:1], b["ws_a"])
            dpia.dpia_scal_f32(W.SCAL_A, b["x"], b["ys"], n, 4)
            b["ev_s"].record(s_comp)
            s_comp.wait_event(b["ev_y"])
            dpia.dpia_dot_f32(b["x"], b["y"], n, st_dot, b["res"][1:2], b["ws_d"])
            b["done_comp"].record(s_comp)
        s_out.wait_event(b["ev_s"])
        with torch.cuda.stream(s_out):
            host_scal[i % 2].copy_(b["ys"], non_blocking=True)
            s_out.wait_event(b["done_comp"])
            host_res[i % 2].copy_(b["res"], non_blocking=True)
            b["done_out"].record(s_out)

    for b in sets:  # initial state: nothing in flight
        for k in ("done_comp", "done_out"):
            b[k].record(torch.cuda.current_stream(device))
    for i in range(4):
        one(i)
    torch.cuda.synchronize(device)
    barrier(dist, device)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s_in)
    for i in range(K):
        one(i)
    cur = torch.cuda.current_stream(device)
    for st_ in (s_in, s_comp, s_out):
        cur.wait_stream(st_)
    t1.record(cur)
    t1.synchronize()
    ms = reduce_max(dist, t0.elapsed_time(t1) / K, device if dist and dist.get_backend() == "nccl" else None)
    # context: the link alone, one 256 MiB pinned copy in each direction
    link = {}
    for name, fn in (("h2d_GB_s", lambda: sets[0]["x"].copy_(px, non_blocking=True)),
                     ("d2h_GB_s", lambda: host_scal[0].copy_(sets[0]["ys"], non_blocking=True))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        a.record()
        for _ in range(5):
            fn()
        b.record()
        b.synchronize()
        link[name] = round(5 * 4 * n / (a.elapsed_time(b) / 1e3) / 1e9, 1)
    world = dist.get_world_size() if dist else 1
    return {"value": round(world * step_bytes / (ms / 1e3) / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 8, "steps": K,
            "ms_per_step": round(ms, 3), "link_alone": link,
            "overlap": "two device buffer sets; host-to-device copies, kernels and device-to-host copies "
                       "on three streams"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline object and --impl reference)
# ---------------------------------------------------------------------------


def oracle_bandwidth_sample(n_sample: int, reps: int, st_dot=None, st_asum=None):
    """Time the oracle (C loop nests, its units on the thread count set by
    loopnest.set_threads) on asum + scal + dot of n_sample elements; returns
    (GB/s, seconds)."""
    from oracle import loopnest
    from oracle import patterns as P
    from synth import workloads as W

    x, y = W.bandwidth("cpu", n=n_sample)
    hx, hy = x.numpy(), y.numpy()
    od = P.Strategy(s=8192, T=256, V=4, second="tree", T2=256, pad=n_sample % 8192 != 0)
    if st_dot is not None:
        od = P.Strategy(s=st_dot.split, T=st_dot.chunk_threads, V=st_dot.vec, thread_map=st_dot.thread_map,
                        second=st_dot.second, T2=st_dot.threads2, pad=n_sample % st_dot.split != 0)
    oa = od
    if st_asum is not None:
        oa = P.Strategy(s=st_asum.split, T=st_asum.chunk_threads, V=st_asum.vec, thread_map=st_asum.thread_map,
                        second=st_asum.second, T2=st_asum.threads2, pad=n_sample % st_asum.split != 0)
    loopnest.lib()
    t0 = time.perf_counter()
    for _ in range(reps):
        loopnest.asum_f32(hx, oa)
        loopnest.scal_f32(W.SCAL_A, hx)
        loopnest.dot_f32(hx, hy, od)
    dt = time.perf_counter() - t0
    step_bytes = 20 * n_sample
    return reps * step_bytes / dt / 1e9, dt


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


def cpu_baseline(st_dot=None, st_asum=None, budget_s: float = 8.0):
    """The oracle on the host: every core this process may run on (the value),
    and one core beside it, each for about budget_s on n = 2^24."""
    from oracle import loopnest

    n_sample = 1 << 24
    res = {}
    old = loopnest.set_threads(1)
    try:
        for cores in (host_cores(), 1):
            loopnest.set_threads(cores)
            _, dt = oracle_bandwidth_sample(n_sample, 1, st_dot, st_asum)
            reps = max(1, int(budget_s / max(dt, 1e-3)))
            gbs, dt = oracle_bandwidth_sample(n_sample, reps, st_dot, st_asum)
            res[cores] = (gbs, reps, dt)
    finally:
        loopnest.set_threads(old)
    cores = host_cores()
    gbs, reps, dt = res[cores]
    g1, r1, d1 = res[1]
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle loop-nest evaluator (C, -O2 -ffp-contract=off; chunks, and scal's elements, on "
                      f"{cores} OpenMP threads, every fold across chunks on one): asum + scal + dot on n=2^24 of "
                      f"the same distribution with the GPU's strategies, {reps} rep(s), {dt:.1f} s",
            "seconds": round(dt, 2),
            "one_core": {"value": round(g1, 3), "unit": "GB/s", "cores": 1, "reps": r1, "seconds": round(d1, 2)}}


def reference_arm(args):
    """The oracle timed as it stands on the host cores: each step asum + scal +
    dot on a bounded sample (n = 2^22) of the bandwidth workload."""
    from oracle import loopnest

    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    cores = host_cores()
    loopnest.set_threads(cores)
    n_sample = 1 << 22
    for _ in range(args.warmup):
        oracle_bandwidth_sample(n_sample, 1)
    gbs, dt = oracle_bandwidth_sample(n_sample, args.steps)
    step_bytes = 20 * n_sample
    ms_step = dt / args.steps * 1e3
    cb = {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
          "sample": f"each step: oracle asum + scal + dot on n=2^22 (1/16 of the 2^26 workload), {cores} threads "
                    f"over chunks"}
    return {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "bandwidth set: asum + scal(a=1.5) + dot, f32, U[-1,1) seed 1 "
                                   "(oracle sample n=2^22 per step)", "n": n_sample, "bytes_per_step": step_bytes},
            "cpu_baseline": cb,
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["bandwidth", "dot", "gemv", "gemm", "batched", "codegen"],
                    default="bandwidth",
                    help="bandwidth (default: the headline step); dot (n=2^20, split 8192), gemv (8192^2 "
                         "forward + backward), gemm (4096^3 BF16 forward + backward, FP32 fold forward), batched "
                         "(4096 dots + 512 GEMVs of uneven sizes, one launch vs one launch per instance), codegen "
                         "(kernels generated from the paper's phrases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="bandwidth workload: skip the summary of the other workloads (dot 2^20, GEMV, GEMM, "
                         "batched) in the headline line")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the split autotuner; use the default strategy (split 16384, tree second level)")
    ap.add_argument("--profile", choices=sorted(PROFILE_CASES),
                    help="run a small case of one kernel --reps times (for ncu captures); no JSON line")
    ap.add_argument("--n", type=int, default=1 << 25, help="elements (or rows x cols) of the --profile case")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cluster", type=int, default=0, choices=[0, 1, 2],
                    help="CTAs per tile of the BF16 GEMM in the gemm --profile case (0 = one)")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1, 2, 3],
                    help="FP32 fold schedule in the gemm --profile case (0 automatic, 1 one launch, 2 half-height "
                         "tail tiles, 3 k-range pieces over two launches)")
    ap.add_argument("--gemm-ksweep", action="store_true",
                    help="gemm workload: also time the forward at K = 512..8192 (M = N = 4096)")
    ap.add_argument("--tile-m", type=int, default=0, choices=[0, 256, 512],
                    help="rows per tile of the BF16 GEMM in the gemm --profile case (512: CTA pairs only)")
    args = ap.parse_args(argv)
    if args.profile:
        return profile_case(args)
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        line = reference_arm(args)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0

    import torch

    global DEFAULT_BW_STRATEGY
    DEFAULT_BW_STRATEGY = _default_bw_strategy()
    world, rank, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = dist_init("nccl") if world > 1 else None
    if args.workload == "bandwidth":
        line = bandwidth_workload(args, device, dist)
        if not args.no_workloads:
            line["workloads"] = secondary_workloads(args, device, dist)
    else:
        line = {"dot": dot_workload, "gemv": gemv_workload, "gemm": gemm_workload,
                "batched": batched_workload, "codegen": codegen_workload}[args.workload](args, device, dist)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            if args.workload == "bandwidth":
                line["cpu_baseline"] = cpu_baseline(_strategy(line, "dot"), _strategy(line, "asum"))
            else:
                line["cpu_baseline"] = cpu_baseline_for(args.workload)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _pick(d: dict, *keys):
    return {k: d[k] for k in keys if k in d}


def secondary_workloads(args, device, dist):
    """The other workloads at full size, each timed on its own (K <= 10 steps
    after W >= 3 warm-ups, its own clock record), summarised for the headline
    line: the 2^20 dot, GEMV 8192^2 forward and backward, GEMM 4096^3 (BF16
    forward and backward, FP32 fold), the batched uneven instances, and the
    reductions generated from phrases as single kernels."""
    import copy

    import torch

    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.gemm_ksweep = max(3, min(args.steps, 10)), 3, False
    out = {}
    for name, fn in (("dot_n2e20", dot_workload), ("gemv_8192", gemv_workload), ("gemm_4096", gemm_workload),
                     ("batched", batched_workload)):
        t0 = time.time()
        try:
            line = fn(sub, device, dist)
        except Exception as exc:  # a failure here must not lose the headline line
            out[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            continue
        finally:
            torch.cuda.empty_cache()
        k, r = line["kernels"], line["roofline"]
        if name == "dot_n2e20":
            d = {"f32_us": k["dot_f32"]["avg_us"], "f32_GB_s": k["dot_f32"]["GB_s"],
                 "i32_us": k["dot_i32"]["avg_us"], "i32_GB_s": k["dot_i32"]["GB_s"], "frac": r["frac"],
                 "empty_launch_us": line["context"]["empty_launch_floor"]["median_us"],
                 "cublas_dot_us": line["context"]["torch_dot_cublas"]["median_us"]}
        elif name == "gemv_8192":
            a = line["kernels_alone"]
            d = {kk: {"GB_s": k[kk]["GB_s"], "frac": round(k[kk]["GB_s"] / r["peak"], 4),
                      "alone_GB_s": a[kk]["GB_s"], "alone_frac": round(a[kk]["GB_s"] / r["peak"], 4)}
                 for kk in ("gemv_fwd", "gemv_bwd_dx", "gemv_bwd_dA")}
        elif name == "gemm_4096":
            d = {kk: {"TFLOP_s": k[kk]["TFLOP_s"], "frac": r["frac_per_launch"][kk]}
                 for kk in ("bf16_fwd", "bf16_bwd_dA", "bf16_bwd_dB")}
            d["bf16_alone_512row_pairs"] = k["alone_by_cluster"]["2x512"]
            d["cublas_bf16_TFLOP_s"] = k["cublas_same_shape"]["TFLOP_s"]
            d["f32_fold_fwd"] = _pick(k["f32_fold_fwd"], "TFLOP_s", "frac", "peak_TFLOP_s", "peak_source",
                                      "schedules_median_us")
            d["cublas_f32_TFLOP_s"] = k["f32_fold_fwd"]["cublas_same_shape"]["TFLOP_s"]
        else:
            d = {"fwd_ms": k["batched_fwd"]["avg_ms"], "bwd_ms": k["batched_bwd"]["avg_ms"],
                 "fwd_GB_s": k["batched_fwd"]["GB_s"], "bwd_GB_s": k["batched_bwd"]["GB_s"],
                 "fwd_frac": r["frac"], "bwd_frac": r["bwd_frac"],
                 "speedup_vs_per_launch": line["value"], "speedup_unit": line["unit"],
                 "policy": line["config"]["policy"]}
        d["value"], d["unit"], d["ms_per_step"] = line["value"], line["unit"], line["ms_per_step"]
        d["roofline"] = _pick(r, "bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")
        d["steps"], d["warmup"], d["clocks"], d["wall_s"] = sub.steps, sub.warmup, line["clocks"], \
            round(time.time() - t0, 1)
        out[name] = d
    # kernels generated from phrases as one launch each, beside the library's
    t0 = time.time()
    clocks = ClockSampler(device.index)
    clocks.start()
    try:
        from synth import workloads as W

        x, y = W.bandwidth(device)
        A, xv, _ = W.gemv(device)
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        single, best = generated_single_launch(device, x, y, A, xv, sms, reps=10)
        out["codegen_single_launch"] = {
            "kernels": single, "best_dot": best[0],
            "generated_dot_over_library_dot_time": round(best[2] / best[1], 3),
            "note": "each kernel timed alone, back-to-back launches; the library's kernel runs the same strategy"}
    except Exception as exc:
        out["codegen_single_launch"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    finally:
        out.setdefault("codegen_single_launch", {})["clocks"] = clocks.stop()
        out["codegen_single_launch"]["wall_s"] = round(time.time() - t0, 1)
        torch.cuda.empty_cache()
    return out


def _strategy(line, op):
    from paper_1710_08332_gb300.strategy import ReduceStrategy

    return ReduceStrategy(**line["config"][f"strategy_{op}"])


if __name__ == "__main__":
    sys.exit(main())
