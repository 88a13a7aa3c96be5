"""Seeded inputs of the five workloads (sizes and distributions of the paper's
BLAS-1/BLAS-2 benchmarks, Section 7, plus the batched and GEMM cases).

Each function draws every tensor of one workload from a single torch generator
seeded with the workload's seed, in a fixed order, on the requested device.
"""
from __future__ import annotations

import math

import torch

from . import generator, loguniform_lengths

DOT_N = 1 << 20          # dot, n = 1,048,576, seed 0
DOT_SPLIT = 8192         # split(8192): 128 chunks
BW_N = 1 << 26           # asum / scal / dot, 256 MiB per vector, seed 1
SCAL_A = 1.5
GEMV_M = GEMV_N = 8192   # GEMV 8192 x 8192, seed 2
GEMM_MNK = 4096          # GEMM 4096^3, seed 4


def dot_f32(device="cpu", n=DOT_N, seed=0):
    g = generator(seed, device)
    x = torch.rand(n, generator=g, device=device).mul_(2).sub_(1)
    y = torch.rand(n, generator=g, device=device).mul_(2).sub_(1)
    return x, y


def dot_i32(device="cpu", n=DOT_N, seed=0):
    g = generator(seed, device)
    x = torch.randint(-100, 101, (n,), generator=g, device=device, dtype=torch.int32)
    y = torch.randint(-100, 101, (n,), generator=g, device=device, dtype=torch.int32)
    return x, y


def bandwidth(device="cpu", n=BW_N, seed=1):
    """x, y ~ U[-1, 1) for asum / scal / dot."""
    return dot_f32(device, n, seed)


def gemv(device="cpu", M=GEMV_M, N=GEMV_N, seed=2):
    """A ~ N(0, 1/N) (M x N row-major), x, dy ~ U[-1, 1)."""
    g = generator(seed, device)
    A = torch.randn(M, N, generator=g, device=device).mul_(1.0 / math.sqrt(N))
    x = torch.rand(N, generator=g, device=device).mul_(2).sub_(1)
    dy = torch.rand(M, generator=g, device=device).mul_(2).sub_(1)
    return A, x, dy


def gemm(device="cpu", M=GEMM_MNK, N=GEMM_MNK, K=GEMM_MNK, seed=4):
    """A (M x K), B (K x N), dC (M x N) ~ N(0, 1)."""
    g = generator(seed, device)
    A = torch.randn(M, K, generator=g, device=device)
    B = torch.randn(K, N, generator=g, device=device)
    dC = torch.randn(M, N, generator=g, device=device)
    return A, B, dC


def batched_shapes(seed=3, n_dots=4096, n_gemvs=512, lo=256, hi=65536, col_lo=256, col_hi=4096):
    """Lengths of the dot instances, and (rows, cols) of the GEMV instances,
    log-uniform in [lo, hi] (cols in [col_lo, col_hi]), from the CPU generator."""
    dots = loguniform_lengths(n_dots, seed, lo, hi)
    rows = loguniform_lengths(n_gemvs, seed + 1000, lo, hi)
    cols = loguniform_lengths(n_gemvs, seed + 2000, col_lo, col_hi)
    return dots, rows, cols
