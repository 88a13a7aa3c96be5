"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws numbers. It holds none of the map/reduce arithmetic: the
CUDA path and the CPU oracle each compute from the bytes produced here, and the
same bytes are handed to both (device tensors are copied to the host for the
oracle).

Recipes (shapes and distributions of the workloads the paper evaluates in its
experimental section: BLAS-1 vectors of 16M/128M elements, GEMV on 4096^2 and
8192^2 matrices, scaled to the sizes used here):

* ``uniform_f32``  -- U[-1, 1) float32, ``rand * 2 - 1``.
* ``randint_i32``  -- integers uniform in {lo .. hi}, int32.
* ``normal_f32``   -- N(0, std^2) float32, ``randn * std``.
* ``loguniform_lengths`` -- ``floor(exp(U(ln lo, ln hi)))`` int64, drawn on the
  CPU generator so lengths do not depend on the device.

Every generator takes an explicit ``seed`` and ``device``; the torch generator is
created on that device, so a CPU draw and a CUDA draw with one seed give
different (but each reproducible) bytes.
"""
from __future__ import annotations

import math

import torch

__all__ = [
    "uniform_f32",
    "randint_i32",
    "normal_f32",
    "loguniform_lengths",
    "generator",
]


def generator(seed: int, device="cpu") -> torch.Generator:
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    return g


def uniform_f32(shape, seed: int, device="cpu", g: torch.Generator | None = None) -> torch.Tensor:
    """U[-1, 1) float32 of ``shape``."""
    g = g or generator(seed, device)
    t = torch.rand(shape, generator=g, device=device, dtype=torch.float32)
    return t.mul_(2.0).sub_(1.0)


def randint_i32(shape, seed: int, lo: int = -100, hi: int = 100, device="cpu",
                g: torch.Generator | None = None) -> torch.Tensor:
    """Integers uniform in {lo .. hi} (inclusive), int32."""
    g = g or generator(seed, device)
    return torch.randint(lo, hi + 1, shape, generator=g, device=device, dtype=torch.int32)


def normal_f32(shape, seed: int, std: float = 1.0, device="cpu",
               g: torch.Generator | None = None) -> torch.Tensor:
    """N(0, std^2) float32 of ``shape``."""
    g = g or generator(seed, device)
    t = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    if std != 1.0:
        t.mul_(std)
    return t


def loguniform_lengths(count: int, seed: int, lo: int, hi: int) -> torch.Tensor:
    """``count`` int64 lengths ``floor(exp(U(ln lo, ln hi)))`` on the CPU generator."""
    g = generator(seed, "cpu")
    u = torch.rand(count, generator=g, dtype=torch.float64)
    v = torch.exp(u * (math.log(hi) - math.log(lo)) + math.log(lo))
    return torch.clamp(torch.floor(v), lo, hi).to(torch.int64)
