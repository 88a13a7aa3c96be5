"""c3: exact and FP64 reference values -- TEST INFRASTRUCTURE ONLY.

These are the plain definitions the strategies must agree with up to rounding:
dot = sum_i x_i y_i (the declarative reading of the first dot expression in
Section 2.1), asum = sum_i |x_i|, gemv y_i = sum_j A_ij x_j, gemm C = A B.

Products of two binary32 numbers are exact in binary64 (24 + 24 < 53 bits), so
``math.fsum`` of the float64 products is the correctly rounded exact dot
product; ``dot_exact`` is therefore the true value to within half an ulp of
float64, not an approximation of it.
"""
from __future__ import annotations

import math

import numpy as np


def dot_exact(x, y) -> float:
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return math.fsum((x * y).tolist())


def asum_exact(x) -> float:
    return math.fsum(np.abs(np.asarray(x, np.float64)).tolist())


def dot_f64(x, y) -> float:
    return float(np.dot(np.asarray(x, np.float64), np.asarray(y, np.float64)))


def abs_dot_f64(x, y) -> float:
    """sum_i |x_i y_i|: the scale of the normwise error bound."""
    return float(np.abs(np.asarray(x, np.float64) * np.asarray(y, np.float64)).sum())


def gemv_f64(A, x):
    return np.asarray(A, np.float64) @ np.asarray(x, np.float64)


def gemv_abs_f64(A, x):
    return np.abs(np.asarray(A, np.float64)) @ np.abs(np.asarray(x, np.float64))


def gemm_f64(A, B):
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64)


def bf16_round(a) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even) and return them as float64.

    bfloat16 keeps the top 16 bits of the binary32 pattern; rounding adds
    0x7FFF plus the lowest kept bit before truncation (NaN is not expected here).
    """
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
