"""c4: gradient references in FP64 -- TEST INFRASTRUCTURE ONLY.

Analytic adjoints follow from the functional forms: the adjoint of reduce(+) is
a broadcast of the incoming gradient, the adjoint of map(x*y) is a pointwise
product, split/join/transpose are re-indexings. They are pinned against central
finite differences of the FP64 forward functions below.
"""
from __future__ import annotations

import numpy as np


def dot_fwd(x, y):
    return float(np.dot(np.asarray(x, np.float64), np.asarray(y, np.float64)))


def dot_adjoint(x, y, g):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return g * y, g * x


def gemv_fwd(A, x):
    return np.asarray(A, np.float64) @ np.asarray(x, np.float64)


def gemv_adjoint(A, x, dy):
    A = np.asarray(A, np.float64)
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    return np.outer(dy, x), A.T @ dy  # dA = dy x^T, dx = A^T dy


def gemm_fwd(A, B):
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64)


def gemm_adjoint(A, B, dC):
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    dC = np.asarray(dC, np.float64)
    return dC @ B.T, A.T @ dC  # dA = dC B^T, dB = A^T dC


def central_fd(f, args, which, dout, h=1e-6):
    """d<dout, f(args)> / d args[which] by central differences, entry by entry."""
    args = [np.array(a, np.float64, copy=True) for a in args]
    a = args[which]
    grad = np.zeros_like(a)
    dout = np.asarray(dout, np.float64)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        old = a[idx]
        a[idx] = old + h
        fp = np.sum(np.asarray(f(*args)) * dout)
        a[idx] = old - h
        fm = np.sum(np.asarray(f(*args)) * dout)
        a[idx] = old
        grad[idx] = (fp - fm) / (2 * h)
    return grad
