"""Shared test helpers: map library strategies onto the oracle's value-defining
parameters, and compare bit patterns."""
from __future__ import annotations

import numpy as np
import torch

from oracle import patterns as P


def oracle_strategy(st) -> P.Strategy:
    """The oracle Strategy with the same tree as a library ReduceStrategy."""
    return P.Strategy(s=st.split, T=st.chunk_threads, V=st.vec, thread_map=st.thread_map,
                      second=st.second, T2=st.threads2, compensated=bool(st.compensated),
                      pad=bool(st.pad))


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def bits(a) -> bytes:
    return np.ascontiguousarray(a).tobytes()


def _same_bits(got: np.ndarray, want: np.ndarray) -> bool:
    if got.dtype != want.dtype or got.shape != want.shape:
        return got.tobytes() == want.tobytes()
    if got.dtype.itemsize in (1, 2, 4, 8) and got.size:
        u = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[got.dtype.itemsize]
        return bool(np.array_equal(got.reshape(-1).view(u), want.reshape(-1).view(u)))
    return got.tobytes() == want.tobytes()


def assert_bits_equal(got, want, what=""):
    got = np.ascontiguousarray(got)
    want = np.ascontiguousarray(want)
    if got.shape != want.shape and got.size == want.size:
        want = want.reshape(got.shape)
    if not _same_bits(got, want):
        g = got.reshape(-1).view(np.uint32) if got.dtype == np.float32 else got.reshape(-1)
        w = want.reshape(-1).view(np.uint32) if want.dtype == np.float32 else want.reshape(-1)
        bad = np.nonzero(g != w)[0]
        i = int(bad[0]) if bad.size else -1
        raise AssertionError(f"{what}: {bad.size} mismatching elements, first at {i}: "
                             f"got {got.reshape(-1)[i]!r} want {want.reshape(-1)[i]!r}")
