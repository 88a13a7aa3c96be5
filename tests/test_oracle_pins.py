"""Pins of the CPU oracle against what the paper and the mathematics fix.

No GPU. The pattern evaluator (c1) is pinned by hand-derived association trees
(tests/golden/dot_trees.txt), by the paper's own strategy expression evaluated
through the primitives, by equational laws (Section 5.3), by closed forms and
exact integer results, and by the textbook error bound of a summation tree. The
loop-nest evaluator (c2) is pinned to c1 bit for bit; the FP64 references (c3)
and the gradient adjoints (c4) by exact sums, library routines and finite
differences.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import grads, loopnest, naive64
from oracle import patterns as P
from tests import treeparse as tp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dot_trees.txt")
U = 2.0 ** -24  # unit roundoff of binary32


def _strategy_from(fields):
    return P.Strategy(
        s=int(fields["s"]), T=int(fields.get("T", 1)), V=int(fields.get("V", 1)),
        thread_map=fields.get("thread_map", "interleaved"),
        second=fields.get("second", "seq"), T2=int(fields.get("T2", 32)),
        compensated=bool(int(fields.get("compensated", 0))), pad=bool(int(fields.get("pad", 0))))


def _sym_eval(entry):
    n = int(entry["n"])
    st = _strategy_from(tp.strategy_fields(entry["strategy"]))
    xs, ys = tp.symbols(n, "x"), tp.symbols(n, "y")
    if entry["kind"] == "dot":
        return P.dot_R(xs, ys, st, ar=P.Sym)
    return P.asum_R(xs, st, ar=P.Sym)


# --------------------------------------------------------------------------
# golden association trees
# --------------------------------------------------------------------------

_ENTRIES = tp.load_golden(GOLDEN)


@pytest.mark.parametrize("entry", _ENTRIES, ids=[e["name"] for e in _ENTRIES])
def test_golden_tree(entry):
    got = tp.normalise(_sym_eval(entry))
    want = tp.normalise(tp.parse(entry["expr"]))
    assert got == want


def test_golden_file_has_all_cases():
    names = {e["name"] for e in _ENTRIES}
    assert {"k1_naive", "k2_two_level_scaled", "interleaved_T2_V2", "contig_T2_V2",
            "tree_T4_second_tree_T2", "opencl_float4_scaled", "asum_interleaved",
            "padded_tail"} <= names


def test_planted_mistakes_are_caught(monkeypatch):
    """A wrong tree pairing or a wrong thread mapping in c1 fails a golden pin."""
    entries = {e["name"]: e for e in _ENTRIES}

    def adjacent_tree(q, add):  # pairs (2l, 2l+1) instead of (l, l + len/2)
        q = list(q)
        while len(q) > 1:
            q = [add(q[2 * l], q[2 * l + 1]) for l in range(len(q) // 2)]
        return q[0]

    def mismatch(entry):
        return tp.normalise(_sym_eval(entry)) != tp.normalise(tp.parse(entry["expr"]))

    with monkeypatch.context() as m:
        m.setattr(P, "halving_tree", adjacent_tree)
        assert mismatch(entries["tree_T4_second_tree_T2"])
    with monkeypatch.context() as m:
        m.setattr(P, "transpose", lambda xss: P.split(len(xss[0]), P.join(xss)))
        assert mismatch(entries["interleaved_T2_V2"])
    with monkeypatch.context() as m:  # drop the last chunk's reduce
        orig = P.second_level
        m.setattr(P, "second_level", lambda parts, st, ar: orig(parts[:-1], st, ar))
        assert mismatch(entries["k2_two_level_scaled"])


# --------------------------------------------------------------------------
# the paper's expressions evaluated through the primitives
# --------------------------------------------------------------------------


def _paper_eq2(xs, ys, per_thread, threads, ar):
    """Section 2.1's two-level dot, with split applied to the work-group chunk:
    reduce (+) 0 (join (mapWorkgroup (lambda zs1. mapLocal (lambda zs2.
    reduce (lambda x a. fst x * snd x + a) 0 zs2) (split per_thread zs1))
    (split (per_thread*threads) (zip xs ys))))."""
    inner = lambda zs2: P.reduce_(lambda x, a: ar.add(ar.mul(P.fst(x), P.snd(x)), a), ar.zero, zs2)
    groups = P.split(per_thread * threads, P.zip_(xs, ys))
    parts = P.join(P.mapWorkgroup(lambda zs1: P.mapLocal(inner, P.split(per_thread, zs1)), groups))
    return P.reduce_(lambda x, a: ar.add(a, x), ar.zero, parts)


def test_paper_eq2_is_thread_per_chunk_strategy_symbolic():
    xs, ys = tp.symbols(16, "x"), tp.symbols(16, "y")
    a = _paper_eq2(xs, ys, per_thread=4, threads=2, ar=P.Sym)
    b = P.dot_R(xs, ys, P.Strategy(s=4, T=1, V=1), ar=P.Sym)
    assert tp.normalise(a) == tp.normalise(b)


def test_paper_eq2_f32_bits():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, 64).astype(np.float32)
    y = rng.uniform(-1, 1, 64).astype(np.float32)
    a = _paper_eq2(list(x), list(y), per_thread=8, threads=4, ar=P.F32)
    b = P.dot_R(list(x), list(y), P.Strategy(s=8, T=1, V=1), ar=P.F32)
    c = loopnest.dot_f32(x, y, P.Strategy(s=8, T=1, V=1))
    assert np.float32(a).tobytes() == np.float32(b).tobytes() == np.float32(c).tobytes()


def test_k1_degenerate_strategy_equals_sequential_loop():
    """s = n, T = 1, V = 1 is the naive translation: one sequential left fold."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, 257).astype(np.float32)
    y = rng.uniform(-1, 1, 257).astype(np.float32)
    acc = np.float32(0)
    for i in range(x.size):  # the pseudo-C loop: accum = accum + tmp[i]
        acc = np.float32(acc + np.float32(x[i] * y[i]))
    st = P.Strategy(s=257, T=1, V=1)
    assert P.dot_K1(list(x), list(y)).tobytes() == acc.tobytes()
    assert np.float32(P.dot_R(list(x), list(y), st)).tobytes() == acc.tobytes()
    assert loopnest.dot_f32(x, y, st).tobytes() == acc.tobytes()


def test_t64_tree_splits_into_two_warps():
    """With 64 threads the tree is two 32-lane halving trees, then their sum."""
    xs = tp.symbols(64, "x")
    t = tp.normalise(P.asum_R(xs, P.Strategy(s=64, T=64, V=1), ar=P.Sym))

    def leaves(node):
        if isinstance(node, str):
            return {node}
        if node[0] == "abs":
            return leaves(node[1])
        return leaves(node[1]) | leaves(node[2])

    assert t[0] == "+"
    halves = sorted([leaves(t[1]), leaves(t[2])], key=lambda s: min(int(v[1:]) for v in s))
    assert halves[0] == {f"x{i}" for i in range(32)}
    assert halves[1] == {f"x{i}" for i in range(32, 64)}
    # deepest pairs of warp 0 are lanes (l, l+16) at the first halving step
    bottom = set()

    def collect(node, depth):
        if isinstance(node, str) or node[0] == "abs":
            return
        if depth == 6:
            bottom.add(frozenset(leaves(node)))
        collect(node[1], depth + 1)
        collect(node[2], depth + 1)

    collect(t, 1)
    assert frozenset({"x0", "x16"}) in bottom and frozenset({"x33", "x49"}) in bottom


# --------------------------------------------------------------------------
# equational laws (Section 5.3 layout agreement, map and reduce properties)
# --------------------------------------------------------------------------


def test_layout_laws():
    xs = list(range(24))
    for n in (1, 2, 3, 4, 6, 8, 12, 24):
        assert P.join(P.split(n, xs)) == xs
    xss = [list(range(i * 4, i * 4 + 4)) for i in range(6)]
    assert P.split(4, P.join(xss)) == xss
    assert P.transpose(P.transpose(xss)) == xss
    assert P.asScalar(P.asVector(4, xs)) == xs
    ys = [v * 10 for v in xs]
    z = P.zip_(xs, ys)
    assert P.map_(P.fst, z) == xs and P.map_(P.snd, z) == ys
    f, g = (lambda v: v + 3), (lambda v: v * 7)
    assert P.map_(f, P.map_(g, xs)) == P.map_(lambda v: f(g(v)), xs)
    # split of a zip is a zip of splits (index rule of zip under split)
    assert P.split(6, z) == [P.zip_(a, b) for a, b in zip(P.split(6, xs), P.split(6, ys))]
    for bad in (5, 7):
        with pytest.raises(ValueError):
            P.split(bad, xs)


def test_reduce_of_join_for_associative_op():
    rng = np.random.default_rng(2)
    v = [int(a) for a in rng.integers(-1000, 1000, 96)]
    whole = P.reduce_(lambda x, a: a + x, 0, v)
    for n in (1, 2, 3, 8, 12, 32, 96):
        chunks = P.split(n, v)
        assert P.reduce_(lambda x, a: a + x, 0, P.map_(lambda c: P.reduce_(lambda x, a: a + x, 0, c),
                                                       chunks)) == whole


STRATS = [
    P.Strategy(s=64, T=1, V=1),
    P.Strategy(s=64, T=1, V=4),
    P.Strategy(s=128, T=32, V=1),
    P.Strategy(s=256, T=32, V=4, thread_map="contig"),
    P.Strategy(s=512, T=64, V=2),
    P.Strategy(s=1024, T=128, V=4, second="tree", T2=32),
    P.Strategy(s=256, T=64, V=4, second="tree", T2=64, thread_map="contig"),
    P.Strategy(s=512, T=32, V=16),
    P.Strategy(s=256, T=32, V=8, pad=True),
]


@pytest.mark.parametrize("st", STRATS, ids=lambda s: f"s{s.s}T{s.T}V{s.V}{s.thread_map[0]}{s.second}")
def test_integer_valued_inputs_are_exact(st):
    """Small integers are exact in binary32 under any bracketing: every element
    must be counted exactly once."""
    rng = np.random.default_rng(3)
    n = st.s * 4 - (37 if st.pad else 0)
    x = rng.integers(-8, 9, n).astype(np.float32)
    y = rng.integers(-8, 9, n).astype(np.float32)
    want = int(np.dot(x.astype(np.int64), y.astype(np.int64)))
    assert float(P.dot_R(list(x), list(y), st)) == want
    assert float(loopnest.dot_f32(x, y, st)) == want
    assert float(P.asum_R(list(x), st)) == float(np.abs(x.astype(np.int64)).sum())
    assert float(loopnest.asum_f32(x, st)) == float(np.abs(x.astype(np.int64)).sum())
    assert loopnest.dot_i32(x.astype(np.int32), y.astype(np.int32), st) == want


def test_index_coverage_closed_form():
    """x = 1, y_i = i: the dot is n(n-1)/2 exactly (n(n-1)/2 < 2^24)."""
    n = 4096
    x = np.ones(n, np.float32)
    y = np.arange(n, dtype=np.float32)
    for st in (P.Strategy(s=1024, T=32, V=4), P.Strategy(s=4096, T=256, V=4, thread_map="contig"),
               P.Strategy(s=512, T=128, V=4, second="tree", T2=128)):
        assert float(loopnest.dot_f32(x, y, st)) == n * (n - 1) / 2
    assert float(loopnest.dot_f32(x, x, P.Strategy(s=64, T=32, V=2))) == n


def test_int32_dot_exact_against_bruteforce():
    rng = np.random.default_rng(4)
    x = rng.integers(-100, 101, 5000).astype(np.int32)
    y = rng.integers(-100, 101, 5000).astype(np.int32)
    want = sum(int(a) * int(b) for a, b in zip(x, y))
    for st in (P.Strategy(s=1000, T=1, V=1), P.Strategy(s=128, T=32, V=4, pad=True),
               P.Strategy(s=256, T=64, V=4, second="tree", T2=32, pad=True)):
        assert loopnest.dot_i32(x, y, st) == want
    assert P.dot_R(list(x), list(y), P.Strategy(s=1000, T=1, V=1), ar=P.Int) == want


def test_int32_dot_beyond_int32_range():
    """Sums past 2^31 need the int64 accumulator (design reading of int32 dot)."""
    n = 1 << 20
    x = np.full(n, 100, np.int32)
    y = np.full(n, 100, np.int32)
    assert loopnest.dot_i32(x, y, P.Strategy(s=8192, T=256, V=4)) == 10000 * n


# --------------------------------------------------------------------------
# c2 == c1 bit for bit
# --------------------------------------------------------------------------

C2_STRATS = STRATS + [
    P.Strategy(s=128, T=32, V=4, compensated=True),
    P.Strategy(s=256, T=64, V=2, compensated=True, second="tree", T2=32),
    P.Strategy(s=96, T=32, V=1, pad=True, compensated=True),
]


@pytest.mark.parametrize("st", C2_STRATS, ids=lambda s: f"s{s.s}T{s.T}V{s.V}{s.thread_map[0]}{s.second}{'k' if s.compensated else ''}")
def test_loopnest_bits_equal_pattern_evaluator(st):
    rng = np.random.default_rng(st.s + st.T)
    n = st.s * 3 - (5 if st.pad else 0)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = rng.uniform(-1, 1, n).astype(np.float32)
    x[::7] *= 1e-3  # spread magnitudes so that bracketing changes the bits
    a = np.float32(P.dot_R(list(x), list(y), st))
    b = loopnest.dot_f32(x, y, st)
    assert a.tobytes() == b.tobytes()
    a = np.float32(P.asum_R(list(x), st))
    b = loopnest.asum_f32(x, st)
    assert a.tobytes() == b.tobytes()


def test_bracketing_changes_bits():
    """The pins above are meaningful: different strategies give different bits."""
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, 1 << 14).astype(np.float32)
    y = rng.uniform(-1, 1, 1 << 14).astype(np.float32)
    vals = {loopnest.dot_f32(x, y, st).tobytes() for st in (
        P.Strategy(s=1 << 14, T=1, V=1), P.Strategy(s=1024, T=32, V=4),
        P.Strategy(s=1024, T=256, V=4), P.Strategy(s=1024, T=256, V=4, thread_map="contig"))}
    assert len(vals) >= 3


def test_partials_are_chunk_results():
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, 4096).astype(np.float32)
    y = rng.uniform(-1, 1, 4096).astype(np.float32)
    st = P.Strategy(s=512, T=64, V=4)
    parts = loopnest.dot_f32_partials(x, y, st)
    for c in range(8):
        one = loopnest.dot_f32(x[c * 512:(c + 1) * 512], y[c * 512:(c + 1) * 512], st)
        assert parts[c].tobytes() == one.tobytes()


# --------------------------------------------------------------------------
# error bounds against the exact value
# --------------------------------------------------------------------------


def _tree_depth(st, n):
    C = -(-n // st.s)
    R = st.s // (st.T * st.V)
    d = R + st.V + int(math.log2(st.T))
    if st.second == "seq":
        d += C
    else:
        d += -(-C // st.T2) + int(math.log2(st.T2))
    return d + 1  # the product's rounding


@pytest.mark.parametrize("st", [P.Strategy(s=8192, T=256, V=4), P.Strategy(s=1024, T=32, V=4),
                                P.Strategy(s=65536, T=1024, V=4, second="tree", T2=256),
                                P.Strategy(s=4096, T=1, V=1)])
def test_within_summation_error_bound(st):
    """|fl(dot) - dot| <= gamma_d * sum|x_i y_i| with d the additions on the
    longest path (Higham, Accuracy and Stability, Section 4.2)."""
    n = 1 << 18
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = rng.uniform(-1, 1, n).astype(np.float32)
    exact = naive64.dot_exact(x, y)
    d = _tree_depth(st, n)
    bound = d * U / (1 - d * U) * naive64.abs_dot_f64(x, y)
    assert abs(float(loopnest.dot_f32(x, y, st)) - exact) <= bound
    exact_a = naive64.asum_exact(x)
    bound_a = d * U / (1 - d * U) * exact_a
    assert abs(float(loopnest.asum_f32(x, st)) - exact_a) <= bound_a


def test_dropped_term_violates_bound():
    n = 1 << 16
    rng = np.random.default_rng(8)
    x = rng.uniform(0.5, 1, n).astype(np.float32)
    y = rng.uniform(0.5, 1, n).astype(np.float32)
    st = P.Strategy(s=1024, T=32, V=4)
    exact = naive64.dot_exact(x[:-1], y[:-1])  # the sum without the last term
    bound = _tree_depth(st, n) * U * naive64.abs_dot_f64(x, y)
    assert abs(float(loopnest.dot_f32(x, y, st)) - exact) > bound


def test_kahan_compensation():
    """Compensated sums obey Kahan's bound |E| <= (2u + O(d u^2)) sum|x_i|
    (Higham, Section 4.3) and, on positive data whose plain sequential sum
    drifts by tens of ulps, land within 2 ulps of the exact value."""
    n = 1 << 16
    rng = np.random.default_rng(10)
    big = rng.uniform(1e3, 1e4, n // 2).astype(np.float32)
    x0 = np.concatenate([big, -big]).astype(np.float32)
    x0 += rng.uniform(-1e-3, 1e-3, n).astype(np.float32)
    x0 = x0[rng.permutation(n)].astype(np.float32)
    x1 = (rng.uniform(0, 1, n) * np.exp(rng.uniform(-10, 10, n))).astype(np.float32)
    y = np.ones(n, np.float32)
    for x in (x0, x1):
        exact = naive64.dot_exact(x, y)
        scale = naive64.abs_dot_f64(x, y)
        for base in (P.Strategy(s=n, T=1, V=1), P.Strategy(s=4096, T=1, V=1),
                     P.Strategy(s=1024, T=64, V=4),
                     P.Strategy(s=2048, T=128, V=2, second="tree", T2=32)):
            comp = float(loopnest.dot_f32(x, y, P.Strategy(**{**base.__dict__, "compensated": True})))
            d = _tree_depth(base, n)
            assert abs(comp - exact) <= (2 * U + d * d * U * U) * scale
            if x is x1:
                assert abs(comp - exact) <= 2 * U * abs(exact)
    for base in (P.Strategy(s=n, T=1, V=1), P.Strategy(s=4096, T=1, V=1)):
        exact = naive64.dot_exact(x1, y)
        plain = float(loopnest.dot_f32(x1, y, base))
        assert abs(plain - exact) > 20 * U * abs(exact)


# --------------------------------------------------------------------------
# maps, GEMV, GEMM
# --------------------------------------------------------------------------


def test_scal_and_dot_bwd():
    rng = np.random.default_rng(12)
    x = rng.integers(-1000, 1000, 1000).astype(np.float32)
    y = rng.uniform(-1, 1, 1000).astype(np.float32)
    assert np.array_equal(loopnest.scal_f32(1.5, x), (x.astype(np.float64) * 1.5).astype(np.float32))
    assert np.array_equal(loopnest.scal_f32(2.0, y), y + y)
    assert np.array_equal(np.array(P.scal(np.float32(2.0), list(y)), np.float32), y + y)
    dx, dy = loopnest.dot_bwd_f32(x, y, 2.0)
    assert np.array_equal(dx, y + y) and np.array_equal(dy, x + x)
    px, py = P.dot_bwd(x[:50], y[:50], np.float32(0.75))
    qx, qy = loopnest.dot_bwd_f32(x[:50], y[:50], 0.75)
    assert np.array_equal(np.array(px, np.float32), qx) and np.array_equal(np.array(py, np.float32), qy)


def test_gemv_pins():
    rng = np.random.default_rng(13)
    M, N = 24, 256
    st = P.Strategy(s=128, T=32, V=4)
    x = rng.uniform(-1, 1, N).astype(np.float32)
    eye = np.eye(M, N, dtype=np.float32)
    assert np.array_equal(loopnest.gemv_f32(eye, x, st), x[:M])
    A = rng.integers(-5, 6, (M, N)).astype(np.float32)
    xi = rng.integers(-5, 6, N).astype(np.float32)
    assert np.array_equal(loopnest.gemv_f32(A, xi, st), (A.astype(np.int64) @ xi.astype(np.int64)).astype(np.float32))
    # ragged rows with padding: each row is the padded dot of the pattern evaluator
    Ar = rng.normal(0, 1, (5, 200)).astype(np.float32)
    xr = rng.uniform(-1, 1, 200).astype(np.float32)
    stp = P.Strategy(s=128, T=32, V=4, pad=True)
    assert np.array(P.gemv_R(Ar, list(xr), stp), np.float32).tobytes() == loopnest.gemv_f32(Ar, xr, stp).tobytes()
    A = rng.normal(0, 1, (M, N)).astype(np.float32)
    c1 = np.array(P.gemv_R(A, list(x), st), np.float32)
    c2 = loopnest.gemv_f32(A, x, st)
    assert c1.tobytes() == c2.tobytes()
    ref = naive64.gemv_f64(A, x)
    bound = _tree_depth(st, N) * U * naive64.gemv_abs_f64(A, x)
    assert np.all(np.abs(c2 - ref) <= bound)


def test_gemv_bwd_pins():
    rng = np.random.default_rng(14)
    M, N = 70, 40
    A = rng.normal(0, 1, (M, N)).astype(np.float32)
    dy = rng.uniform(-1, 1, M).astype(np.float32)
    x = rng.uniform(-1, 1, N).astype(np.float32)
    for Rs in (1, 16, 32, 70, 128):
        c1 = np.array(P.gemv_bwd_dx(A, list(dy), Rs), np.float32)
        c2 = loopnest.gemv_bwd_dx_f32(A, dy, Rs)
        assert c1.tobytes() == c2.tobytes()
        ref = A.astype(np.float64).T @ dy.astype(np.float64)
        assert np.all(np.abs(c2 - ref) <= (M + 2) * U * (np.abs(A).T @ np.abs(dy)))
    eye = np.eye(M, N, dtype=np.float32)
    assert np.array_equal(loopnest.gemv_bwd_dx_f32(eye, dy, 32), dy[:N])
    dA = loopnest.gemv_bwd_dA_f32(x, dy)
    assert dA.tobytes() == np.array(P.gemv_bwd_dA(list(x), list(dy)), np.float32).tobytes()
    assert np.array_equal(dA, np.outer(dy, x).astype(np.float32))  # one rounding of an exact product


def test_fma_closed_form():
    a = np.float32(1 + 2 ** -23)
    b = np.float32(1 - 2 ** -23)
    # a*b = 1 - 2^-46 exactly: fused keeps it, separate rounding loses it
    assert float(P.F32.fma(a, b, np.float32(-1.0))) == -(2.0 ** -46)
    assert float(P.F32.add(P.F32.mul(a, b), np.float32(-1.0))) == 0.0
    assert float(P.F32.fma(np.float32(3), np.float32(5), np.float32(7))) == 22.0
    z = P.F32.fma(np.float32(-0.0), np.float32(1.0), np.float32(-0.0))
    assert z == 0 and math.copysign(1.0, float(z)) < 0
    tiny = P.F32.fma(np.float32(-1e-30), np.float32(1e-30), np.float32(0.0))
    assert tiny == 0 and math.copysign(1.0, float(tiny)) < 0  # underflow keeps the sign


def test_gemm_fold_pins():
    rng = np.random.default_rng(15)
    M, N, K = 9, 11, 37
    A = rng.normal(0, 1, (M, K)).astype(np.float32)
    B = rng.normal(0, 1, (K, N)).astype(np.float32)
    for fma in (False, True):
        c1 = np.array(P.gemm_fold(A, B, fma), np.float32)
        c2 = loopnest.gemm_f32(A, B, False, False, fma)
        assert c1.tobytes() == c2.tobytes()
        # transposed storage gives the same values
        c3 = loopnest.gemm_f32(np.ascontiguousarray(A.T), np.ascontiguousarray(B.T), True, True, fma)
        assert c3.tobytes() == c2.tobytes()
        ref = naive64.gemm_f64(A, B)
        assert np.all(np.abs(c2 - ref) <= (K + 1) * U * (np.abs(A) @ np.abs(B)))
    eye = np.eye(K, N, dtype=np.float32)
    for fma in (False, True):
        assert np.array_equal(loopnest.gemm_f32(A, eye, False, False, fma), A[:, :N])


def test_gemm_fma_differs_from_separate():
    rng = np.random.default_rng(16)
    A = rng.normal(0, 1, (16, 64)).astype(np.float32)
    B = rng.normal(0, 1, (64, 16)).astype(np.float32)
    assert loopnest.gemm_f32(A, B, contract_fma=True).tobytes() != loopnest.gemm_f32(A, B, contract_fma=False).tobytes()


def test_bf16_round_matches_torch_cast():
    rng = np.random.default_rng(17)
    a = rng.normal(0, 3, 10000).astype(np.float32)
    a[:4] = [0.0, -0.0, 1e-40, -3.0e38]
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(naive64.bf16_round(a), want)


# --------------------------------------------------------------------------
# gradients
# --------------------------------------------------------------------------


def test_gradient_adjoints_match_finite_differences():
    rng = np.random.default_rng(18)
    x = rng.uniform(-1, 1, 7)
    y = rng.uniform(-1, 1, 7)
    gx, gy = grads.dot_adjoint(x, y, 1.3)
    assert np.allclose(gx, grads.central_fd(grads.dot_fwd, [x, y], 0, 1.3), atol=1e-7)
    assert np.allclose(gy, grads.central_fd(grads.dot_fwd, [x, y], 1, 1.3), atol=1e-7)
    A = rng.normal(0, 1, (5, 6))
    xv = rng.uniform(-1, 1, 6)
    dy = rng.uniform(-1, 1, 5)
    dA, dx = grads.gemv_adjoint(A, xv, dy)
    assert np.allclose(dA, grads.central_fd(grads.gemv_fwd, [A, xv], 0, dy), atol=1e-7)
    assert np.allclose(dx, grads.central_fd(grads.gemv_fwd, [A, xv], 1, dy), atol=1e-7)
    B = rng.normal(0, 1, (6, 4))
    dC = rng.normal(0, 1, (5, 4))
    gA, gB = grads.gemm_adjoint(A, B, dC)
    assert np.allclose(gA, grads.central_fd(grads.gemm_fwd, [A, B], 0, dC), atol=1e-6)
    assert np.allclose(gB, grads.central_fd(grads.gemm_fwd, [A, B], 1, dC), atol=1e-6)


@pytest.mark.parametrize("st", [P.Strategy(s=256, T=32, V=4), P.Strategy(s=512, T=64, V=2, thread_map="contig"),
                                P.Strategy(s=1024, T=128, V=4, second="tree", T2=64, pad=True),
                                P.Strategy(s=256, T=32, V=4, compensated=True, pad=True),
                                P.Strategy(s=512, T=64, V=1, second="tree", T2=32, compensated=True)],
                         ids=["plain", "contig", "tree-pad", "kahan-pad", "kahan-tree"])
def test_loopnest_threads_do_not_change_bits(st):
    """c2 with its units (chunks, rows, columns, GEMM entries) on several host
    threads equals c2 on one thread bit for bit: every fold across units still
    runs on one thread in the strategy's order."""
    rng = np.random.default_rng(21)
    n = 64 * st.s - (37 if st.pad else 0)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = rng.uniform(-1, 1, n).astype(np.float32)
    xi = rng.integers(-100, 101, n).astype(np.int32)
    A = rng.standard_normal((40, 300)).astype(np.float32)
    B = rng.standard_normal((300, 50)).astype(np.float32)
    xv = rng.uniform(-1, 1, 300).astype(np.float32)
    dy = rng.uniform(-1, 1, 40).astype(np.float32)
    gst = P.Strategy(s=64, T=8, V=4, pad=True, compensated=st.compensated)

    def run():
        return [loopnest.dot_f32(x, y, st).tobytes(), loopnest.asum_f32(x, st).tobytes(),
                loopnest.dot_f32_partials(x, y, P.Strategy(s=st.s, T=st.T, V=st.V, thread_map=st.thread_map,
                                                          pad=st.pad)).tobytes(),
                loopnest.dot_i32(xi, xi, st), loopnest.gemv_f32(A, xv, gst).tobytes(),
                loopnest.gemv_bwd_dx_f32(A, dy, 7).tobytes(), loopnest.gemv_bwd_dA_f32(xv, dy).tobytes(),
                loopnest.gemm_f32(A, B).tobytes(), loopnest.scal_f32(1.5, x).tobytes(),
                b"".join(a.tobytes() for a in loopnest.dot_bwd_f32(x, y, 0.75))]

    old = loopnest.set_threads(1)
    try:
        one = run()
        loopnest.set_threads(8)
        many = run()
    finally:
        loopnest.set_threads(old)
    assert one == many


@pytest.mark.parametrize("kind", ["dot", "asum"])
@pytest.mark.parametrize("tm,V", [("interleaved", 1), ("interleaved", 4), ("contig", 2), ("contig", 4)])
def test_lane_partials_equal_pattern_evaluator(kind, tm, V):
    """c2's un-reduced lane partials (Section 6's kernel stores them) equal c1's
    join (mapWorkgroup (mapLocal (reduce lanewise))) over asVector V, and
    folding each thread's lanes in lane order and reducing the threads by the
    block tree gives c2's chunk partials."""
    rng = np.random.default_rng(77)
    n, s, T = 4096, 512, 16
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y = rng.uniform(-1, 1, n).astype(np.float32)
    st = P.Strategy(s=s, T=T, V=V, thread_map=tm)
    got = loopnest.lane_partials_f32(kind, x, y if kind == "dot" else None, st)
    F = P.F32
    zero = (F.zero,) * V
    if kind == "dot":
        items = P.zip_(P.asVector(V, list(x)), P.asVector(V, list(y)))
        g = lambda p: tuple(F.mul(a, b) for a, b in zip(p[0], p[1]))
    else:
        items = P.asVector(V, list(x))
        g = lambda v: tuple(F.abs(a) for a in v)
    cols = (lambda ch: P.transpose(P.split(T, ch))) if tm == "interleaved" else (lambda ch: P.split(len(ch) // T, ch))
    want = P.asScalar(P.join(P.mapWorkgroup(
        lambda ch: P.mapLocal(lambda col: P.reduce_(lambda v, a: tuple(F.add(p, q) for p, q in zip(a, g(v))),
                                                     zero, col), cols(ch)),
        P.split(s // V, items))))
    assert np.asarray(want, np.float32).tobytes() == got.tobytes()
    if kind == "dot":
        lanes = got.reshape(n // s, T, V)
        chunk = []
        for c in range(n // s):
            th = [P.reduce_(lambda v, a: F.add(a, v), F.zero, list(lanes[c, t])) for t in range(T)]
            chunk.append(P.halving_tree(P.join([[P.halving_tree(g_, F.add)] for g_ in P.split(min(32, T), th)]),
                                        F.add))
        assert np.asarray(chunk, np.float32).tobytes() == loopnest.dot_f32_partials(x, y, st).tobytes()
