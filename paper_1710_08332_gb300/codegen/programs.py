"""The paper's running examples as phrases (Sections 2.1 and 7): each program
is one or two kernels, the second folding the first one's partial results.

    dot   partials = join (mapWorkgroup (lambda chunk.
                       mapLocal (lambda col. reduceSeq (+) 0 (map (*) col))
                                (columns chunk)) (split s (zip x y)))
          result   = reduceSeq (+) 0 partials
    asum  the same with map abs
    scal  mapGlobal (lambda v. a * v) x
    dA    mapWorkgroup (lambda d. mapLocal (lambda v. d * v) x) dy
    dx    partials = mapWorkgroup (lambda (rows, dys). mapLocal (lambda col.
                       reduceSeq (+) 0 (map (*) (zip col dys))) (transpose rows))
                       (zip (split R A) (split R dy));  dx = mapGlobal fold (columns of partials)
    gemv  partials = join (mapWorkgroup (lambda row.
                       mapLocal (lambda col. reduceSeq (+) 0 (map (*) col))
                                (columns (zip row x))) A)
          y        = mapGlobal (lambda p. reduceSeq (+) 0 p) (split T partials)

With V > 1 the streams are read as ``asVector V`` (128-bit loads at V = 4),
the fold runs lane-wise on num<V> and each thread's V lane sums are written
out un-reduced; the next kernel folds them like any other partials.
``columns`` is the thread mapping: interleaved (``transpose (split T c)``:
thread t folds items r*T + t) or contiguous (``split (len/T) c``: thread t folds
items t*R .. t*R + R - 1, the paper's form). The map (*) is fused into the
fold's step function, as the paper's strategies do.
"""
from __future__ import annotations

from . import phrase as P


def columns(chunk, T: int, thread_map: str):
    n = chunk.type.n
    if n % T:
        raise ValueError(f"{n} items do not split over {T} threads")
    if thread_map == "interleaved":
        return P.transpose(P.split(T, chunk))
    if thread_map == "contig":
        return P.split(n // T, chunk)
    raise ValueError(f"unknown thread map {thread_map}")


def _vec(e, V):
    return e if V == 1 else P.asVector(V, e)


def _zero(V):
    return P.lit(0.0) if V == 1 else P.vlit(0.0, V)


def dot_partials(n: int, s: int, T: int, thread_map: str = "interleaved", V: int = 1):
    """(phrase, inputs): the per-thread partial sums of x . y (C*T of them, C = n/s).
    With V > 1 the inputs are read as asVector V and each thread keeps V lane
    sums, written out un-reduced (Section 6's float4 kernel): C*T*V partials."""
    x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
    e = P.join(P.mapWorkgroup(
        lambda chunk: P.mapLocal(
            lambda col: P.reduceSeq(lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p))), _zero(V), col),
            columns(chunk, T, thread_map)),
        P.split(s // V, P.zip_(_vec(x, V), _vec(y, V)))))
    return e, [x, y]


def asum_partials(n: int, s: int, T: int, thread_map: str = "interleaved", V: int = 1):
    x = P.inp("x", P.arr(n, P.F32))
    e = P.join(P.mapWorkgroup(
        lambda chunk: P.mapLocal(
            lambda col: P.reduceSeq(lambda v, acc: P.add(acc, P.abs_(v)), _zero(V), col),
            columns(chunk, T, thread_map)),
        P.split(s // V, _vec(x, V))))
    return e, [x]


def fold_all(m: int):
    """The second kernel: reduceSeq (+) 0 over m partials."""
    p = P.inp("p", P.arr(m, P.F32))
    return P.reduceSeq(lambda v, acc: P.add(acc, v), 0.0, p), [p]


def scal(n: int, a: float, V: int = 1):
    x = P.inp("x", P.arr(n, P.F32))
    if V == 1:
        return P.mapGlobal(lambda v: P.mul(P.lit(a), v), x), [x]
    return P.asScalar(P.mapGlobal(lambda v: P.mul(P.vlit(a, V), v), P.asVector(V, x))), [x]


def gemv_partials(M: int, N: int, T: int, thread_map: str = "interleaved", V: int = 1):
    """Per-row, per-thread partials of A x (M*T of them, or M*T*V lane sums)."""
    A, x = P.inp("A", P.arr(M, N, P.F32)), P.inp("x", P.arr(N, P.F32))
    e = P.join(P.mapWorkgroup(
        lambda row: P.mapLocal(
            lambda col: P.reduceSeq(lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p))), _zero(V), col),
            columns(P.zip_(_vec(row, V), _vec(x, V)), T, thread_map)),
        A))
    return e, [A, x]


def fold_rows(M: int, T: int):
    """The GEMV second kernel: y_i = reduceSeq (+) 0 over row i's T partials."""
    p = P.inp("p", P.arr(M * T, P.F32))
    return P.mapGlobal(lambda r: P.reduceSeq(lambda v, acc: P.add(acc, v), 0.0, r), P.split(T, p)), [p]


def fold_cols(rows: int, g: int):
    """A folding kernel over strided groups: rows outputs, output j the fold of
    p[j], p[rows + j], .., p[(g - 1) rows + j] in that order (the transpose of
    split rows: consecutive threads read consecutive partials)."""
    p = P.inp("p", P.arr(rows * g, P.F32))
    return P.mapGlobal(lambda col: P.reduceSeq(lambda v, acc: P.add(acc, v), 0.0, col),
                       P.transpose(P.split(rows, p))), [p]


def dot_K1(n: int):
    """The single-thread dot of Section 2.2 (one kernel, one thread)."""
    x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
    return P.reduceSeq(lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p))), 0.0, P.zip_(x, y)), [x, y]


def gemv_bwd_dA(M: int, N: int):
    """dA = dy x^T: map (lambda d. map (lambda v. d * v) x) dy, a workgroup per row,
    the row's columns over the workgroup's threads."""
    dy, x = P.inp("dy", P.arr(M, P.F32)), P.inp("x", P.arr(N, P.F32))
    return P.mapWorkgroup(lambda d: P.mapLocal(lambda v: P.mul(d, v), x), dy), [dy, x]


def gemv_bwd_dx_partials(M: int, N: int, R: int):
    """The first kernel of dx = A^T dy split over rows: for each chunk of R rows
    (a workgroup) and each column (the workgroup's threads), the column's fold
    over the chunk's rows in row order -- (M/R) x N partials."""
    A, dy = P.inp("A", P.arr(M, N, P.F32)), P.inp("dy", P.arr(M, P.F32))
    e = P.mapWorkgroup(
        lambda c: P.mapLocal(
            lambda col: P.reduceSeq(lambda q, acc: P.add(acc, P.mul(P.fst(q), P.snd(q))), 0.0,
                                    P.zip_(col, P.snd(c))),
            P.transpose(P.fst(c))),
        P.zip_(P.split(R, A), P.split(R, dy)))
    return e, [A, dy]


def gemv_bwd_dx_fold(C: int, N: int):
    """The second kernel: dx_j = the fold of column j's C chunk partials in chunk order."""
    p = P.inp("p", P.arr(C * N, P.F32))
    return P.mapGlobal(lambda col: P.reduceSeq(lambda v, acc: P.add(acc, v), 0.0, col),
                       P.transpose(P.split(N, p))), [p]


# ---------------------------------------------------------------------------
# compensated (Kahan) folds: the accumulator is a pair (s, c)
# ---------------------------------------------------------------------------


def kahan_step(acc, e):
    """One compensated step: y = e - c; t = s + y; c' = (t - s) - y; s' = t."""
    s, c = P.fst(acc), P.snd(acc)
    y = P.sub(e, c)
    t = P.add(s, y)
    return P.pair(t, P.sub(P.sub(t, s), y))


def kahan_merge(acc, other_s, other_c):
    """Merge another compensated partial (s2, c2): a step with e = s2 - c2."""
    return kahan_step(acc, P.sub(other_s, other_c))


def _zero_pair():
    return P.pair(P.lit(0.0), P.lit(0.0))


def dot_partials_kahan(n: int, s: int, T: int, thread_map: str = "interleaved"):
    """Per-thread compensated sums of x . y: C*T pairs (s, c), stored as 2 numbers each."""
    x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
    e = P.join(P.mapWorkgroup(
        lambda chunk: P.mapLocal(
            lambda col: P.reduceSeq(lambda p, acc: kahan_step(acc, P.mul(P.fst(p), P.snd(p))), _zero_pair(), col),
            columns(chunk, T, thread_map)),
        P.split(s, P.zip_(x, y))))
    return e, [x, y]


def _pair_items(p, m):
    """The m pairs stored as 2m numbers, as an array of 2-element arrays."""
    return P.split(2, p)


def fold_pairs_rows(rows: int, g: int):
    """rows groups of g stored pairs, each merged in order from (0, 0): rows pairs out."""
    from .translate import IConst

    p = P.inp("p", P.arr(2 * rows * g, P.F32))
    return P.mapGlobal(
        lambda grp: P.reduceSeq(lambda pr, acc: kahan_merge(acc, P.Idx(pr, IConst(0)), P.Idx(pr, IConst(1))),
                                _zero_pair(), grp),
        P.split(g, _pair_items(p, rows * g))), [p]


def fold_pairs_all(m: int):
    """The compensated sum of m stored pairs: s of their in-order merge."""
    from .translate import IConst

    p = P.inp("p", P.arr(2 * m, P.F32))
    return P.fst(P.reduceSeq(lambda pr, acc: kahan_merge(acc, P.Idx(pr, IConst(0)), P.Idx(pr, IConst(1))),
                             _zero_pair(), _pair_items(p, m))), [p]
