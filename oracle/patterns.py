"""c1: functional pattern evaluator -- TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Arrays are Python lists; an element of type ``n.delta`` is a list of n deltas,
``delta1 x delta2`` is a 2-tuple, and the vector type ``num<V>`` (Section 6,
"Vectorisation") is a V-tuple of scalars. Every primitive is its plain
set-theoretic meaning (Section 5.1 interprets ``n.delta`` as functions from
{0..n-1} to delta), so nothing here is blocked, fused or reordered.

Scalar arithmetic is pluggable (``Arith``): ``F32`` rounds every + and * to
IEEE binary32 (round to nearest even, subnormals kept), ``Int`` is exact integer
arithmetic (int32 inputs, int64 sums), ``Sym`` builds expression trees so that a
test can read off exactly which elements a strategy adds in which association.

Strategy expressions at the bottom (``reduce_R``, ``dot_R`` ...) compose the
primitives the way the paper's strategy-annotated dot product does (Section 2.1,
the two-level expression with split/mapWorkgroup/mapLocal/reduce/join), with the
in-chunk thread tree, the lane fold of ``asVector`` and the second-level reduce
defined in the build's design notes (the paper fixes the chunk split and the
per-thread sequential reduce, not the tree; see ``Strategy``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Scalar arithmetic
# ---------------------------------------------------------------------------


class F32:
    """IEEE binary32, each operation rounded separately (no contraction)."""

    name = "f32"
    zero = np.float32(0.0)

    @staticmethod
    def lit(v):
        return np.float32(v)

    @staticmethod
    def add(a, b):
        return np.float32(np.float32(a) + np.float32(b))

    @staticmethod
    def sub(a, b):
        return np.float32(np.float32(a) - np.float32(b))

    @staticmethod
    def mul(a, b):
        return np.float32(np.float32(a) * np.float32(b))

    @staticmethod
    def fma(a, b, c):
        # a*b + c rounded once: the exact value of a*b+c is representable in
        # float64 when a, b, c are binary32 with |exponent| in range, except for
        # double rounding; go through Python's exact rational arithmetic instead.
        from fractions import Fraction

        exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
        return _round_fraction_to_f32(exact, sign_hint=_fma_zero_sign(a, b, c))

    @staticmethod
    def abs(a):
        return np.float32(abs(np.float32(a)))


def _fma_zero_sign(a, b, c):
    """Sign of an exact-zero a*b+c under round-to-nearest (IEEE 754 6.3)."""
    pa = math.copysign(1.0, float(a)) * math.copysign(1.0, float(b))
    pc = math.copysign(1.0, float(c))
    return -1.0 if (pa < 0 and pc < 0) else 1.0


def _round_fraction_to_f32(q, sign_hint=1.0):
    """Round an exact rational to binary32, round-to-nearest-even."""
    from fractions import Fraction

    if q == 0:
        return np.float32(math.copysign(0.0, sign_hint))
    neg = q < 0
    a = -q if neg else q
    # exponent e with 2^e <= a < 2^(e+1)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)  # subnormal range keeps the quantum at 2^-149
    quantum = Fraction(2) ** (e - 23)
    m = a / quantum
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = fl * quantum
    if val >= Fraction(2) ** 128:
        out = np.float32(np.inf)
    else:
        out = np.float32(float(val))
    return np.float32(-out) if neg else out


class Int:
    """Exact integers: int32 inputs, products and sums held as int64 values."""

    name = "int"
    zero = 0

    @staticmethod
    def lit(v):
        return int(v)

    @staticmethod
    def add(a, b):
        return int(a) + int(b)

    @staticmethod
    def sub(a, b):
        return int(a) - int(b)

    @staticmethod
    def mul(a, b):
        return int(a) * int(b)

    @staticmethod
    def abs(a):
        return abs(int(a))


class Sym:
    """Expression trees: leaves are names, nodes are ('+'|'-'|'*', l, r)."""

    name = "sym"
    zero = "0"

    @staticmethod
    def lit(v):
        return str(v)

    @staticmethod
    def add(a, b):
        return ("+", a, b)

    @staticmethod
    def sub(a, b):
        return ("-", a, b)

    @staticmethod
    def mul(a, b):
        return ("*", a, b)

    @staticmethod
    def abs(a):
        return ("abs", a)


# ---------------------------------------------------------------------------
# Functional primitives (Fig. "Functional primitives"; Section 5.1 semantics)
# ---------------------------------------------------------------------------


def map_(f, xs):
    """map n d1 d2 f xs : element i of the result is f(xs[i])."""
    return [f(x) for x in xs]


def reduce_(f, init, xs):
    """reduce n d1 d2 f init xs: a left fold, f(element, accumulator).

    reduceI's implementation (Section 4.2) visits the elements in index order,
    starting from ``init`` -- the fold below is exactly that loop.
    """
    acc = init
    for x in xs:
        acc = f(x, acc)
    return acc


def zip_(xs, ys):
    """zip n d1 d2 : element i is the pair (xs[i], ys[i])."""
    if len(xs) != len(ys):
        raise ValueError("zip of unequal lengths")
    return [(x, y) for x, y in zip(xs, ys)]


def split(n, xs):
    """split n m : nm.d -> m.n.d with out[i][j] = xs[i*n + j] (Stage III index rule)."""
    if n <= 0 or len(xs) % n != 0:
        raise ValueError(f"split {n} of an array of {len(xs)} elements")
    return [xs[i * n:(i + 1) * n] for i in range(len(xs) // n)]


def join(xss):
    """join n m : n.m.d -> nm.d with out[i] = xss[i // m][i % m]."""
    return [x for xs in xss for x in xs]


def pair(a, b):
    return (a, b)


def fst(p):
    return p[0]


def snd(p):
    return p[1]


def transpose(xss):
    """out[i][j] = xss[j][i]. Not a primitive of the paper; a re-indexing like split/join."""
    if not xss:
        return []
    m = len(xss[0])
    return [[xss[j][i] for j in range(len(xss))] for i in range(m)]


def asVector(V, xs):
    """asVector_V : mV.num -> m.num<V>; behaves like split V (Section 6)."""
    return [tuple(c) for c in split(V, xs)]


def asScalar(xvs):
    """asScalar_V : m.num<V> -> mV.num; behaves like join (Section 6)."""
    return [x for v in xvs for x in v]


# Level and address-space annotations are the identity on meaning (Section 6:
# "Semantically, all these variants ... are equivalent to the originals").
mapGlobal = map_
mapWorkgroup = map_
mapWarp = map_
mapLocal = map_
mapSeq = map_


def toGlobal(f):
    return f


def toLocal(f):
    return f


def toPrivate(f):
    return f


# ---------------------------------------------------------------------------
# Strategy R: split / map over chunks / per-thread fold / tree / second level
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Strategy:
    """Value-defining parameters of the canonical reduction strategy.

    s      -- chunk elements: ``split s`` of the (zipped) input.
    T      -- threads that cooperate on one chunk (1 = one thread folds the whole
              chunk sequentially, as ``mapGlobal``/``mapSeq``; 32 = one warp;
              larger = one block). Power of two.
    V      -- lanes per thread (``asVector V``), 1, 2, 4, 8 or 16.
    thread_map -- "interleaved": thread t folds vector r*T + t for r = 0, 1, ...
                  (``transpose (split T chunk)``); "contig": thread t folds the
                  vectors t*R .. t*R+R-1 (``split R chunk``, the paper's
                  per-thread contiguous sub-chunk).
    second -- "seq": left fold of the chunk results in chunk order (the paper's
              final sequential loop); "tree": the chunk results are reduced
              again by the same one-chunk algorithm with ``T2`` threads, V = 1,
              interleaved.
    compensated -- every fold step is a Kahan step (see ``kahan_step``).
    pad    -- if the length is not a multiple of s, append (+0, +0) pairs
              (the identity of the reduce) up to a multiple of s.
    """

    s: int
    T: int = 1
    V: int = 1
    thread_map: str = "interleaved"
    second: str = "seq"
    T2: int = 32
    compensated: bool = False
    pad: bool = False


def halving_tree(q, add):
    """Pairwise tree over a power-of-two list: q[l] <- q[l] + q[l + len/2], repeated."""
    q = list(q)
    if len(q) & (len(q) - 1):
        raise ValueError("halving tree over a non power of two")
    while len(q) > 1:
        h = len(q) // 2
        q = [add(q[l], q[l + h]) for l in range(h)]
    return q[0]


def kahan_step(ar, state, e):
    """One compensated-summation step (Kahan 1965; Higham, Algorithm 4.2).

    y = e - c; t = s + y; c' = (t - s) - y; s' = t.
    """
    s, c = state
    y = ar.sub(e, c)
    t = ar.add(s, y)
    c2 = ar.sub(ar.sub(t, s), y)
    return (t, c2)


def kahan_combine(ar, a, b):
    """Merge two compensated partial sums: a step of ``a`` with e = b.s - b.c."""
    return kahan_step(ar, a, ar.sub(b[0], b[1]))


def _thread_columns(chunk_vecs, st: Strategy):
    """Which vector elements each of the T threads folds, in fold order."""
    nvec = len(chunk_vecs)
    if nvec % st.T != 0:
        raise ValueError("chunk vectors not divisible by T")
    R = nvec // st.T
    if st.T == 1:
        return [chunk_vecs]
    if st.thread_map == "interleaved":
        return transpose(split(st.T, chunk_vecs))
    if st.thread_map == "contig":
        return split(R, chunk_vecs)
    raise ValueError(st.thread_map)


def _block_tree(thread_results, T, combine):
    """treeLanes over groups of min(32, T) threads, then treeWarps over the group sums."""
    L = min(32, T)
    warps = split(L, thread_results)
    return halving_tree(map_(lambda w: halving_tree(w, combine), warps), combine)


def chunk_reduce(chunk, st: Strategy, ar, elem):
    """One chunk of s elements -> its partial (plain) or (s, c) state (compensated).

    ``chunk`` is a list of s/V vector elements (each a V-tuple of input items);
    ``elem`` maps one input item to the number that is summed (x*y for dot, |x|
    for asum). Thread t: per-lane fold seeded with 0 over its column, then the
    V lanes folded in lane order (asScalar then reduce), then the thread tree.
    """
    V = st.V
    cols = _thread_columns(chunk, st)
    if not st.compensated:
        def lane_fold(col):
            return reduce_(lambda xv, acc: tuple(ar.add(acc[v], elem(xv[v])) for v in range(V)),
                           tuple([ar.zero] * V), col)

        def thread(col):
            return reduce_(lambda lane, acc: ar.add(acc, lane), ar.zero, list(lane_fold(col)))

        return _block_tree(mapLocal(thread, cols), st.T, ar.add)

    zero = (ar.zero, ar.zero)

    def lane_fold_c(col):
        return reduce_(lambda xv, acc: tuple(kahan_step(ar, acc[v], elem(xv[v])) for v in range(V)),
                       tuple([zero] * V), col)

    def thread_c(col):
        return reduce_(lambda lane, acc: kahan_combine(ar, acc, lane), zero, list(lane_fold_c(col)))

    return _block_tree(mapLocal(thread_c, cols), st.T, lambda a, b: kahan_combine(ar, a, b))


def second_level(partials, st: Strategy, ar):
    """Reduce the chunk partials (join of the per-chunk results)."""
    if st.second == "seq":
        if st.compensated:
            return reduce_(lambda p, acc: kahan_combine(ar, acc, p), (ar.zero, ar.zero), partials)
        return reduce_(lambda p, acc: ar.add(acc, p), ar.zero, partials)
    if st.second == "tree":
        T2 = st.T2
        ident = (ar.zero, ar.zero) if st.compensated else ar.zero
        padded = list(partials) + [ident] * ((-len(partials)) % T2)
        cols = transpose(split(T2, padded))
        if st.compensated:
            comb = lambda a, b: kahan_combine(ar, a, b)
            th = mapLocal(lambda col: reduce_(lambda p, acc: comb(acc, p), ident, col), cols)
            return _block_tree(th, T2, comb)
        th = mapLocal(lambda col: reduce_(lambda p, acc: ar.add(acc, p), ar.zero, col), cols)
        return _block_tree(th, T2, ar.add)
    raise ValueError(st.second)


def reduce_R(items, st: Strategy, ar, elem, pad_item):
    """The whole strategy over a list of input items (pairs for dot, scalars for asum).

    reduce2nd (join (mapWorkgroup chunk_reduce (split (s/V) (asVector V items)))).
    """
    n = len(items)
    if n == 0:
        return ar.zero
    if n % st.s != 0:
        if not st.pad:
            raise ValueError("split does not divide n")
        items = list(items) + [pad_item] * ((-n) % st.s)
    if st.s % (st.T * st.V) != 0:
        raise ValueError("s must be a multiple of T*V")
    vecs = asVector(st.V, items)
    chunks = split(st.s // st.V, vecs)
    partials = mapWorkgroup(lambda ch: chunk_reduce(ch, st, ar, elem), chunks)
    r = second_level(partials, st, ar)
    return r[0] if st.compensated else r


def dot_R(xs, ys, st: Strategy, ar=F32):
    """Dot product under strategy R: reduce of map (fst x * snd x) over zip xs ys."""
    return reduce_R(zip_(list(xs), list(ys)), st, ar,
                    lambda p: ar.mul(fst(p), snd(p)), (ar.zero, ar.zero))


def asum_R(xs, st: Strategy, ar=F32):
    """asum under strategy R: reduce of map |x|."""
    return reduce_R(list(xs), st, ar, ar.abs, ar.zero)


def dot_K1(xs, ys, ar=F32):
    """The paper's first dot translation: tmp = map (x*y) (zip xs ys), then a
    sequential loop accum = accum + tmp[i] from accum = 0 (Section 2.2)."""
    tmp = map_(lambda p: ar.mul(fst(p), snd(p)), zip_(list(xs), list(ys)))
    return reduce_(lambda t, acc: ar.add(acc, t), ar.zero, tmp)


def scal(a, xs, ar=F32):
    """scal: map (lambda x. a * x)."""
    return map_(lambda x: ar.mul(a, x), list(xs))


def gemv_R(A, x, st: Strategy, ar=F32):
    """y = map (lambda row. reduce_R (zip row x)) A -- rows are independent."""
    return mapWorkgroup(lambda row: dot_R(row, x, st, ar), [list(r) for r in A])


def gemv_bwd_dx(A, dy, row_split, ar=F32):
    """dx = A^T dy: map over columns of a split-over-rows fold.

    dx_j = reduce2nd_seq (map (lambda rows. fold (A_ij * dy_i)) (split row_split (zip col_j dy))),
    each row chunk folded sequentially from 0 in row order, then the chunk
    results folded in chunk order (rows past M are the identity pairs).
    """
    cols = transpose([list(r) for r in A])
    st = Strategy(s=row_split, T=1, V=1, second="seq", pad=True)
    return map_(lambda col: dot_R(col, dy, st, ar), cols)


def gemv_bwd_dA(x, dy, ar=F32):
    """dA = dy x^T: map (lambda d. map (lambda xj. d * xj) x) dy."""
    return map_(lambda d: map_(lambda xj: ar.mul(d, xj), list(x)), list(dy))


def dot_bwd(x, y, g, ar=F32):
    """Adjoint of reduce(+) is a broadcast of g; adjoint of map(*) a pointwise product."""
    return map_(lambda yi: ar.mul(g, yi), list(y)), map_(lambda xi: ar.mul(g, xi), list(x))


def gemm_fold(A, B, contract_fma: bool, ar=F32):
    """C = map (lambda a. map (lambda b. fold_k) (transpose B)) A.

    fold_k: acc = 0; for k in order acc = acc + a_k*b_k (two roundings), or
    acc = fma(a_k, b_k, acc) when the contraction is declared.
    """
    Bt = transpose([list(r) for r in B])

    def cell(a, b):
        if contract_fma:
            return reduce_(lambda p, acc: ar.fma(p[0], p[1], acc), ar.zero, zip_(a, b))
        return reduce_(lambda p, acc: ar.add(acc, ar.mul(p[0], p[1])), ar.zero, zip_(a, b))

    return map_(lambda a: map_(lambda b: cell(a, b), Bt), [list(r) for r in A])
