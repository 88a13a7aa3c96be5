"""The paper's running examples as phrases (Sections 2.1 and 7): each program
is one or two kernels, the second folding the first one's partial results.

    dot   partials = join (mapWorkgroup (lambda chunk.
                       mapLocal (lambda col. reduceSeq (+) 0 (map (*) col))
                                (columns chunk)) (split s (zip x y)))
          result   = reduceSeq (+) 0 partials
    asum  the same with map abs
    scal  mapGlobal (lambda v. a * v) x
    dA    mapWorkgroup (lambda d. mapLocal (lambda v. d * v) x) dy
    dot dx = mapGlobal (lambda v. g * v) y
    gemm  mapWorkgroup (lambda a. mapLocal (lambda b. reduceSeq (+) 0
                       (map (*) (zip a b))) (transpose B)) A
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


def gemv_bwd_dx_partials(M: int, N: int, R: int, V: int = 1):
    """The first kernel of dx = A^T dy split over rows: for each chunk of R rows
    (a workgroup) and each column (the workgroup's threads), the column's fold
    over the chunk's rows in row order -- (M/R) x N partials. With V > 1 a
    thread folds V adjacent columns as one num<V> (dy_r widened), each lane its
    own column's fold in the same order."""
    A, dy = P.inp("A", P.arr(M, N, P.F32)), P.inp("dy", P.arr(M, P.F32))
    if V == 1:
        e = P.mapWorkgroup(
            lambda c: P.mapLocal(
                lambda col: P.reduceSeq(lambda q, acc: P.add(acc, P.mul(P.fst(q), P.snd(q))), 0.0,
                                        P.zip_(col, P.snd(c))),
                P.transpose(P.fst(c))),
            P.zip_(P.split(R, A), P.split(R, dy)))
        return e, [A, dy]
    if N % V:
        raise ValueError("vector columns need N a multiple of V")
    rows = P.split(R, P.split(N // V, P.asVector(V, P.join(A))))  # (M/R) x R x (N/V) vectors
    e = P.mapWorkgroup(
        lambda c: P.asScalar(P.mapLocal(
            lambda col: P.reduceSeq(lambda q, acc: P.add(acc, P.mul(P.fst(q), P.splat(V, P.snd(q)))),
                                    P.vlit(0.0, V), P.zip_(col, P.snd(c))),
            P.transpose(P.fst(c)))),
        P.zip_(rows, P.split(R, dy)))
    return e, [A, dy]


def gemv_bwd_dx_fold(C: int, N: int):
    """The second kernel: dx_j = the fold of column j's C chunk partials in chunk order."""
    p = P.inp("p", P.arr(C * N, P.F32))
    return P.mapGlobal(lambda col: P.reduceSeq(lambda v, acc: P.add(acc, v), 0.0, col),
                       P.transpose(P.split(N, p))), [p]


def dot_bwd(n: int, V: int = 1):
    """One half of the dot's backward pass: map (lambda v. g * v) over y gives dx
    (and over x gives dy) -- the adjoint of the reduce broadcasts the incoming
    gradient g, the adjoint of the zip-map multiplies pointwise. g is a
    one-element input (the gradient as the autodiff leaves it, in memory)."""
    from .translate import IConst

    g, v = P.inp("g", P.arr(1, P.F32)), P.inp("v", P.arr(n, P.F32))
    gv = P.Idx(g, IConst(0))
    if V == 1:
        return P.mapGlobal(lambda e: P.mul(gv, e), v), [g, v]
    return P.asScalar(P.mapGlobal(lambda e: P.mul(P.splat(V, gv), e), P.asVector(V, v))), [g, v]


def gemm(M: int, N: int, K: int, V: int = 1, transA: bool = False, transB: bool = False):
    """C = map (lambda a. map (lambda b. reduceSeq (+) 0 (map (*) (zip a b)))
    (transpose B)) A: a workgroup per row of C, the row's columns over the
    workgroup's threads, each C_ij one sequential fold over k from +0 (the
    product and the sum rounded separately). op(A) is A (M x K) or, with
    transA, the transpose of a stored K x M matrix; op(B) is B (K x N) or,
    with transB, the transpose of a stored N x K matrix -- transposes are
    views, so the backward products dA = dC B^T and dB = A^T dC are the same
    phrase. With V > 1 (B not transposed) a thread folds V adjacent columns
    as one num<V>: a_ik widened to a vector times the V entries of row k of
    B, each lane its own fold, in the same order."""
    A = P.inp("A", P.arr(K, M, P.F32) if transA else P.arr(M, K, P.F32))
    B = P.inp("B", P.arr(N, K, P.F32) if transB else P.arr(K, N, P.F32))
    rows = P.transpose(A) if transA else A
    if V == 1:
        cols = B if transB else P.transpose(B)
        e = P.mapWorkgroup(
            lambda a: P.mapLocal(
                lambda b: P.reduceSeq(lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p))), 0.0, P.zip_(a, b)),
                cols),
            rows)
        return e, [A, B]
    if transB or N % V:
        raise ValueError("vector columns need B stored K x N with N a multiple of V")
    cols = P.transpose(P.split(N // V, P.asVector(V, P.join(B))))  # (N/V) x K of num<V>
    e = P.mapWorkgroup(
        lambda a: P.asScalar(P.mapLocal(
            lambda b: P.reduceSeq(lambda p, acc: P.add(acc, P.mul(P.splat(V, P.fst(p)), P.snd(p))),
                                  P.vlit(0.0, V), P.zip_(a, b)),
            cols)),
        rows)
    return e, [A, B]


def gemm_tiled(M: int, N: int, K: int, R: int = 8, Cn: int = 8, V: int = 4, KV: int = 1, transA: bool = False,
               transB: bool = False, contract: str = "off"):
    """The GEMM with a register tile per thread: a workgroup per block of R rows
    of C, its threads over blocks of Cn columns, each thread's R x Cn block of C
    one fold over k whose accumulator is a private array (Cn/V vectors per row):

        join (mapWorkgroup (lambda rows. transpose (mapLocal (lambda cols.
          reduceSeq (lambda (a, b) acc. mapSeq (lambda (a_r, acc_r). mapSeq
            (lambda (b_q, c). c + splat a_r * b_q) (zip b acc_r)) (zip a acc))
            0 (zip (transpose rows) cols)) colblocks)) (split R op(A)))

    a is column k of the row block (R numbers), b row k of the column block
    (Cn/V vectors of B, read with V-wide loads). With KV > 1 the fold runs over
    groups of KV consecutive k: the row block's A is read as vectors along k
    (asVector KV, one load per row for KV steps), their lanes staged in a
    private array, and the group's KV steps folded in k order by an inner
    reduceSeq whose initial value is the outer accumulator. Every element of C
    is still one sequential fold over k from +0, product and sum rounded
    separately, so the result equals the plain fold (and the untiled gemm) bit
    for bit; the tile only keeps each loaded value in registers for several
    products. The transposes are views; V > 1 needs B stored K x N and KV > 1
    needs A stored M x K (the adjacent numbers a vector load reads). With
    contract = "fma" each step is fma(a_r, b_q, c), one rounding (the
    contraction the library's FP32 fold declares by default)."""
    if contract not in ("off", "fma"):
        raise ValueError(f"contract {contract!r}: off or fma")
    if M % R or N % Cn or Cn % V or K % KV:
        raise ValueError("R must divide M, Cn must divide N, V must divide Cn and KV must divide K")
    if (V > 1 and transB) or (KV > 1 and transA):
        raise ValueError("vector loads need B stored K x N (V > 1) and A stored M x K (KV > 1)")
    A = P.inp("A", P.arr(K, M, P.F32) if transA else P.arr(M, K, P.F32))
    B = P.inp("B", P.arr(N, K, P.F32) if transB else P.arr(K, N, P.F32))
    if KV > 1:
        rows = P.split(R, P.split(K // KV, P.asVector(KV, P.join(A))))  # (M/R) x R x (K/KV) vectors
    else:
        rows = P.split(R, P.transpose(A) if transA else A)  # (M/R) x R x K
    if transB:
        colblocks, col_view = P.split(Cn, B), P.transpose  # (N/Cn) x Cn x K, each viewed K x Cn
    elif V == 1:
        colblocks, col_view = P.transpose(P.split(N // Cn, P.split(Cn, P.join(B)))), (lambda c: c)
    else:
        colblocks = P.transpose(P.split(N // Cn, P.split(Cn // V, P.asVector(V, P.join(B)))))
        col_view = lambda c: c  # noqa: E731  (N/Cn) x K x (Cn/V) vectors
    elt = P.F32 if V == 1 else P.VecT(V, P.F32)
    zero = P.alit(0.0, P.arr(R, Cn // V, elt))

    def madd(a_r, b_q, c):
        a_r = a_r if V == 1 else P.splat(V, a_r)
        return P.fma(a_r, b_q, c) if contract == "fma" else P.add(c, P.mul(a_r, b_q))

    def step(p, acc):  # one k: a (R numbers), b (Cn/V numbers or vectors)
        a, b = P.fst(p), P.snd(p)
        return P.mapSeq(lambda q: P.mapSeq(lambda s: madd(P.fst(q), P.fst(s), P.snd(s)),
                                           P.zip_(b, P.snd(q))), P.zip_(a, acc))

    def group(p, acc):  # KV consecutive k: R vectors of A along k, KV rows of the column block
        ak = P.transpose(P.to_private(P.mapSeq(lambda v: P.lanes(v), P.fst(p))))  # KV x R numbers
        return P.reduceSeq(step, acc, P.zip_(ak, P.snd(p)))

    def fold(rb, cb):
        if KV == 1:
            return P.reduceSeq(step, zero, P.zip_(P.transpose(rb), col_view(cb)))
        return P.reduceSeq(group, zero, P.zip_(P.transpose(rb), P.split(KV, col_view(cb))))

    e = P.join(P.mapWorkgroup(lambda rb: P.transpose(P.mapLocal(lambda cb: fold(rb, cb), colblocks)), rows))
    if V > 1:
        e = P.asScalar(P.join(P.join(e)))
    return e, [A, B]


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


# ---------------------------------------------------------------------------
# the whole strategy in one kernel: per-thread folds, the in-block tree (lane
# trees within warps, then over the warp sums), and the second level in the
# last work-group
# ---------------------------------------------------------------------------


def _plus(a, b):
    return P.add(a, b)


def block_tree(cols, column, combine=None):
    """The block's tree over its T thread results, T = len(cols) a power of two
    (1..1024), thread t's result being column(cols[t]): the columns are split
    into groups of min(32, T), a warp per group; lane l computes its column's
    result straight into its register of a lane tree over the group, and a lane
    tree over the group sums (a local temporary: other warps wrote it) gives the
    one-element array of the work-group's result. The same tree as a halving
    tree within each group of 32 consecutive thread results, then over the
    group sums."""
    combine = combine or _plus
    T = cols.type.n
    L = min(P.WARP, T)
    sums = P.mapWarp(lambda g: P.reduceTree(combine, P.mapLane(column, g)), P.split(L, cols))
    W = T // L
    if W == 1:
        return sums
    return P.mapWarp(lambda g: P.reduceTree(combine, g), P.split(W, P.to_local(sums)))


def column_result(V: int, step):
    """A thread's result: its column folded from +0 with ``step`` (lane-wise on
    num<V>), then its V lanes folded in lane order from +0."""
    def column(col):
        acc = P.reduceSeq(step, _zero(V), col)
        if V == 1:
            return acc
        return P.reduceSeq(lambda v, a: P.add(a, v), P.lit(0.0), P.lanes(acc))
    return column


def chunk_result(chunk, T: int, thread_map: str, V: int, step):
    """The chunk's first level: T thread folds of its columns, then the block tree."""
    return block_tree(columns(chunk, T, thread_map), column_result(V, step))


def second_level(parts, second: str, T2: int):
    """The fold of the C chunk results: in chunk order from +0 by one thread
    (seq), or T2 threads each folding results r*T2 + t from +0, then the block
    tree (tree; C must be a multiple of T2)."""
    C = parts.type.n
    if second == "seq":
        return P.reduceSeq(lambda v, a: P.add(a, v), 0.0, parts)
    if C % T2:
        raise ValueError(f"a tree second level over {C} results needs a thread count dividing it, not {T2}")
    return block_tree(P.transpose(P.split(T2, parts)), lambda col: P.reduceSeq(lambda v, a: P.add(a, v), 0.0, col))


def _reduce_R(items, n_items: int, s: int, T: int, thread_map: str, V: int, second: str, T2: int, step):
    if s % (T * V) or n_items % s:
        raise ValueError(f"split {s} over {T} threads x {V} lanes does not divide {n_items} items")
    chunks = P.split(s // V, items)
    parts = P.join(P.mapWorkgroup(lambda ch: chunk_result(ch, T, thread_map, V, step), chunks))
    return P.secondLevel(parts, lambda p: second_level(p, second, T2))


def _kahan_combine(a, b):
    """Merge compensated partial b into a: a Kahan step of a with e = b.s - b.c."""
    return kahan_merge(a, P.fst(b), P.snd(b))


def _reduce_R_kahan(items, n_items: int, s: int, T: int, thread_map: str, V: int, second: str, T2: int, elem):
    """The canonical strategy with every fold step a Kahan step: each lane keeps
    (s, c) (lane-wise on num<V>), a thread merges its V lane pairs in lane order
    from (0, 0), the trees and the second level merge pairs, and the result is
    the final s -- the library's compensated reduction."""
    if s % (T * V) or n_items % s:
        raise ValueError(f"split {s} over {T} threads x {V} lanes does not divide {n_items} items")

    def column(col):
        zero = P.pair(_zero(V), _zero(V))
        acc = P.reduceSeq(lambda it, a: kahan_step(a, elem(it)), zero, col)
        if V == 1:
            return acc
        lane_pairs = P.lanes(acc)  # lane v's (s, c): the accumulator read once
        return P.reduceSeq(lambda lp, a: kahan_merge(a, P.fst(lp), P.snd(lp)), _zero_pair(), lane_pairs)

    def fold_pairs(col):
        return P.reduceSeq(lambda p, a: _kahan_combine(a, p), _zero_pair(), col)

    chunks = P.split(s // V, items)
    parts = P.join(P.mapWorkgroup(
        lambda ch: block_tree(columns(ch, T, thread_map), column, _kahan_combine), chunks))

    def second_level_kahan(p):
        C = p.type.n
        if second == "seq":
            return P.fst(fold_pairs(p))
        if C % T2:
            raise ValueError(f"a tree second level over {C} results needs a thread count dividing it, not {T2}")
        return P.mapSeq(lambda r: P.fst(r), block_tree(P.transpose(P.split(T2, p)), fold_pairs, _kahan_combine))

    return P.secondLevel(parts, second_level_kahan)


def dot_R_kahan(n: int, s: int, T: int, V: int = 4, thread_map: str = "interleaved", second: str = "tree",
                T2: int = 256):
    """x . y in one kernel with the canonical strategy, compensated (Kahan) at
    every level: the library's dot with compensated = 1."""
    x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
    return _reduce_R_kahan(P.zip_(_vec(x, V), _vec(y, V)), n, s, T, thread_map, V, second, T2,
                           lambda p: P.mul(P.fst(p), P.snd(p))), [x, y]


def asum_R_kahan(n: int, s: int, T: int, V: int = 4, thread_map: str = "interleaved", second: str = "tree",
                 T2: int = 256):
    """sum |x_i| in one kernel, compensated at every level."""
    x = P.inp("x", P.arr(n, P.F32))
    return _reduce_R_kahan(_vec(x, V), n, s, T, thread_map, V, second, T2, P.abs_), [x]


def dot_R(n: int, s: int, T: int, V: int = 4, thread_map: str = "interleaved", second: str = "tree",
          T2: int = 256):
    """x . y in one kernel with the canonical strategy (split s, T threads per
    chunk, V lanes, the thread map, the second level): the same tree as the
    library's dot and the oracle's loop nest."""
    x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
    step = lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p)))
    return _reduce_R(P.zip_(_vec(x, V), _vec(y, V)), n, s, T, thread_map, V, second, T2, step), [x, y]


def asum_R(n: int, s: int, T: int, V: int = 4, thread_map: str = "interleaved", second: str = "tree",
           T2: int = 256):
    """sum |x_i| in one kernel with the canonical strategy."""
    x = P.inp("x", P.arr(n, P.F32))
    step = lambda v, acc: P.add(acc, P.abs_(v))
    return _reduce_R(_vec(x, V), n, s, T, thread_map, V, second, T2, step), [x]


def gemv_R(M: int, N: int, T: int, V: int = 4, thread_map: str = "interleaved"):
    """y = A x with a work-group per row (one chunk per row: split N): each row's
    T thread folds and the block tree, in one kernel -- the library's GEMV with
    rows at block level and split = N."""
    if N % (T * V):
        raise ValueError(f"a row of {N} does not split over {T} threads x {V} lanes")
    A, x = P.inp("A", P.arr(M, N, P.F32)), P.inp("x", P.arr(N, P.F32))
    step = lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p)))
    e = P.join(P.mapWorkgroup(
        lambda row: chunk_result(P.zip_(_vec(row, V), _vec(x, V)), T, thread_map, V, step), A))
    return e, [A, x]


def gemv_R_warp(M: int, N: int, rows_per_block: int, V: int = 4):
    """y = A x with rows at warp level: a work-group takes rows_per_block rows,
    a warp per row; lane l folds the row's items l, l + 32, .. (interleaved, on
    num<V>), folds its lanes, and the lane tree reduces the 32 results -- the
    library's GEMV with rows at warp level and split = N."""
    if N % (P.WARP * V) or M % rows_per_block:
        raise ValueError("rows of N items over 32 lanes x V, and M rows over blocks of rows_per_block")
    A, x = P.inp("A", P.arr(M, N, P.F32)), P.inp("x", P.arr(N, P.F32))
    step = lambda p, acc: P.add(acc, P.mul(P.fst(p), P.snd(p)))

    def lane_result(col):
        acc = P.reduceSeq(step, _zero(V), col)
        return acc if V == 1 else P.reduceSeq(lambda v, a: P.add(a, v), 0.0, P.lanes(acc))

    e = P.join(P.mapWorkgroup(
        lambda rows: P.mapWarp(
            lambda row: P.reduceTree(_plus, P.mapLane(lane_result,
                                                      columns(P.zip_(_vec(row, V), _vec(x, V)), P.WARP,
                                                              "interleaved"))),
            rows),
        P.split(rows_per_block, A)))
    return e, [A, x]
