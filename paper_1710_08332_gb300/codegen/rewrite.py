"""Rewrite-based exploration of strategies (the search Section 2.1 points to).

A computation starts as a strategy-free expression over a small grammar

    E ::= Reduce E | Map f E | Each B E | Split s E | Columns T m E | Vec V E | Input xs
        | Tree E | Last k T2 E | Rows l B E
    B ::= E with a Hole for the element

from ``Reduce (Map f (Input xs))`` (dot: f = (*) over zip x y; asum: f = abs;
asum_scal: f = abs over the map (a *) of x, the sum of |a x_i|) or, for GEMV,
``Rows block (Reduce (Map (*) Hole)) (Input A)`` (each row's reduce of its
products with x). Rules rewrite the tree; each holds in real arithmetic for
the associative + with identity 0:

  split(s)       Reduce (Map f X)          -> Reduce (Each (Reduce (Map f Hole)) (Split s X))
  columns(T, m)  Reduce (Map f Hole), per chunk (or per row)
                                           -> Reduce (Each (Reduce (Map f Hole)) (Columns T m Hole))
  vectorize(V)   ... Split s (Input xs)     -> ... Split (s/V) (Vec V (Input xs)) (a row: Vec V);
                 the map and the column folds then run lane-wise on num<V>
  tree           Reduce (Each ... (Columns ..)) -> Tree (Each ... (Columns ..)): a chunk's (or a
                 row's) column results reduced by the halving tree (lane trees within warps,
                 then over the warp sums) instead of a fold
  second(k, T2)  Reduce (Each (Tree ..) (Split s X)) -> Last k T2 (Each (Tree ..) (Split s X)):
                 the chunk results reduced in the same kernel by the last work-group to finish
                 (k = seq: a fold in chunk order; tree: T2 strided folds, then the tree)
  rows(l)        Rows block B A -> Rows l B A: a GEMV's rows mapped to work-groups (block) or to
                 the warps of a work-group (warp; its columns are then the 32 lanes)
  fuse_maps      Reduce (Map f (Map g X)) -> Reduce (Map (f . g) X): the inner map's result is
                 never written out
                 (one kernel instead of two; the value of every element is the same)
  fuse, lower    Reduce (Map f col) -> reduceSeq (lambda (x, a). a + f x) 0 col; the Each
                 over Split -> mapWorkgroup, the Each over Columns -> mapLocal (mapLane for rows
                 at warp level); an outermost Reduce over the per-thread partials becomes folding
                 kernels (it reads what other blocks wrote: a kernel boundary), a Last becomes
                 the second level in the last work-group of the same kernel

GEMM, the map of maps of a fold over k (``Map (Map (Reduce (Map (*) (zip a b))))``), has
rules of its own; each keeps every C_ij the same fold over k in order, so all GEMM
derivations give the same bits:

  vectorize(V)   the column map over groups of V adjacent columns, each group one num<V> fold
                 (the map of a fold over vectors = the vector of the folds)
  tile(R, Cn)    the row map split by R and the column map by Cn, the R x Cn maps moved
                 inside the fold (map-reduce interchange): one fold over k whose accumulator
                 is the R x Cn array
  vectorize_k(KV) the fold over k split into groups of KV (a left fold over k is the fold
                 over groups, each group folded in order from the running value), A read as
                 num<KV> along k

GEMV's backward dx = A^T dy (a map over columns of a fold over rows): split_rows(R) splits
each column's fold into chunks of R rows, a work-group per chunk, then a fold of the chunk
results in chunk order (each R its own tree); vectorize(V) folds V adjacent columns as one
num<V> (no value changes).

``derivations`` enumerates rule sequences over parameter grids, ``rewrite``
applies one to the start expression (each rule checks the shape it rewrites),
and ``lower`` turns the resulting tree into kernel phrases. Each derivation's
result is exact for its own tree; different derivations round differently
(except fuse_maps, which changes no value).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

from . import phrase as P
from . import programs as PR

SCALE = 1.5  # the a of asum_scal (the bandwidth workload's scal factor)

# ---------------------------------------------------------------------------
# the strategy-free grammar
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Input:
    name: str            # "dot" (zip x y), "asum" / "asum_scal" (x), "gemv" (A)


@dataclass(frozen=True)
class Hole:
    pass


@dataclass(frozen=True)
class Map:
    f: str               # "mul" (fst * snd), "abs", "scale" (a *), or "abs.scale" (fused)
    e: object


@dataclass(frozen=True)
class Reduce:
    e: object


@dataclass(frozen=True)
class Each:
    body: object         # expression with a Hole
    e: object


@dataclass(frozen=True)
class Split:
    s: int
    e: object


@dataclass(frozen=True)
class Columns:
    T: int
    m: str               # "interleaved" or "contig"
    e: object


@dataclass(frozen=True)
class Vec:
    V: int
    e: object


@dataclass(frozen=True)
class Tree:
    e: object


@dataclass(frozen=True)
class Last:
    kind: str            # "seq" or "tree"
    T2: int
    e: object


@dataclass(frozen=True)
class Rows:
    level: str           # "block" or "warp"
    body: object
    e: object


HOLE = Hole()


def start(kind: str):
    """The strategy-free expression of kind "dot", "asum", "asum_scal" or "gemv"."""
    if kind == "gemv":
        return Rows("block", Reduce(Map("mul", HOLE)), Input("gemv"))
    if kind == "asum_scal":
        return Reduce(Map("abs", Map("scale", Input(kind))))
    return Reduce(Map({"dot": "mul", "asum": "abs"}[kind], Input(kind)))


class RuleError(ValueError):
    pass


# ---------------------------------------------------------------------------
# rules
# ---------------------------------------------------------------------------


def _is_stream(x) -> bool:
    """An input, or a map of one that is written out by a kernel of its own."""
    return isinstance(x, Input) or (isinstance(x, Map) and isinstance(x.e, Input))


def r_split(e, s: int):
    if not (isinstance(e, Reduce) and isinstance(e.e, Map) and _is_stream(e.e.e)):
        raise RuleError("split rewrites Reduce (Map f (Input xs))")
    return Reduce(Each(Reduce(Map(e.e.f, HOLE)), Split(s, e.e.e)))


def _columns_of(body, T: int, m: str):
    if not (isinstance(body, Reduce) and isinstance(body.e, Map) and body.e.e == HOLE):
        raise RuleError("columns rewrites a per-chunk (or per-row) Reduce (Map f Hole)")
    return Reduce(Each(Reduce(Map(body.e.f, HOLE)), Columns(T, m, HOLE)))


def r_columns(e, T: int, m: str):
    if isinstance(e, Rows):
        if e.level == "warp" and (T, m) != (P.WARP, "interleaved"):
            raise RuleError("a row at warp level has the warp's 32 lanes as its interleaved columns")
        return Rows(e.level, _columns_of(e.body, T, m), e.e)
    if not (isinstance(e, Reduce) and isinstance(e.e, Each)):
        raise RuleError("columns rewrites the per-chunk Reduce (Map f Hole)")
    return Reduce(Each(_columns_of(e.e.body, T, m), e.e.e))


def r_vectorize(e, V: int):
    if isinstance(e, Rows):
        if not isinstance(e.e, Input):
            raise RuleError("vectorize applies once")
        return Rows(e.level, e.body, Vec(V, e.e))

    def go(x):
        if isinstance(x, Split) and _is_stream(x.e):
            if x.s % V:
                raise RuleError(f"split {x.s} is not a multiple of the width {V}")
            return Split(x.s // V, Vec(V, x.e))
        if isinstance(x, Reduce):
            return Reduce(go(x.e))
        if isinstance(x, Each):
            return Each(x.body, go(x.e))
        raise RuleError("vectorize needs the split input")
    return go(e)


def _tree_of(body):
    if not (isinstance(body, Reduce) and isinstance(body.e, Each) and isinstance(body.e.e, Columns)):
        raise RuleError("tree rewrites the Reduce over a chunk's (or row's) columns")
    return Tree(body.e)


def r_tree(e):
    if isinstance(e, Rows):
        return Rows(e.level, _tree_of(e.body), e.e)
    if not (isinstance(e, Reduce) and isinstance(e.e, Each)):
        raise RuleError("tree rewrites the Reduce over a chunk's columns")
    return Reduce(Each(_tree_of(e.e.body), e.e.e))


def r_second(e, kind: str, T2: int):
    if not (isinstance(e, Reduce) and isinstance(e.e, Each) and isinstance(e.e.body, Tree)):
        raise RuleError("second rewrites the Reduce over the chunks' tree results")
    if kind not in ("seq", "tree"):
        raise RuleError(f"second level {kind}: seq or tree")
    return Last(kind, T2, e.e)


def r_rows(e, level: str):
    if not isinstance(e, Rows) or level not in ("block", "warp"):
        raise RuleError("rows rewrites a GEMV's row map to block or warp level")
    return Rows(level, e.body, e.e)


def r_fuse_maps(e):
    if not (isinstance(e, Reduce) and isinstance(e.e, Map) and isinstance(e.e.e, Map)):
        raise RuleError("fuse_maps rewrites Reduce (Map f (Map g X))")
    return Reduce(Map(f"{e.e.f}.{e.e.e.f}", e.e.e.e))


RULES = {"split": r_split, "columns": r_columns, "vectorize": r_vectorize, "tree": r_tree, "second": r_second,
         "rows": r_rows, "fuse_maps": r_fuse_maps}


@dataclass(frozen=True)
class Rule:
    name: str
    args: tuple = ()

    def __str__(self):
        return f"{self.name}({', '.join(map(str, self.args))})" if self.args else self.name


@dataclass
class Derivation:
    rules: list = field(default_factory=list)

    def __str__(self):
        return " ; ".join(map(str, self.rules))


def rewrite(kind: str, d: Derivation):
    """The start expression with the derivation's rules applied in order
    (fuse and lower are carried out by ``lower``)."""
    e = start(kind)
    for r in d.rules:
        if r.name in RULES:
            e = RULES[r.name](e, *r.args)
    return e


# ---------------------------------------------------------------------------
# lowering to phrases
# ---------------------------------------------------------------------------


def _elem_fn(f: str, V: int = 1):
    """The per-item function of a map: mul (fst * snd), abs, or abs of (a *)."""
    if f == "mul":
        return lambda x: P.mul(P.fst(x), P.snd(x))
    if f == "abs":
        return lambda x: P.abs_(x)
    if f == "abs.scale":
        a = P.lit(SCALE) if V == 1 else P.vlit(SCALE, V)
        return lambda x: P.abs_(P.mul(a, x))
    raise RuleError(f"no element function {f}")


def _stream(kind: str, n: int, V: int, materialized: bool):
    """(inputs, the item stream) of a reduction: zip x y for dot, x otherwise (y,
    the output of the map kernel before it, when the inner map is written out)."""
    if kind == "dot":
        x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
        return [x, y], (P.zip_(x, y) if V == 1 else P.zip_(P.asVector(V, x), P.asVector(V, y)))
    x = P.inp("y" if materialized else "x", P.arr(n, P.F32))
    return [x], (x if V == 1 else P.asVector(V, x))


def lower(kind: str, d: Derivation, n: int, M: int = 0):
    """Kernel phrases for a derivation: [(name, phrase, inputs), ...], run in
    order, each reading the previous one's output. Reductions: the per-thread
    partials and then folding kernels down to one number (the paper's form), or
    one kernel when the chunk results are reduced in the last work-group (a
    materialized inner map adds a kernel in front). GEMV (n = columns, M rows):
    one kernel, or partials and row folds."""
    if kind == "gemv_dx":
        return lower_gemv_dx(d, M, n)
    e = rewrite(kind, d)
    if kind == "gemv":
        return _lower_gemv(e, M, n)
    kernels = []
    top = e
    try:
        chunk_each = top.e
        body = chunk_each.body
        col_each = body.e
        f = col_each.body.e.f
        T, m = col_each.e.T, col_each.e.m
        sp = chunk_each.e
        s, stream = sp.s, sp.e
    except AttributeError as exc:
        raise RuleError(f"derivation {d} does not reach the lowerable shape") from exc
    V = stream.V if isinstance(stream, Vec) else 1
    base = stream.e if isinstance(stream, Vec) else stream
    materialized = isinstance(base, Map)
    if materialized:  # the inner map is a kernel of its own that writes its result out
        ph, ins = PR.scal(n, SCALE, V=V)
        kernels.append(("map_scale", ph, ins))
    ins, xs = _stream(kind, n, V, materialized)
    g = _elem_fn(f, V)
    zero = P.lit(0.0) if V == 1 else P.vlit(0.0, V)
    if isinstance(top, Last):
        if not isinstance(body, Tree):
            raise RuleError("the second level needs the chunks' tree results")
        step = lambda v, a: P.add(a, g(v))
        s_items = s * V  # the split counted in numbers (s counts the stream's vectors)
        T2 = min(top.T2, n // s_items) if top.kind == "tree" else 1
        ph = PR._reduce_R(xs, n, s_items, T, m, V, top.kind, T2, step)
        kernels.append(("one_kernel", ph, ins))
        return kernels
    if isinstance(body, Tree):
        raise RuleError("a chunk tree needs the second level in the same kernel (second)")
    first = P.join(P.mapWorkgroup(
        lambda chunk: P.mapLocal(lambda col: P.reduceSeq(lambda v, a: P.add(a, g(v)), zero, col),
                                 PR.columns(chunk, T, m)),
        P.split(s, xs)))
    kernels.append(("partials", first, ins))
    left = n // (s * V) * T * V
    for grp in fold_plan(left):
        if grp == left:
            ph, i2 = PR.fold_all(left)
            kernels.append((f"fold{left}", ph, i2))
        else:
            ph, i2 = PR.fold_cols(left // grp, grp)
            kernels.append((f"fold{grp}", ph, i2))
        left //= grp
    return kernels


def _lower_gemv(e, M: int, N: int):
    try:
        level, body, src = e.level, e.body, e.e
        V = src.V if isinstance(src, Vec) else 1
        col_each = body.e
        T, m = col_each.e.T, col_each.e.m
    except AttributeError as exc:
        raise RuleError("a GEMV derivation needs its columns") from exc
    if level == "warp":
        if not isinstance(body, Tree):
            raise RuleError("rows at warp level reduce their lanes by the tree")
        rpb = next(r for r in (8, 4, 2, 1) if M % r == 0)
        ph, ins = PR.gemv_R_warp(M, N, rpb, V)
        return [("one_kernel", ph, ins)]
    if isinstance(body, Tree):
        ph, ins = PR.gemv_R(M, N, T, V, m)
        return [("one_kernel", ph, ins)]
    ph, ins = PR.gemv_partials(M, N, T, m, V)
    ph2, i2 = PR.fold_rows(M, T * V)
    return [("partials", ph, ins), ("rows", ph2, i2)]


def fold_plan(m: int) -> list:
    """Group sizes of the folding kernels that reduce m partials to one: groups
    of up to 128 (a thread folds a group with its loads in a few batches), so
    that 2^21 partials take three kernels (2^21 -> 16384 -> 128 -> 1); a group
    size divides what is left, and the last group folds what remains. A
    stage's groups are strided (fold_cols): output j folds partials j,
    j + rows, .. so that the threads' loads are coalesced."""
    plan = []
    while m > 1:
        g = m if m <= 128 else next((d for d in (128, 64, 32, 16, 8, 4, 2) if m % d == 0), m)
        plan.append(g)
        m //= g
    return plan


def derivations(n: int, splits=(1 << 14, 1 << 15, 1 << 16), threads=(128, 256, 512),
                maps=("interleaved", "contig"), widths=(1, 4), forms=("paper",), kind: str = "dot"):
    """Every derivation over the parameter grids whose rules apply. forms:
    "paper" (per-thread partials, then folding kernels) and/or "single" (the
    chunk's tree and the second level in the last work-group: one kernel); for
    asum_scal each derivation comes with and without fuse_maps."""
    out = []
    fuse_opts = (False, True) if kind == "asum_scal" else (False,)
    for s, T, m, V, form, fm in itertools.product(splits, threads, maps, widths, forms, fuse_opts):
        if n % s or (s // V) % T or s % V:
            continue
        rules = ([Rule("fuse_maps")] if fm else []) + [Rule("split", (s,)), Rule("columns", (T, m))]
        if V > 1:
            rules.append(Rule("vectorize", (V,)))
        if form == "single":
            rules += [Rule("tree"), Rule("second", ("tree", min(256, T, n // s)))]
        rules += [Rule("fuse"), Rule("lower")]
        out.append(Derivation(rules))
    return out


def gemv_derivations(M: int, N: int, threads=(64, 128, 256), widths=(1, 4)):
    """GEMV derivations: rows at block level (T columns, interleaved or contig,
    the row's tree in one kernel or partials and row folds) and at warp level."""
    out = []
    for T, m, V, tree in itertools.product(threads, ("interleaved", "contig"), widths, (True, False)):
        if N % (T * V):
            continue
        rules = [Rule("columns", (T, m))] + ([Rule("vectorize", (V,))] if V > 1 else [])
        out.append(Derivation(rules + ([Rule("tree")] if tree else []) + [Rule("fuse"), Rule("lower")]))
    for V in widths:
        if N % (P.WARP * V) == 0:
            out.append(Derivation([Rule("rows", ("warp",)), Rule("columns", (P.WARP, "interleaved"))]
                                  + ([Rule("vectorize", (V,))] if V > 1 else []) + [Rule("tree"), Rule("fuse"),
                                                                                     Rule("lower")]))
    return out


def gemv_dx_derivations(M: int, N: int, row_splits=(16, 32, 64, 128, 256, 512), widths=(1, 4)):
    """GEMV backward dx = A^T dy (a map over columns of a fold over rows):
    split_rows(R) splits each column's fold into chunks of R rows (a
    work-group per chunk, then a fold of the chunk partials in chunk order),
    vectorize(V) folds V adjacent columns as one num<V>. Each R is its own tree
    (a different association); V changes no bit."""
    out = []
    for R, V in itertools.product(row_splits, widths):
        if M % R or N % V:
            continue
        out.append(Derivation([Rule("split_rows", (R,))] + ([Rule("vectorize", (V,))] if V > 1 else [])))
    return out


def lower_gemv_dx(d: Derivation, M: int, N: int):
    """The two kernels of a dx derivation: the chunk partials and their fold."""
    args = {r.name: r.args for r in d.rules}
    if "split_rows" not in args or set(args) - {"split_rows", "vectorize"}:
        raise RuleError(f"a dx derivation is split_rows(R) [; vectorize(V)], not {d}")
    R = args["split_rows"][0]
    V = args.get("vectorize", (1,))[0]
    return [("partials", *PR.gemv_bwd_dx_partials(M, N, R, V)), ("fold", *PR.gemv_bwd_dx_fold(M // R, N))]


def gemm_derivations(M: int, N: int, K: int, tiles=((1, 1), (4, 8), (8, 4), (8, 8), (16, 8)), widths=(1, 4),
                     kwidths=(1, 4)):
    """GEMM derivations: the plain map of maps (vector columns or not) and the
    register tiles, with and without A read along k; only those whose rules'
    shapes divide (M, N, K)."""
    out = []
    for (R, Cn), V, KV in itertools.product(tiles, widths, kwidths):
        if (R, Cn) == (1, 1):
            if KV == 1 and N % V == 0:
                out.append(Derivation([Rule("vectorize", (V,))] if V > 1 else []))
            continue
        if M % R or N % Cn or Cn % V or K % KV:
            continue
        out.append(Derivation([Rule("tile", (R, Cn))] + ([Rule("vectorize", (V,))] if V > 1 else [])
                              + ([Rule("vectorize_k", (KV,))] if KV > 1 else [])))
    return out


def lower_gemm(d: Derivation, M: int, N: int, K: int, contract: str = "off"):
    """The GEMM phrase of a derivation (programs.gemm or programs.gemm_tiled)."""
    args = {r.name: r.args for r in d.rules}
    unknown = set(args) - {"tile", "vectorize", "vectorize_k"}
    if unknown:
        raise RuleError(f"no GEMM rule {sorted(unknown)}")
    R, Cn = args.get("tile", (1, 1))
    V = args.get("vectorize", (1,))[0]
    KV = args.get("vectorize_k", (1,))[0]
    if (R, Cn) == (1, 1):
        if KV > 1 or contract != "off":
            raise RuleError("vectorize_k and fma apply to tiled GEMMs")
        return PR.gemm(M, N, K, V)
    return PR.gemm_tiled(M, N, K, R, Cn, V, KV, contract=contract)


def explore_gemm(A, B, M: int, N: int, K: int, derivs=None, blocks=(128, 256), reps: int = 3):
    """Time every GEMM derivation (at each block size; the plain maps at their
    default launch) on A (M x K) and B (K x N); return [(ms, derivation, block)]
    fastest first."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch

    from ..tune import time_call
    from .build import compile_cuda

    derivs = derivs or gemm_derivations(M, N, K)

    def build(d):
        tag = "_".join(str(a) for r in d.rules for a in r.args) or "plain"
        return compile_cuda(f"xgemm_{M}_{N}_{K}_{tag}", *lower_gemm(d, M, N, K), unroll=1 if any(
            r.name == "tile" for r in d.rules) else 4)

    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    with ThreadPoolExecutor(workers) as pool:
        kernels = list(pool.map(build, derivs))
    C = torch.empty(M * N, device=A.device)
    results = []
    for d, k in zip(derivs, kernels):
        tiled = any(r.name == "tile" for r in d.rules)
        for blk in (blocks if tiled else (None,)):
            results.append((time_call(lambda: k.run(A, B, C, block=blk), reps=reps, warmup=1), d, blk))
    results.sort(key=lambda t: t[0])
    return results


# ---------------------------------------------------------------------------
# exploration: compile every derivation, time it, keep the fastest
# ---------------------------------------------------------------------------


def compile_pipeline(kind: str, d: Derivation, n: int, M: int = 0):
    """CUDA kernels of a derivation with their launch shapes: [(kernel, grid, block)]."""
    from .build import compile_cuda

    out = []
    for name, ph, ins in lower(kind, d, n, M):
        tag = f"{kind}_{name}_" + "_".join(str(a) for r in d.rules for a in r.args) + \
            ("_fm" if any(r.name == "fuse_maps" for r in d.rules) else "")
        k = compile_cuda(("x" + tag).replace("-", "_").replace(".", "_").replace(",", "_").replace(" ", ""),
                         ph, ins, unroll=4 if name in ("partials", "one_kernel") else 64)
        grid, block = k.default_launch()
        if name.startswith("fold") and name != "partials":  # a thread per group, blocks of 64 over many SMs
            rows = ph.type.n if isinstance(ph.type, P.Arr) else 1
            block = min(64, rows) if rows > 1 else 1
            grid = max(1, rows // block) if rows > 1 else 1
        out.append((k, grid, block))
    return out


def pipeline_buffers(pipe, device="cuda"):
    """Each kernel's output and zero-filled temporaries, allocated once (a
    kernel leaves its temporaries as it found them where that matters: the last
    block's ticket counter returns to zero)."""
    import torch

    bufs = []
    for k, _, _ in pipe:
        count = next(c for (_, _, c, role) in k.params if role == "out")
        bufs.append((torch.empty(count, device=device), k.temps_like(device)))
    return bufs


def run_pipeline(pipe, inputs, device="cuda", bufs=None):
    """Launch the kernels in order (into bufs, if given: nothing is allocated);
    return the final output tensor."""
    bufs = bufs or pipeline_buffers(pipe, device)
    cur = list(inputs)
    out = None
    for (k, grid, block), (out, temps) in zip(pipe, bufs):
        k.run(*cur, out, *temps, grid=grid, block=block)
        cur = [out]
    return out


def explore(kind: str, inputs, n: int, derivs=None, reps: int = 5, M: int = 0):
    """Time every derivation's pipeline on the inputs; return [(ms, derivation)]
    fastest first. The pipelines are compiled first, on several host threads."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    from ..tune import time_call

    derivs = derivs or (gemv_derivations(M, n) if kind == "gemv" else
                        gemv_dx_derivations(M, n) if kind == "gemv_dx" else derivations(n, kind=kind))
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    with ThreadPoolExecutor(workers) as pool:
        pipes = list(pool.map(lambda d: compile_pipeline(kind, d, n, M), derivs))
    results = []
    for d, pipe in zip(derivs, pipes):
        bufs = pipeline_buffers(pipe)  # timed: the launches only
        results.append((time_call(lambda: run_pipeline(pipe, inputs, bufs=bufs), reps=reps, warmup=2), d))
        del bufs
    results.sort(key=lambda t: t[0])
    return results
