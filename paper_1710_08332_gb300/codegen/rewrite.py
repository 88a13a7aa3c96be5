"""Rewrite-based exploration of strategies (the search Section 2.1 points to).

A reduction starts as a strategy-free expression over a small grammar

    E ::= Reduce E | Map f E | Each B E | Split s E | Columns T m E | Vec V E | Input xs
    B ::= E with a Hole for the element

starting from ``Reduce (Map f (Input xs))`` (dot: f = (*) over zip x y; asum:
f = abs). Rules rewrite the tree; each holds in real arithmetic for the
associative + with identity 0:

  split(s)       Reduce (Map f X)          -> Reduce (Each (Reduce (Map f Hole)) (Split s X))
  columns(T, m)  Each (Reduce (Map f Hole)) C
                                           -> Each (Reduce (Each (Reduce (Map f Hole))
                                                                 (Columns T m Hole))) C
  vectorize(V)   ... Split s (Input xs)     -> ... Split (s/V) (Vec V (Input xs)), the map and
                 the column folds then run lane-wise on num<V>, and each thread's V lane
                 results join the partials
  fuse, lower    Reduce (Map f col) -> reduceSeq (lambda (x, a). a + f x) 0 col; the Each
                 over Split -> mapWorkgroup, the Each over Columns -> mapLocal; the
                 outermost Reduce over the per-thread partials becomes folding kernels
                 (it reads what other blocks wrote: a kernel boundary)

``derivations`` enumerates rule sequences over parameter grids, ``rewrite``
applies one to the start expression (each rule checks the shape it rewrites),
and ``lower`` turns the resulting tree into kernel phrases. Each derivation's
result is exact for its own tree; different derivations round differently.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

from . import phrase as P
from . import programs as PR

# ---------------------------------------------------------------------------
# the strategy-free grammar
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Input:
    name: str            # "dot" (zip x y) or "asum" (x)


@dataclass(frozen=True)
class Hole:
    pass


@dataclass(frozen=True)
class Map:
    f: str               # "mul" (fst * snd) or "abs"
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


HOLE = Hole()


def start(kind: str):
    """Reduce (Map f (Input xs)) for kind in {"dot", "asum"}."""
    return Reduce(Map({"dot": "mul", "asum": "abs"}[kind], Input(kind)))


class RuleError(ValueError):
    pass


# ---------------------------------------------------------------------------
# rules
# ---------------------------------------------------------------------------


def r_split(e, s: int):
    if not (isinstance(e, Reduce) and isinstance(e.e, Map) and isinstance(e.e.e, Input)):
        raise RuleError("split rewrites Reduce (Map f (Input xs))")
    return Reduce(Each(Reduce(Map(e.e.f, HOLE)), Split(s, e.e.e)))


def r_columns(e, T: int, m: str):
    ok = (isinstance(e, Reduce) and isinstance(e.e, Each) and isinstance(e.e.body, Reduce)
          and isinstance(e.e.body.e, Map) and e.e.body.e.e == HOLE)
    if not ok:
        raise RuleError("columns rewrites the per-chunk Reduce (Map f Hole)")
    f = e.e.body.e.f
    return Reduce(Each(Reduce(Each(Reduce(Map(f, HOLE)), Columns(T, m, HOLE))), e.e.e))


def r_vectorize(e, V: int):
    def go(x):
        if isinstance(x, Split) and isinstance(x.e, Input):
            if x.s % V:
                raise RuleError(f"split {x.s} is not a multiple of the width {V}")
            return Split(x.s // V, Vec(V, x.e))
        if isinstance(x, Reduce):
            return Reduce(go(x.e))
        if isinstance(x, Each):
            return Each(x.body, go(x.e))
        raise RuleError("vectorize needs the split input")
    return go(e)


RULES = {"split": r_split, "columns": r_columns, "vectorize": r_vectorize}


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


def _elem_fn(f: str):
    if f == "mul":
        return lambda x: P.mul(P.fst(x), P.snd(x))
    return lambda x: P.abs_(x)


def lower(kind: str, d: Derivation, n: int):
    """Kernel phrases for a derivation: [(name, phrase, inputs), ...]: the
    per-thread partials, then folding kernels down to one number."""
    e = rewrite(kind, d)
    # expected shape: Reduce (Each (Reduce (Each (Reduce (Map f Hole)) (Columns T m Hole))) (Split s S))
    try:
        chunk_each = e.e
        col_each = chunk_each.body.e
        f = col_each.body.e.f
        T, m = col_each.e.T, col_each.e.m
        sp = chunk_each.e
        s, stream = sp.s, sp.e
    except AttributeError as exc:
        raise RuleError(f"derivation {d} does not reach the lowerable shape") from exc
    V = stream.V if isinstance(stream, Vec) else 1
    if kind == "dot":
        x, y = P.inp("x", P.arr(n, P.F32)), P.inp("y", P.arr(n, P.F32))
        ins = [x, y]
        xs = P.zip_(x, y) if V == 1 else P.zip_(P.asVector(V, x), P.asVector(V, y))
    else:
        x = P.inp("x", P.arr(n, P.F32))
        ins = [x]
        xs = x if V == 1 else P.asVector(V, x)
    g = _elem_fn(f)
    zero = P.lit(0.0) if V == 1 else P.vlit(0.0, V)
    first = P.join(P.mapWorkgroup(
        lambda chunk: P.mapLocal(lambda col: P.reduceSeq(lambda v, a: P.add(a, g(v)), zero, col),
                                 PR.columns(chunk, T, m)),
        P.split(s, xs)))
    kernels = [("partials", first, ins)]
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
                maps=("interleaved", "contig"), widths=(1, 4)):
    """Every derivation over the parameter grids whose rules apply."""
    out = []
    for s, T, m, V in itertools.product(splits, threads, maps, widths):
        if n % s or (s // V) % T or s % V:
            continue
        rules = [Rule("split", (s,)), Rule("columns", (T, m))]
        if V > 1:
            rules.append(Rule("vectorize", (V,)))
        rules += [Rule("fuse"), Rule("lower")]
        out.append(Derivation(rules))
    return out


# ---------------------------------------------------------------------------
# exploration: compile every derivation, time it, keep the fastest
# ---------------------------------------------------------------------------


def compile_pipeline(kind: str, d: Derivation, n: int):
    """CUDA kernels of a derivation with their launch shapes: [(kernel, grid, block)]."""
    from .build import compile_cuda

    out = []
    for name, ph, ins in lower(kind, d, n):
        tag = f"{kind}_{name}_" + "_".join(str(a) for r in d.rules for a in r.args)
        k = compile_cuda(("x" + tag).replace("-", "_"), ph, ins, unroll=4 if name == "partials" else 64)
        grid, block = k.default_launch()
        if name.startswith("fold") and name != "partials":  # a thread per group, blocks of 64 over many SMs
            rows = ph.type.n if isinstance(ph.type, P.Arr) else 1
            block = min(64, rows) if rows > 1 else 1
            grid = max(1, rows // block) if rows > 1 else 1
        out.append((k, grid, block))
    return out


def run_pipeline(pipe, inputs, device="cuda"):
    """Launch the kernels in order; return the final one-element tensor."""
    import torch

    cur = list(inputs)
    out = None
    for k, grid, block in pipe:
        count = next(c for (_, _, c, role) in k.params if role == "out")
        out = torch.empty(count, device=device)
        k.run(*cur, out, *k.temps_like(device), grid=grid, block=block)
        cur = [out]
    return out


def explore(kind: str, inputs, n: int, derivs=None, reps: int = 5):
    """Time every derivation's pipeline on the inputs; return [(ms, derivation)] fastest first."""
    from ..tune import time_call

    results = []
    for d in derivs or derivations(n):
        pipe = compile_pipeline(kind, d, n)
        results.append((time_call(lambda: run_pipeline(pipe, inputs), reps=reps, warmup=2), d))
    results.sort(key=lambda t: t[0])
    return results
