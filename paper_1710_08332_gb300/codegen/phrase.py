"""Functional phrases: the data-parallel primitives of the paper's source
language (Sections 2.1, 3.3 and 6.2), with their types.

A phrase is built from inputs (``Ident``), literals, arithmetic on numbers,
``map`` at a level of the GPU hierarchy (mapGlobal / mapWorkgroup / mapLocal /
mapSeq, and between work-group and work-item the warp: mapWarp over a block's
warps, mapLane over a warp's 32 lanes), the sequential ``reduce``
(reduceSeq), and the data-layout primitives ``zip``, ``fst``, ``snd``,
``split``, ``join``, ``transpose``, ``asVector`` and ``asScalar`` (vectors
num<V> of Section 6.2, + - * lane-wise) and ``lanes`` (a vector's V numbers
as an array); ``to_private`` / ``to_local`` / ``to_global`` choose the
address space of a map's output when it becomes a temporary (Section 6.2,
address spaces). Types are checked as the phrase is built: a number type, an
array ``n.d`` or a pair.

Two constructs go beyond the paper's primitives, each with a plain meaning:
``reduceTree lane f xs`` reduces L <= 32 numbers (L a power of two) by the
halving tree -- element l becomes f(x_l, x_{l + L/2}), repeated until one
remains -- one number per lane of a warp (on the GPU, warp shuffles); and
``secondLevel parts f`` is f applied to the array ``parts`` that a work-group
map produces: the work-groups write their parts, and f runs in one work-group
once all of them have (the join and second-level reduce of Section 2.1 in
the same kernel, by the last work-group to finish).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

LEVELS = ("global", "workgroup", "warp", "lane", "local", "seq")
WARP = 32  # lanes of a warp
SPACES = ("global", "local", "private")

# ---------------------------------------------------------------------------
# data types
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Num:
    dtype: str  # "f32", "i32" or "i64"

    def __post_init__(self):
        if self.dtype not in ("f32", "i32", "i64"):
            raise TypeError(f"unknown number type {self.dtype}")

    def __str__(self):
        return self.dtype


@dataclass(frozen=True)
class Arr:
    n: int
    elem: object

    def __post_init__(self):
        if not isinstance(self.n, int) or self.n < 0:
            raise TypeError(f"array length must be a natural number, not {self.n!r}")

    def __str__(self):
        return f"{self.n}.{self.elem}"


@dataclass(frozen=True)
class PairT:
    a: object
    b: object

    def __str__(self):
        return f"({self.a} x {self.b})"


@dataclass(frozen=True)
class VecT:
    """num<V> (Section 6.2's vector data type): V numbers handled as one value."""
    n: int
    num: Num

    def __post_init__(self):
        if self.n not in (2, 4):
            raise TypeError(f"vector width {self.n} (2 or 4)")
        if self.num.dtype != "f32":
            raise TypeError("vectors of f32 only")

    def __str__(self):
        return f"{self.num}<{self.n}>"


F32, I32, I64 = Num("f32"), Num("i32"), Num("i64")


def is_scalar(t) -> bool:
    """A number or a vector of numbers: a value one thread holds in registers."""
    return isinstance(t, (Num, VecT))


def is_value(t) -> bool:
    """A number, a vector, or a pair of them (e.g. a compensated sum's (s, c))."""
    return is_scalar(t) or (isinstance(t, PairT) and is_scalar(t.a) and is_scalar(t.b))


def _num_or_num_pair(t) -> bool:
    """A number, or a pair of two numbers of one type (a compensated sum's (s, c))."""
    return isinstance(t, Num) or (isinstance(t, PairT) and isinstance(t.a, Num) and t.a == t.b)


def is_num_array(t) -> bool:
    """An array (of arrays ...) of numbers or of vectors of numbers."""
    return isinstance(t, Arr) and isinstance(base_elem(t), (Num, VecT))


def arr(*dims_and_elem):
    """arr(n, m, F32) is the type n.m.f32."""
    *dims, elem = dims_and_elem
    t = elem
    for d in reversed(dims):
        t = Arr(int(d), t)
    return t


def scalar_count(t) -> int:
    """Numbers in a value of type t (arrays of numbers, vectors or pairs of numbers)."""
    if isinstance(t, Num):
        return 1
    if isinstance(t, VecT):
        return t.n
    if isinstance(t, PairT) and isinstance(t.a, Num) and t.a == t.b:
        return 2
    if isinstance(t, Arr):
        return t.n * scalar_count(t.elem)
    raise TypeError(f"{t} is not an array of numbers")


def base_num(t) -> Num:
    while isinstance(t, Arr):
        t = t.elem
    if isinstance(t, VecT):
        return t.num
    if isinstance(t, PairT) and isinstance(t.a, Num) and t.a == t.b:
        return t.a
    if not isinstance(t, Num):
        raise TypeError(f"{t} is not an array of numbers")
    return t


def base_elem(t):
    """The number or vector type at the bottom of an array type."""
    while isinstance(t, Arr):
        t = t.elem
    return t


# ---------------------------------------------------------------------------
# phrases
# ---------------------------------------------------------------------------

_names = itertools.count()


def fresh(prefix: str) -> str:
    return f"{prefix}{next(_names)}"


class Phrase:
    type: object

    def children(self):
        return ()

    def computes(self) -> bool:
        """True if evaluating the phrase runs a map or a reduce (it is not a
        pure view of its inputs or arithmetic on numbers)."""
        return any(c.computes() for c in self.children())


@dataclass(eq=False)
class Ident(Phrase):
    name: str
    type: object
    temp: str | None = None  # address space if the identifier names a temporary


@dataclass(eq=False)
class Lit(Phrase):
    value: float
    type: object = F32


@dataclass(eq=False)
class Bin(Phrase):
    op: str  # "+", "-", "*"
    a: Phrase
    b: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if self.op not in ("+", "-", "*"):
            raise TypeError(f"unknown operator {self.op}")
        if not is_scalar(self.a.type) or self.a.type != self.b.type:
            raise TypeError(f"{self.op} needs two numbers (or vectors) of one type, "
                            f"not {self.a.type} and {self.b.type}")
        self.type = self.a.type

    def children(self):
        return (self.a, self.b)


@dataclass(eq=False)
class Fma(Phrase):
    """fma a b c: a * b + c rounded once (the contraction a strategy may
    declare), on numbers or lane by lane on vectors."""
    a: Phrase
    b: Phrase
    c: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.a.type
        if not (t == F32 or (isinstance(t, VecT) and t.num == F32)) or self.b.type != t or self.c.type != t:
            raise TypeError(f"fma needs three f32 numbers (or vectors) of one type, not "
                            f"{self.a.type}, {self.b.type}, {self.c.type}")
        self.type = t

    def children(self):
        return (self.a, self.b, self.c)


@dataclass(eq=False)
class Abs(Phrase):
    a: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if self.a.type != F32 and not isinstance(self.a.type, VecT):
            raise TypeError("abs of a non-f32")
        self.type = self.a.type

    def children(self):
        return (self.a,)


@dataclass(eq=False)
class Splat(Phrase):
    """splat V e: the vector num<V> whose V lanes are all the number e (the
    widening of a number to a vector in vector arithmetic, Section 6.2)."""
    n: int
    a: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if self.a.type != F32:
            raise TypeError(f"splat of a {self.a.type} (f32 numbers only)")
        self.type = VecT(self.n, self.a.type)

    def children(self):
        return (self.a,)


@dataclass(eq=False)
class Lam:
    """A function of one or two phrases (the body refers to the parameters)."""
    params: tuple
    body: Phrase


def lam(param_types, fn):
    """lam([t1, t2], lambda a, b: ...) builds a function phrase."""
    params = tuple(Ident(fresh("p"), t) for t in param_types)
    return Lam(params, fn(*params))


@dataclass(eq=False)
class Map(Phrase):
    level: str
    f: Lam
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if self.level not in LEVELS:
            raise TypeError(f"unknown level {self.level}")
        if not isinstance(self.e.type, Arr):
            raise TypeError(f"map over a non-array {self.e.type}")
        if len(self.f.params) != 1 or self.f.params[0].type != self.e.type.elem:
            raise TypeError(f"map function takes {[p.type for p in self.f.params]}, elements are {self.e.type.elem}")
        self.type = Arr(self.e.type.n, self.f.body.type)

    def children(self):
        return (self.e, self.f.body)

    def computes(self):
        return True


@dataclass(eq=False)
class Reduce(Phrase):
    """reduceSeq f init e: a left fold, f(element, accumulator) (Section 4.2's reduceI).
    The accumulator is a number, a vector, a pair of them, or an array of
    numbers (a private array: e.g. a thread's tile of C in a GEMM)."""
    f: Lam
    init: Phrase
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if not isinstance(self.e.type, Arr):
            raise TypeError(f"reduce over a non-array {self.e.type}")
        if not (is_value(self.init.type) or is_num_array(self.init.type)):
            raise TypeError("reduce accumulates numbers, vectors, pairs of them or arrays of numbers")
        ps = self.f.params
        if len(ps) != 2 or ps[0].type != self.e.type.elem or ps[1].type != self.init.type:
            raise TypeError("reduce function must take (element, accumulator)")
        if self.f.body.type != self.init.type:
            raise TypeError("reduce function must return the accumulator type")
        self.type = self.init.type

    def children(self):
        return (self.init, self.e, self.f.body)

    def computes(self):
        return True


@dataclass(eq=False)
class Zip(Phrase):
    a: Phrase
    b: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        ta, tb = self.a.type, self.b.type
        if not (isinstance(ta, Arr) and isinstance(tb, Arr) and ta.n == tb.n):
            raise TypeError(f"zip of {ta} and {tb}")
        self.type = Arr(ta.n, PairT(ta.elem, tb.elem))

    def children(self):
        return (self.a, self.b)


@dataclass(eq=False)
class Pair(Phrase):
    """pair a b of two numbers (or vectors)."""
    a: Phrase
    b: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if not (is_scalar(self.a.type) and is_scalar(self.b.type)):
            raise TypeError(f"pair of {self.a.type} and {self.b.type}")
        self.type = PairT(self.a.type, self.b.type)

    def children(self):
        return (self.a, self.b)


@dataclass(eq=False)
class Proj(Phrase):
    k: int  # 0 = fst, 1 = snd
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if not isinstance(self.e.type, PairT):
            raise TypeError(f"projection of a non-pair {self.e.type}")
        self.type = self.e.type.a if self.k == 0 else self.e.type.b

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class Split(Phrase):
    n: int
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if not isinstance(t, Arr) or self.n <= 0 or t.n % self.n:
            raise TypeError(f"split {self.n} of {t}")
        self.type = Arr(t.n // self.n, Arr(self.n, t.elem))

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class Join(Phrase):
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if not (isinstance(t, Arr) and isinstance(t.elem, Arr)):
            raise TypeError(f"join of {t}")
        self.type = Arr(t.n * t.elem.n, t.elem.elem)

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class Transpose(Phrase):
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if not (isinstance(t, Arr) and isinstance(t.elem, Arr)):
            raise TypeError(f"transpose of {t}")
        self.type = Arr(t.elem.n, Arr(t.n, t.elem.elem))

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class AsVector(Phrase):
    """asVector V: (mV).num -> m.num<V> (Section 6.2), read as V-wide loads."""
    n: int
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if not (isinstance(t, Arr) and isinstance(t.elem, Num) and t.n % self.n == 0):
            raise TypeError(f"asVector {self.n} of {t}")
        self.type = Arr(t.n // self.n, VecT(self.n, t.elem))

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class AsScalar(Phrase):
    """asScalar: m.num<V> -> (mV).num."""
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if not (isinstance(t, Arr) and isinstance(t.elem, VecT)):
            raise TypeError(f"asScalar of {t}")
        self.type = Arr(t.n * t.elem.n, t.elem.num)

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class To(Phrase):
    """to_global / to_local / to_private: where e's result lives if it becomes a temporary."""
    space: str
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        if self.space not in SPACES:
            raise TypeError(f"unknown address space {self.space}")
        self.type = self.e.type

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class Idx(Phrase):
    """Element i of an array phrase (i an index expression); produced by the translation."""
    e: Phrase
    i: object
    type: object = field(init=False)

    def __post_init__(self):
        if not isinstance(self.e.type, Arr):
            raise TypeError(f"index into a non-array {self.e.type}")
        self.type = self.e.type.elem

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class Lanes(Phrase):
    """lanes: num<V> -> V.num, the vector's numbers as an array (a view); of a
    pair of vectors (num<V> x num<V>) -> V.(num x num), lane v's pair."""
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if isinstance(t, VecT):
            self.type = Arr(t.n, t.num)
        elif isinstance(t, PairT) and isinstance(t.a, VecT) and t.a == t.b:
            self.type = Arr(t.a.n, PairT(t.a.num, t.a.num))
        else:
            raise TypeError(f"lanes of a non-vector {t}")

    def children(self):
        return (self.e,)


@dataclass(eq=False)
class ReduceTree(Phrase):
    """reduceTree lane f xs: the halving tree over L = len xs numbers, L a power
    of two no larger than a warp: while L > 1, x_l := f(x_l, x_{l + L/2}) for
    l < L/2, L := L/2; the result is x_0."""
    level: str
    f: Lam
    e: Phrase
    type: object = field(init=False)

    def __post_init__(self):
        t = self.e.type
        if self.level != "lane":
            raise TypeError(f"reduceTree at level {self.level}: trees run over the lanes of a warp")
        if not (isinstance(t, Arr) and _num_or_num_pair(t.elem) and t.n >= 1 and t.n & (t.n - 1) == 0
                and t.n <= WARP):
            raise TypeError(f"reduceTree over {t}: a power-of-two array of at most {WARP} numbers "
                            f"(or pairs of numbers)")
        ps = self.f.params
        if len(ps) != 2 or ps[0].type != t.elem or ps[1].type != t.elem or self.f.body.type != t.elem:
            raise TypeError("reduceTree's function combines two elements into one")
        self.type = t.elem

    def children(self):
        return (self.e, self.f.body)

    def computes(self):
        return True


@dataclass(eq=False)
class SecondLevel(Phrase):
    """secondLevel parts f: f applied to the array of per-work-group parts, in
    one work-group after every work-group has written its part."""
    parts: Phrase
    f: Lam
    type: object = field(init=False)

    def __post_init__(self):
        if not isinstance(self.parts.type, Arr) or not _num_or_num_pair(base_elem(self.parts.type)):
            raise TypeError(f"second level over {self.parts.type}: an array of numbers (or pairs of numbers)")
        if len(self.f.params) != 1 or self.f.params[0].type != self.parts.type:
            raise TypeError("the second level's function takes the array of parts")
        self.type = self.f.body.type

    def children(self):
        return (self.parts, self.f.body)

    def computes(self):
        return True


# ---------------------------------------------------------------------------
# constructors in the paper's notation
# ---------------------------------------------------------------------------


def map_at(level, f, e, *, param_type=None):
    """map at a level; f is a Python function of one phrase."""
    t = e.type.elem if isinstance(e.type, Arr) else None
    return Map(level, lam([param_type or t], f), e)


def mapGlobal(f, e):
    return map_at("global", f, e)


def mapWorkgroup(f, e):
    return map_at("workgroup", f, e)


def mapLocal(f, e):
    return map_at("local", f, e)


def mapSeq(f, e):
    return map_at("seq", f, e)


def mapWarp(f, e):
    """map over the warps of a work-group (one element per warp)."""
    return map_at("warp", f, e)


def mapLane(f, e):
    """map over the 32 lanes of a warp (one element per lane)."""
    return map_at("lane", f, e)


def lanes(e):
    return Lanes(e)


def reduceTree(f, e, level="lane"):
    """f is a Python function (a, b) -> combined element."""
    t = e.type.elem if isinstance(e.type, Arr) else None
    return ReduceTree(level, lam([t, t], f), e)


def secondLevel(parts, fn):
    """fn is a Python function of the array of parts."""
    return SecondLevel(parts, lam([parts.type], fn))


def reduceSeq(f, init, e):
    """f is a Python function (element, accumulator) -> accumulator."""
    if not isinstance(init, Phrase):
        init = Lit(float(init), F32)
    return Reduce(lam([e.type.elem, init.type], f), init, e)


def zip_(a, b):
    return Zip(a, b)


def fst(e):
    return Proj(0, e)


def snd(e):
    return Proj(1, e)


def pair(a, b):
    return Pair(a, b)


def split(n, e):
    return Split(int(n), e)


def join(e):
    return Join(e)


def transpose(e):
    return Transpose(e)


def asVector(n, e):
    return AsVector(int(n), e)


def asScalar(e):
    return AsScalar(e)


def alit(v, t):
    """The array of type t (of numbers) with every element v."""
    if not is_num_array(t):
        raise TypeError(f"an array literal of {t}: arrays of numbers or vectors only")
    return Lit(v, t)


def vlit(v, n=4):
    """The vector with every lane v."""
    return Lit(v, VecT(n, F32))


def splat(n, e):
    """The vector of n copies of the number e."""
    return Splat(n, e)


def to_private(e):
    return To("private", e)


def to_local(e):
    return To("local", e)


def to_global(e):
    return To("global", e)


def lit(v, t=F32):
    return Lit(v, t)


def add(a, b):
    return Bin("+", a, b)


def mul(a, b):
    return Bin("*", a, b)


def sub(a, b):
    return Bin("-", a, b)


def fma(a, b, c):
    """a * b + c with one rounding."""
    return Fma(a, b, c)


def abs_(a):
    return Abs(a)


def inp(name, t):
    """A kernel input of type t (an array of numbers, or a number)."""
    return Ident(name, t)


# ---------------------------------------------------------------------------
# substitution (beta reduction of a function applied to a phrase)
# ---------------------------------------------------------------------------


def subst(p: Phrase, env: dict) -> Phrase:
    """p with every identifier named in env replaced by env[name]."""
    if isinstance(p, Ident):
        return env.get(p.name, p)
    if isinstance(p, Lit):
        return p
    if isinstance(p, Bin):
        return Bin(p.op, subst(p.a, env), subst(p.b, env))
    if isinstance(p, Abs):
        return Abs(subst(p.a, env))
    if isinstance(p, Splat):
        return Splat(p.n, subst(p.a, env))
    if isinstance(p, Fma):
        return Fma(subst(p.a, env), subst(p.b, env), subst(p.c, env))
    if isinstance(p, Map):
        return Map(p.level, Lam(p.f.params, subst(p.f.body, env)), subst(p.e, env))
    if isinstance(p, Reduce):
        return Reduce(Lam(p.f.params, subst(p.f.body, env)), subst(p.init, env), subst(p.e, env))
    if isinstance(p, Zip):
        return Zip(subst(p.a, env), subst(p.b, env))
    if isinstance(p, Proj):
        return Proj(p.k, subst(p.e, env))
    if isinstance(p, Pair):
        return Pair(subst(p.a, env), subst(p.b, env))
    if isinstance(p, Split):
        return Split(p.n, subst(p.e, env))
    if isinstance(p, Join):
        return Join(subst(p.e, env))
    if isinstance(p, Transpose):
        return Transpose(subst(p.e, env))
    if isinstance(p, To):
        return To(p.space, subst(p.e, env))
    if isinstance(p, AsVector):
        return AsVector(p.n, subst(p.e, env))
    if isinstance(p, AsScalar):
        return AsScalar(subst(p.e, env))
    if isinstance(p, Idx):
        return Idx(subst(p.e, env), p.i)
    if isinstance(p, Lanes):
        return Lanes(subst(p.e, env))
    if isinstance(p, ReduceTree):
        return ReduceTree(p.level, Lam(p.f.params, subst(p.f.body, env)), subst(p.e, env))
    if isinstance(p, SecondLevel):
        return SecondLevel(subst(p.parts, env), Lam(p.f.params, subst(p.f.body, env)))
    raise TypeError(f"cannot substitute into {type(p).__name__}")


def apply(f: Lam, *args: Phrase) -> Phrase:
    if len(args) != len(f.params):
        raise TypeError("wrong number of arguments")
    return subst(f.body, {p.name: a for p, a in zip(f.params, args)})
