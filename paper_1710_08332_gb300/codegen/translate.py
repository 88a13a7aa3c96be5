"""From functional phrases to an imperative loop nest (the paper's Stages I
and II, Sections 4.1 and 4.2).

Stage I is the pair of translations: the acceptor-passing translation
``A(E, out)`` produces a command that writes the value of E through the
acceptor ``out``, and the continuation-passing translation ``C(E, k)``
produces a command that computes E and hands the resulting expression to the
continuation k. Data-layout primitives (zip, split, join, transpose, fst,
snd) never compute: C passes them on as views and A pushes them onto the
acceptor (a split value is written through a "split acceptor", and so on).
Stage II replaces the intermediate combinators by their definitions: mapI at
a level becomes a parallel for at that level, and reduceI becomes a new
private accumulator, its initialisation, a sequential for loop and the
continuation applied to the accumulator.

The result is a command tree of ``New`` (a temporary in an address space),
``For`` (a loop at a level), ``Assign`` (acceptor := expression) and ``Seq``,
plus ``TreeReduce`` (a lane tree: each lane's element written into a
buffer, then the halving tree over it) and ``LastBlock`` (a command run by
the last work-group to finish the kernel's work-group loop: the second level).
Nested maps must run at strictly finer levels (workgroup > local > seq;
workgroup > warp > lane > seq; global > seq), the legality rule the paper's
conclusion asks for.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import phrase as P

# ---------------------------------------------------------------------------
# index expressions
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class IVar:
    name: str


@dataclass(frozen=True)
class IConst:
    v: int


@dataclass(frozen=True)
class IOp:
    op: str  # "+", "*", "/", "%"
    a: object
    b: object


def iadd(a, b):
    if isinstance(a, IConst) and a.v == 0:
        return b
    if isinstance(b, IConst) and b.v == 0:
        return a
    if isinstance(a, IConst) and isinstance(b, IConst):
        return IConst(a.v + b.v)
    # (x / n) * n + x % n = x for the non-negative x of an index (a join of a split)
    if (isinstance(a, IOp) and a.op == "*" and isinstance(a.a, IOp) and a.a.op == "/" and a.a.b == a.b
            and isinstance(b, IOp) and b.op == "%" and b.b == a.b and b.a == a.a.a):
        return b.a
    return IOp("+", a, b)


def imul(a, n: int):
    if n == 0:
        return IConst(0)
    if n == 1:
        return a
    if isinstance(a, IConst):
        return IConst(a.v * n)
    return IOp("*", a, IConst(n))


def _multiple(a, n: int) -> bool:
    """a is a multiple of n for every value of its variables (a sum of multiples)."""
    if isinstance(a, IConst):
        return a.v % n == 0
    if isinstance(a, IOp):
        if a.op == "+":
            return _multiple(a.a, n) and _multiple(a.b, n)
        if a.op == "*" and isinstance(a.b, IConst):
            return a.b.v % n == 0 or _multiple(a.a, n)
    return False


def idiv(a, n: int):
    if n == 1:
        return a
    if isinstance(a, IConst):
        return IConst(a.v // n)
    if isinstance(a, IOp) and a.op == "*" and isinstance(a.b, IConst) and a.b.v % n == 0:
        return imul(a.a, a.b.v // n)
    if isinstance(a, IOp) and a.op == "+" and _multiple(a.a, n) and _multiple(a.b, n):
        return iadd(idiv(a.a, n), idiv(a.b, n))
    return IOp("/", a, IConst(n))


def imod(a, n: int):
    if n == 1 or _multiple(a, n):
        return IConst(0)
    if isinstance(a, IConst):
        return IConst(a.v % n)
    return IOp("%", a, IConst(n))


# ---------------------------------------------------------------------------
# acceptors and commands
# ---------------------------------------------------------------------------


@dataclass(eq=False)
class Temp:
    """A temporary (Section 4's new): its type, address space and the
    parallel loops it is hoisted out of (Section 6.4) -- filled in later."""
    name: str
    type: object
    space: str
    hoist: list = field(default_factory=list)  # [(loop variable, trip count)] outermost first
    lanes: bool = False  # a lane tree's buffer: element l belongs to lane l of the warp


class Acc:
    pass


@dataclass(eq=False)
class AOut(Acc):
    """The kernel's output array, or a temporary."""
    name: str
    type: object
    temp: Temp | None = None


@dataclass(eq=False)
class AIdx(Acc):
    acc: Acc
    i: object


@dataclass(eq=False)
class ASplit(Acc):
    """A(split n e, out) writes e through ASplit(n, out): e's element [q] goes
    to out[q / n][q % n]."""
    n: int
    acc: Acc


@dataclass(eq=False)
class AJoin(Acc):
    """A(join e, out) writes e (inner length m) through AJoin(m, out): e's
    element [i][j] goes to out[i*m + j]."""
    m: int
    acc: Acc


@dataclass(eq=False)
class AProj(Acc):
    """Acceptor for one component (0 = fst, 1 = snd) of a pair acceptor."""
    k: int
    acc: Acc


@dataclass(eq=False)
class AAsScalar(Acc):
    """A(asScalar e, out) writes e's vectors (width V) whole into the scalar array out."""
    V: int
    acc: Acc


@dataclass(eq=False)
class ATranspose(Acc):
    """Acceptor for a transposed value: element [i][j] goes to acc[j][i]."""
    acc: Acc


class Comm:
    pass


@dataclass(eq=False)
class Seq(Comm):
    cs: list


@dataclass(eq=False)
class Assign(Comm):
    acc: Acc
    e: P.Phrase


@dataclass(eq=False)
class New(Comm):
    temp: Temp
    body: Comm


@dataclass(eq=False)
class For(Comm):
    var: IVar
    n: int
    level: str
    body: Comm


@dataclass(eq=False)
class TreeReduce(Comm):
    """fill writes element l of buf (an L-array, L a power of two <= 32) at
    level ``level``; then, while L > 1, buf[l] := f(buf[l], buf[l + L/2]) for
    l < L/2 and L := L/2; finally res := buf[0]."""
    level: str
    buf: Temp
    fill: Comm
    f: object  # P.Lam of two elements
    res: Temp


@dataclass(eq=False)
class LastBlock(Comm):
    """body runs once, in the last work-group to finish everything before it
    (every work-group takes a ticket from the counter ``ticket``; the one that
    draws the last runs body and puts the counter back to zero)."""
    body: Comm
    ticket: Temp


class TranslationError(Exception):
    pass


# ---------------------------------------------------------------------------
# Stage I + II
# ---------------------------------------------------------------------------

# the levels a parallel map at each level may contain (sequential maps nest anywhere)
FINER = {"workgroup": ("local", "warp"), "warp": ("lane",)}


class Translator:
    def __init__(self):
        self.count = 0

    def ivar(self, prefix="i"):
        self.count += 1
        return IVar(f"{prefix}{self.count}")

    def temp(self, t, space):
        self.count += 1
        return Temp(f"t{self.count}", t, space)

    # -- legality of nested levels ------------------------------------------

    @staticmethod
    def check_nesting(outer: list, level: str):
        if level == "seq":
            return
        if not outer:
            if level in ("warp", "lane"):
                raise TranslationError(f"illegal nesting: a {level} map outside a "
                                       f"{'workgroup' if level == 'warp' else 'warp'} map")
            return
        last = outer[-1]
        if level not in FINER.get(last, ()):
            raise TranslationError(f"illegal nesting: a {level} map inside a {last} map "
                                   f"(a nested map must run at a strictly finer level)")

    # -- A: acceptor-passing ------------------------------------------------

    def A(self, e: P.Phrase, out: Acc, levels: list) -> Comm:
        if isinstance(e, P.Map):
            self.check_nesting(levels, e.level)

            def body(x):
                i = self.ivar()
                inner = self.A(P.apply(e.f, P.Idx(x, i)), AIdx(out, i), levels + [e.level])
                return For(i, e.e.type.n, e.level, inner)

            return self.C(e.e, body, levels)
        if isinstance(e, P.Reduce):
            return self.C(e, lambda v: self.assign(out, v, levels), levels)
        if isinstance(e, P.SecondLevel):
            return self.second_level(e, out, levels)
        if isinstance(e, P.Split):
            return self.A(e.e, ASplit(e.n, out), levels)
        if isinstance(e, P.Join):
            return self.A(e.e, AJoin(e.e.type.elem.n, out), levels)
        if isinstance(e, P.Transpose):
            return self.A(e.e, ATranspose(out), levels)
        if isinstance(e, P.To):
            return self.A(e.e, out, levels)
        if isinstance(e, P.AsScalar) and e.computes():
            return self.A(e.e, AAsScalar(e.e.type.elem.n, out), levels)
        if isinstance(e, P.Pair):
            return Seq([self.A(e.a, AProj(0, out), levels), self.A(e.b, AProj(1, out), levels)])
        if isinstance(e.type, P.PairT) and P.is_value(e.type):
            return self.C(e, lambda v: Seq([Assign(AProj(0, out), P.Proj(0, v)),
                                            Assign(AProj(1, out), P.Proj(1, v))]), levels)
        if P.is_scalar(e.type):
            return self.C(e, lambda v: Assign(out, v), levels)
        if isinstance(e.type, P.Arr) and not e.computes():
            # a view of arrays written out element by element (mapSeq id)
            return self.copy(e, out, levels)
        if isinstance(e, (P.Zip, P.Proj)):
            return self.C(e, lambda v: self.copy(v, out, levels), levels)
        raise TranslationError(f"cannot write a {type(e).__name__} through an acceptor")

    def assign(self, out, v, levels):
        if P.is_scalar(v.type):
            return Assign(out, v)
        if isinstance(v.type, P.PairT):
            return Seq([Assign(AProj(0, out), P.Proj(0, v)), Assign(AProj(1, out), P.Proj(1, v))])
        return self.copy(v, out, levels)

    def copy(self, v: P.Phrase, out: Acc, levels: list) -> Comm:
        if P.is_scalar(v.type):
            return Assign(out, v)
        if not isinstance(v.type, P.Arr):
            raise TranslationError(f"cannot copy a value of type {v.type}")
        i = self.ivar()
        return For(i, v.type.n, "seq", self.copy(P.Idx(v, i), AIdx(out, i), levels + ["seq"]))

    def second_level(self, e: P.SecondLevel, out: Acc, levels: list) -> Comm:
        """The work-groups write their parts into a global temporary; the last
        to finish applies f to it in one work-group (levels: inside a
        work-group), writing the kernel's output."""
        if levels:
            raise TranslationError("the second level closes a kernel: it must be the kernel's whole expression")
        g = self.temp(e.parts.type, "global")
        gv = P.Ident(g.name, g.type, temp="global")
        ticket = self.temp(P.I32, "global")
        first = self.A(e.parts, AOut(g.name, g.type, g), [])
        body = self.A(P.apply(e.f, gv), out, ["workgroup"])
        return New(g, New(ticket, Seq([first, LastBlock(body, ticket)])))

    def tree(self, e: P.ReduceTree, k, levels: list) -> Comm:
        """reduceTree lane: inside a warp map, lane l holds element l of the
        array (a lane map fills it directly), then the halving tree."""
        if not levels or levels[-1] != "warp":
            raise TranslationError("a lane tree runs directly inside a warp map")
        L = e.e.type.n
        buf = self.temp(e.e.type, "private")
        buf.lanes = True
        res = self.temp(e.type, "private")
        bacc = AOut(buf.name, buf.type, buf)
        src = e.e
        if isinstance(src, P.Map) and src.level == "lane":
            fill = self.A(src, bacc, levels)
        elif not src.computes():
            i = self.ivar("l")
            fill = For(i, L, "lane", self.A(P.Idx(src, i), AIdx(bacc, i), levels + ["lane"]))
        else:
            def copy_in(v):
                i = self.ivar("l")
                return For(i, L, "lane", self.A(P.Idx(v, i), AIdx(bacc, i), levels + ["lane"]))
            fill = self.C(src, copy_in, levels)
        rv = P.Ident(res.name, res.type, temp="private")
        return New(res, Seq([TreeReduce("lane", buf, fill, e.f, res), k(rv)]))

    # -- C: continuation-passing --------------------------------------------

    def C(self, e: P.Phrase, k, levels: list) -> Comm:
        if not e.computes():
            return k(e)
        if isinstance(e, P.Reduce):
            # reduceI: new accumulator := init; for i: acc := f(x[i], acc); k(acc)
            def body(x):
                t = self.temp(e.type, "private")
                tv = P.Ident(t.name, t.type, temp="private")
                acc = AOut(t.name, t.type, t)
                i = self.ivar("r")
                init = self.A(e.init, acc, levels)
                if not isinstance(e.type, (P.PairT, P.Arr)):
                    step = self.A(P.apply(e.f, P.Idx(x, i), tv), acc, levels + ["seq"])
                else:
                    # a pair (or an array) is written component by component: the
                    # step goes to a fresh one first, so that every component still
                    # reads the old accumulator, then replaces the accumulator
                    nt = self.temp(e.type, "private")
                    nv = P.Ident(nt.name, nt.type, temp="private")
                    step = New(nt, Seq([self.A(P.apply(e.f, P.Idx(x, i), tv), AOut(nt.name, nt.type, nt),
                                               levels + ["seq"]),
                                        self.assign(acc, nv, levels + ["seq"])]))
                return New(t, Seq([init, For(i, e.e.type.n, "seq", step), k(tv)]))

            return self.C(e.e, body, levels)
        if isinstance(e, (P.Map, P.To)):
            space = e.space if isinstance(e, P.To) else "global"
            inner = e.e if isinstance(e, P.To) else e
            if isinstance(inner, P.Map) and inner.level in ("global", "workgroup") and levels == []:
                # the consumer would read elements other blocks wrote: that needs a kernel boundary
                raise TranslationError("the result of a global or workgroup map is consumed in the same "
                                       "kernel; split the program into two kernels")
            t = self.temp(e.type, space)
            tv = P.Ident(t.name, t.type, temp=space)
            return New(t, Seq([self.A(inner, AOut(t.name, t.type, t), levels), k(tv)]))
        if isinstance(e, P.Bin):
            return self.C(e.a, lambda a: self.C(e.b, lambda b: k(P.Bin(e.op, a, b)), levels), levels)
        if isinstance(e, P.Abs):
            return self.C(e.a, lambda a: k(P.Abs(a)), levels)
        if isinstance(e, P.Splat):
            return self.C(e.a, lambda a: k(P.Splat(e.n, a)), levels)
        if isinstance(e, P.Fma):
            return self.C(e.a, lambda a: self.C(e.b, lambda b: self.C(e.c, lambda c: k(P.Fma(a, b, c)), levels),
                                                levels), levels)
        if isinstance(e, P.Zip):
            return self.C(e.a, lambda a: self.C(e.b, lambda b: k(P.Zip(a, b)), levels), levels)
        if isinstance(e, P.Proj):
            return self.C(e.e, lambda v: k(P.Proj(e.k, v)), levels)
        if isinstance(e, P.Pair):
            return self.C(e.a, lambda a: self.C(e.b, lambda b: k(P.Pair(a, b)), levels), levels)
        if isinstance(e, P.Split):
            return self.C(e.e, lambda v: k(P.Split(e.n, v)), levels)
        if isinstance(e, P.Join):
            return self.C(e.e, lambda v: k(P.Join(v)), levels)
        if isinstance(e, P.Transpose):
            return self.C(e.e, lambda v: k(P.Transpose(v)), levels)
        if isinstance(e, P.Idx):
            return self.C(e.e, lambda v: k(P.Idx(v, e.i)), levels)
        if isinstance(e, P.AsVector):
            return self.C(e.e, lambda v: k(P.AsVector(e.n, v)), levels)
        if isinstance(e, P.AsScalar):
            return self.C(e.e, lambda v: k(P.AsScalar(v)), levels)
        if isinstance(e, P.Lanes):
            return self.C(e.e, lambda v: k(P.Lanes(v)), levels)
        if isinstance(e, P.ReduceTree):
            return self.tree(e, k, levels)
        if isinstance(e, P.SecondLevel):
            raise TranslationError("the second level's value is the kernel's output, not an operand")
        raise TranslationError(f"cannot translate {type(e).__name__}")


def translate(e: P.Phrase, out_name: str = "out") -> tuple[Comm, AOut]:
    """The command writing the value of e to the output array ``out_name``."""
    out = AOut(out_name, e.type)
    return Translator().A(e, out, []), out


# ---------------------------------------------------------------------------
# hoisting (Section 6.4): temporaries in global memory move out of parallel
# loops, each iteration getting its own slice
# ---------------------------------------------------------------------------


def hoist(c: Comm, loops=()) -> list:
    """Record, for each global temporary, the parallel loops around it; return
    every temporary found (in order)."""
    found = []
    if isinstance(c, Seq):
        for x in c.cs:
            found += hoist(x, loops)
    elif isinstance(c, New):
        if c.temp.space == "global":
            c.temp.hoist = [(v, n) for (v, n, lvl) in loops if lvl != "seq"]
        found.append(c.temp)
        found += hoist(c.body, loops)
    elif isinstance(c, For):
        found += hoist(c.body, loops + ((c.var, c.n, c.level),))
    elif isinstance(c, TreeReduce):
        found += [c.buf, c.res]
        found += hoist(c.fill, loops)
    elif isinstance(c, LastBlock):
        found += hoist(c.body, ())
    return found
