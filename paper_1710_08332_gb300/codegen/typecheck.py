"""A type checker for the translated imperative phrases (the paper's DPIA
type system, Section 3, applied to the commands Stages I and II produce).

Phrase types: an expression has type exp[d] (passive: it only reads), an
acceptor acc[d] and a command comm (active: they write). The checker derives
the data type d of every acceptor from its construction -- the kernel output
or a temporary, an element (AIdx), and the re-indexing views of split, join,
transpose, pair projection and asScalar -- and requires every assignment to
write an expression of exactly that type.

Parallel loops follow the discipline of the paper's parfor: the body of a
parallel loop over i receives the i-th element acceptor of its output and may
write only through it (or through temporaries it declares itself); every
other identifier it uses must be passive, i.e. only read. Because every view
re-indexes injectively, the i-th elements of an acceptor are disjoint for
distinct i, so a program that checks is race-free by construction. Every
index, written or read, is bounded by the length of the array it indexes
(a loop's trip count may not exceed it). Further:
the body may not read a temporary that the same parallel loop writes (the
acceptor of a variable and its expression would interfere), and parallel
loops nest at strictly finer levels (workgroup > local; workgroup > warp >
lane; global, local and lane hold only sequential loops; nothing parallel
inside a sequential loop). A lane tree's fill is a lane loop writing its own
element of the tree's buffer, and its function combines two elements into
one; the last block's second level is checked as the body of one work-group.
"""
from __future__ import annotations

from . import phrase as P
from . import translate as T

PARALLEL = ("global", "workgroup", "warp", "lane", "local")


class TypeCheckError(Exception):
    pass


# ---------------------------------------------------------------------------
# data types of acceptors
# ---------------------------------------------------------------------------


def acc_type(a: T.Acc):
    """The data type d of an acceptor of type acc[d]."""
    if isinstance(a, T.AOut):
        return a.type
    if isinstance(a, T.AIdx):
        t = acc_type(a.acc)
        if not isinstance(t, P.Arr):
            raise TypeCheckError(f"element acceptor of a non-array acceptor acc[{t}]")
        return t.elem
    if isinstance(a, T.ASplit):  # out: acc[m.n.d]  ->  acc[(m n).d]
        t = acc_type(a.acc)
        if not (isinstance(t, P.Arr) and isinstance(t.elem, P.Arr) and t.elem.n == a.n):
            raise TypeCheckError(f"split acceptor of width {a.n} over acc[{t}]")
        return P.Arr(t.n * a.n, t.elem.elem)
    if isinstance(a, T.AJoin):  # out: acc[(k m).d]  ->  acc[k.m.d]
        t = acc_type(a.acc)
        if not isinstance(t, P.Arr) or a.m <= 0 or t.n % a.m:
            raise TypeCheckError(f"join acceptor of inner length {a.m} over acc[{t}]")
        return P.Arr(t.n // a.m, P.Arr(a.m, t.elem))
    if isinstance(a, T.ATranspose):  # out: acc[b.a.d]  ->  acc[a.b.d]
        t = acc_type(a.acc)
        if not (isinstance(t, P.Arr) and isinstance(t.elem, P.Arr)):
            raise TypeCheckError(f"transpose acceptor over acc[{t}]")
        return P.Arr(t.elem.n, P.Arr(t.n, t.elem.elem))
    if isinstance(a, T.AProj):
        t = acc_type(a.acc)
        if not isinstance(t, P.PairT):
            raise TypeCheckError(f"projection acceptor over acc[{t}]")
        return t.a if a.k == 0 else t.b
    if isinstance(a, T.AAsScalar):  # out: acc[(n V).num]  ->  acc[n.num<V>]
        t = acc_type(a.acc)
        if not (isinstance(t, P.Arr) and isinstance(t.elem, P.Num) and t.n % a.V == 0):
            raise TypeCheckError(f"asScalar acceptor of width {a.V} over acc[{t}]")
        return P.Arr(t.n // a.V, P.VecT(a.V, t.elem))
    raise TypeCheckError(f"unknown acceptor {type(a).__name__}")


def index_max(i, trips: dict):
    """The largest value the index expression takes while every loop variable v
    runs over 0..trips[v]-1, or None if it cannot be bounded (an unknown
    variable, a negative constant or an unsupported operation)."""
    if isinstance(i, T.IConst):
        return i.v if i.v >= 0 else None
    if isinstance(i, T.IVar):
        n = trips.get(i.name)
        return None if n is None else max(n - 1, 0)
    if isinstance(i, T.IOp):
        a = index_max(i.a, trips)
        if i.op == "%" and isinstance(i.b, T.IConst) and i.b.v > 0:
            return min(a, i.b.v - 1) if a is not None else i.b.v - 1
        b = index_max(i.b, trips)
        if a is None or b is None:
            return None
        if i.op == "+":
            return a + b
        if i.op == "*":
            return a * b
        if i.op == "/" and isinstance(i.b, T.IConst) and i.b.v > 0:
            return a // i.b.v
    return None


def _check_bound(i, n: int, trips: dict, what: str):
    m = index_max(i, trips)
    if m is None:
        raise TypeCheckError(f"{what}: cannot bound the index by the loops around it")
    if m >= n:
        raise TypeCheckError(f"{what}: the index reaches {m}, past the {n} elements of the array "
                             f"(a loop runs longer than the array it indexes)")


def _acc_bounds(a: T.Acc, trips: dict):
    """Every element acceptor on the way to the root indexes within its array."""
    while not isinstance(a, T.AOut):
        if isinstance(a, T.AIdx):
            t = acc_type(a.acc)
            _check_bound(a.i, t.n, trips, f"write through element acceptor of acc[{t}]")
        a = a.acc


def _exp_bounds(e: P.Phrase, trips: dict):
    """Every element read (Idx) indexes within its array."""
    if isinstance(e, P.Idx):
        _check_bound(e.i, e.e.type.n, trips, f"read of an element of exp[{e.e.type}]")
    for child in e.children():
        _exp_bounds(child, trips)


def _root(a: T.Acc) -> T.AOut:
    while not isinstance(a, T.AOut):
        a = a.acc
    return a


def _owned_by(a: T.Acc, var: T.IVar) -> bool:
    """The acceptor lies inside the var-th element of an acceptor: somewhere
    on its way to the root it takes element ``var`` (exactly the loop index)."""
    while not isinstance(a, T.AOut):
        if isinstance(a, T.AIdx) and isinstance(a.i, T.IVar) and a.i.name == var.name:
            return True
        a = a.acc
    return False


# ---------------------------------------------------------------------------
# reads
# ---------------------------------------------------------------------------


def _temps_read(e: P.Phrase, out: set):
    """Names of temporaries an expression reads."""
    if isinstance(e, P.Ident):
        if e.temp:
            out.add(e.name)
        return
    if isinstance(e, (P.Map, P.Reduce)):
        raise TypeCheckError(f"a {type(e).__name__.lower()} left in a translated command")
    for child in e.children():
        _temps_read(child, out)


def _reads(c: T.Comm, out: set):
    if isinstance(c, T.Seq):
        for x in c.cs:
            _reads(x, out)
    elif isinstance(c, T.New):
        _reads(c.body, out)
    elif isinstance(c, T.For):
        _reads(c.body, out)
    elif isinstance(c, T.Assign):
        _temps_read(c.e, out)
    elif isinstance(c, T.TreeReduce):
        _reads(c.fill, out)
    elif isinstance(c, T.LastBlock):
        _reads(c.body, out)


# ---------------------------------------------------------------------------
# commands
# ---------------------------------------------------------------------------


class _Frame:
    """A parallel loop being checked: its index and the temporaries declared
    inside its body (each iteration's own)."""

    def __init__(self, var: T.IVar, level: str):
        self.var, self.level = var, level
        self.local = set()
        self.written = set()  # temporaries declared outside and written inside


def _check(c: T.Comm, frames: list, levels: list, trips: dict, out: T.AOut | None):
    if isinstance(c, T.Seq):
        for x in c.cs:
            _check(x, frames, levels, trips, out)
    elif isinstance(c, T.New):
        if c.temp.space not in P.SPACES:
            raise TypeCheckError(f"temporary {c.temp.name} in unknown address space {c.temp.space}")
        for f in frames:  # declared inside every enclosing parallel loop: each iteration's own
            f.local.add(c.temp.name)
        _check(c.body, frames, levels, trips, out)
    elif isinstance(c, T.For):
        if not isinstance(c.n, int) or c.n < 0:
            raise TypeCheckError(f"loop over {c.var.name} with trip count {c.n!r}")
        if c.level not in P.LEVELS:
            raise TypeCheckError(f"loop over {c.var.name} at unknown level {c.level}")
        if c.level in PARALLEL and levels:
            last = levels[-1]
            if c.level not in T.FINER.get(last, ()):
                raise TypeCheckError(f"a {c.level} loop inside a {last} loop (parallel loops nest at "
                                     f"strictly finer levels, never inside a sequential loop)")
        if c.level in ("warp", "lane") and (not levels or levels[-1] != {"warp": "workgroup",
                                                                         "lane": "warp"}[c.level]):
            raise TypeCheckError(f"a {c.level} loop outside a {'workgroup' if c.level == 'warp' else 'warp'} loop")
        inner = {**trips, c.var.name: c.n}
        if c.level in PARALLEL:
            f = _Frame(c.var, c.level)
            _check(c.body, frames + [f], levels + [c.level], inner, out)
            read = set()
            _reads(c.body, read)
            clash = sorted(read & f.written)
            if clash:
                raise TypeCheckError(f"the {c.level} loop over {c.var.name} reads temporar"
                                     f"{'ies' if len(clash) > 1 else 'y'} {', '.join(clash)} that its "
                                     f"iterations write (interference)")
        else:
            _check(c.body, frames, levels + [c.level], inner, out)
    elif isinstance(c, T.Assign):
        if not isinstance(c.e, P.Phrase):
            raise TypeCheckError("assignment of something that is not an expression")
        d = acc_type(c.acc)
        if d != c.e.type:
            raise TypeCheckError(f"acc[{d}] := exp[{c.e.type}]: the types differ")
        _acc_bounds(c.acc, trips)
        _exp_bounds(c.e, trips)
        root = _root(c.acc)
        if out is not None and root.temp is None and root.name != out.name:
            raise TypeCheckError(f"the command writes {root.name}, which is neither its output {out.name} "
                                 f"nor a temporary")
        for f in frames:  # every enclosing parallel loop must own the write
            if root.name in f.local or _owned_by(c.acc, f.var):
                continue
            raise TypeCheckError(f"the {f.level} loop over {f.var.name} writes {root.name} outside its "
                                 f"own element acceptor (its body must be passive but for that acceptor)")
        for f in frames:  # temporaries declared outside a loop and written inside it
            if root.temp is not None and root.name not in f.local:
                f.written.add(root.name)
    elif isinstance(c, T.TreeReduce):
        t = c.buf.type
        if not (isinstance(t, P.Arr) and t.n & (t.n - 1) == 0 and t.n <= P.WARP and c.res.type == t.elem):
            raise TypeCheckError(f"lane tree over acc[{t}] into {c.res.type}")
        ps = c.f.params
        if len(ps) != 2 or any(p.type != t.elem for p in ps) or c.f.body.type != t.elem:
            raise TypeCheckError("a lane tree's function combines two elements into one")
        if not levels or levels[-1] != "warp":
            raise TypeCheckError("a lane tree runs directly inside a warp loop")
        for f in frames:  # the buffer and the result belong to this iteration
            f.local.update((c.buf.name, c.res.name))
        _check(c.fill, frames, levels, trips, out)
    elif isinstance(c, T.LastBlock):
        if frames or levels:
            raise TypeCheckError("the last block's second level runs outside every loop")
        _check(c.body, [], ["workgroup"], trips, out)
    else:
        raise TypeCheckError(f"unknown command {type(c).__name__}")


def typecheck(c: T.Comm, out: T.AOut | None = None) -> None:
    """Raise TypeCheckError unless the command is well typed: every assignment
    writes an expression of its acceptor's data type, every parallel loop
    writes only through its own element acceptor or its own temporaries and
    reads none of the temporaries it writes, loops nest legally, and every
    element index, written or read, stays below the length of the array it
    indexes for all values of the loop variables around it (the paper's parfor
    over n hands each of its n iterations one of the n elements). ``out`` is
    the kernel's output acceptor: every write that is not to a temporary must
    go to it."""
    if out is not None and not isinstance(out, T.AOut):
        raise TypeCheckError("the output must be an output acceptor")
    _check(c, [], [], {}, out)
