"""Race freedom of a loop nest, checked before code is emitted.

The paper obtains race freedom from its type system: a parallel for hands
each iteration its own acceptor, and no other active phrase may be used in
the body (SCIR's interference control). This module checks the property on
the imperative program itself, so that it also holds for loop nests built by
hand: for every parallel loop L and every assignment inside it whose target
is shared by L's iterations (an output, a global or local temporary declared
outside L, or a private variable declared outside L), the written offset, as
a function of L's variable and the variables of the loops between L and the
assignment, must be injective -- two different iterations of L can then never
write the same place. Offsets are linear forms in the loop variables
(quotient and remainder by the same divisor are recombined first); a form is
injective on its box when its coefficients, in increasing order, each exceed
the largest value the smaller terms can add up to (a mixed-radix numbering).
Every write, parallel or not, must also stay inside its place: the largest
offset over all loop variables is below the number of elements written into.
"""
from __future__ import annotations

from . import phrase as P
from . import translate as T


class RaceError(Exception):
    pass


def _dims(t):
    d = []
    while isinstance(t, P.Arr):
        d.append(t.n)
        t = t.elem
    return d


def _linear(idx, shape):
    off = T.IConst(0)
    for i, n in zip(idx, shape):
        off = T.iadd(T.imul(off, n), i)
    return off


def target(acc, path):
    """(place name, temp or None, offset index expression) written through acc."""
    proj = None
    while True:
        if isinstance(acc, T.AProj):
            proj = acc.k
        elif isinstance(acc, T.AIdx):
            path = [acc.i] + path
        elif isinstance(acc, T.ASplit):
            path = [T.idiv(path[0], acc.n), T.imod(path[0], acc.n)] + path[1:]
        elif isinstance(acc, T.AJoin):
            path = [T.iadd(T.imul(path[0], acc.m), path[1])] + path[2:]
        elif isinstance(acc, T.ATranspose):
            path = [path[1], path[0]] + path[2:]
        elif isinstance(acc, T.AAsScalar):
            path = [T.imul(path[0], acc.V)] + path[1:]
        elif isinstance(acc, T.AOut):
            t = acc.temp
            shape = _dims(acc.type)
            off = _linear(path, shape) if shape else T.IConst(0)
            if proj is not None and t is None:  # arrays of pairs: two numbers per element
                off = T.iadd(T.imul(off, 2), T.IConst(proj))
            if t is not None and t.space == "global" and t.hoist:
                h = _linear([v for v, _ in t.hoist], [n for _, n in t.hoist])
                off = T.iadd(T.imul(h, P.scalar_count(t.type)), off)
            return acc.name, t, off
        else:
            raise RaceError(f"unknown acceptor {type(acc).__name__}")
        acc = acc.acc


def linear_form(e):
    """{variable name: coefficient} and a constant, or None if e is not linear."""
    terms = []

    def flat(x, k):
        if isinstance(x, T.IOp) and x.op == "+":
            flat(x.a, k)
            flat(x.b, k)
        elif isinstance(x, T.IOp) and x.op == "*" and isinstance(x.b, T.IConst):
            flat_mul(x.a, k * x.b.v)
        else:
            terms.append((x, k))

    def flat_mul(x, k):
        if isinstance(x, T.IOp) and x.op == "+":
            flat(x.a, k)
            flat(x.b, k)
        elif isinstance(x, T.IOp) and x.op == "*" and isinstance(x.b, T.IConst):
            flat_mul(x.a, k * x.b.v)
        else:
            terms.append((x, k))

    flat(e, 1)
    # recombine (q / n) * n + q % n into q
    changed = True
    while changed:
        changed = False
        for a in range(len(terms)):
            xa, ka = terms[a]
            if isinstance(xa, T.IOp) and xa.op == "/" and isinstance(xa.b, T.IConst) and ka % xa.b.v == 0:
                n = xa.b.v
                for b in range(len(terms)):
                    xb, kb = terms[b]
                    if (b != a and isinstance(xb, T.IOp) and xb.op == "%" and xb.b == xa.b and xb.a == xa.a
                            and kb * n == ka):
                        q = xa.a
                        rest = [t for i, t in enumerate(terms) if i not in (a, b)]
                        terms[:] = rest
                        terms.append((q, kb))
                        changed = True
                        break
            if changed:
                break
        if changed:  # q may itself be a sum: flatten it again
            x, k = terms.pop()
            if isinstance(x, (T.IVar, T.IConst)):
                terms.append((x, k))
            else:
                flat(x, k)
    form, const = {}, 0
    for x, k in terms:
        if isinstance(x, T.IConst):
            const += x.v * k
        elif isinstance(x, T.IVar):
            form[x.name] = form.get(x.name, 0) + k
        else:
            return None
    return {v: c for v, c in form.items() if c != 0}, const


def injective(form: dict, ranges: dict) -> bool:
    """The linear form (variables with trip counts in ranges) takes distinct
    values on distinct points of the box."""
    terms = sorted(((abs(c), ranges[v]) for v, c in form.items() if ranges.get(v, 1) > 1), key=lambda t: t[0])
    span = 0
    for c, n in terms:
        if c <= span:
            return False
        span += c * (n - 1)
    return True


def place_size(acc) -> int:
    """Numbers in the place an acceptor writes into (an output, or a temporary
    with one slice per iteration of the parallel loops it is hoisted out of)."""
    while not isinstance(acc, T.AOut):
        acc = acc.acc
    if not isinstance(acc.type, (P.Arr, P.PairT)) and not P.is_scalar(acc.type):
        raise RaceError(f"cannot size {acc.name} of type {acc.type}")
    if isinstance(acc.type, P.PairT):  # a private pair (of numbers or vectors): one place per component
        return 2
    n = P.scalar_count(acc.type) if not isinstance(acc.type, P.VecT) else 1
    if isinstance(P.base_elem(acc.type), P.VecT):
        n = max(1, n // P.base_elem(acc.type).n)  # vector outputs are addressed by vector
    if acc.temp is not None and acc.temp.space == "global":
        for _, k in acc.temp.hoist:
            n *= k
    return n


def check(comm) -> None:
    """Raise RaceError if two iterations of a parallel loop may write one place,
    or if a write may fall outside the place it writes into."""
    _walk(comm, [], {})


def _walk(c, loops, declared):
    if isinstance(c, T.Seq):
        for x in c.cs:
            _walk(x, loops, declared)
    elif isinstance(c, T.New):
        d = dict(declared)
        d[c.temp.name] = len(loops)  # declared inside the first len(loops) loops
        _walk(c.body, loops, d)
    elif isinstance(c, T.For):
        _walk(c.body, loops + [c], declared)
    elif isinstance(c, T.TreeReduce):
        # the buffer and the result are the enclosing iteration's own; the fill's
        # lane loop writes element l of the buffer (the halving steps then write
        # buf[l] for l < h from buf[l + h], never a place another step reads)
        d = dict(declared)
        d[c.buf.name] = d[c.res.name] = len(loops)
        _walk(c.fill, loops, d)
    elif isinstance(c, T.LastBlock):
        _walk(c.body, [], declared)  # one block, after every block's loop
    elif isinstance(c, T.Assign):
        from .typecheck import index_max

        name, temp, off = target(c.acc, [])
        top = index_max(off, {L.var.name: L.n for L in loops})
        size = place_size(c.acc)
        if top is None or top >= size:
            raise RaceError(f"a write to {name} may fall outside its {size} elements "
                            f"(offset {'unbounded' if top is None else f'up to {top}'})")
        for k, L in enumerate(loops):
            if L.level == "seq":
                continue
            if temp is not None and declared.get(name, -1) > k:
                continue  # declared inside L: each iteration has its own
            inner = loops[k:]
            form = linear_form(off)
            if form is None:
                raise RaceError(f"cannot prove that iterations of the {L.level} loop {L.var.name} write "
                                f"distinct places of {name}: offset is not linear")
            coeffs, _ = form
            if coeffs.get(L.var.name, 0) == 0 or not injective(
                    {v: cf for v, cf in coeffs.items() if v in {l.var.name for l in inner}},
                    {l.var.name: l.n for l in inner}):
                raise RaceError(f"iterations of the {L.level} loop {L.var.name} may write the same place "
                                f"of {name}")
