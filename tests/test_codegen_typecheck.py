"""The type checker of translated phrases (no GPU): every program the
generator emits is well typed, and planted mistakes -- a type mismatch, a
parallel loop writing outside its own element acceptor, reading what it
writes, an illegal nesting -- are rejected. The write-race checker, which
works on the index arithmetic instead of the types, rejects the same races."""
import pytest

from paper_1710_08332_gb300.codegen import check as CK
from paper_1710_08332_gb300.codegen import phrase as P
from paper_1710_08332_gb300.codegen import programs as PR
from paper_1710_08332_gb300.codegen import rewrite as RW
from paper_1710_08332_gb300.codegen import translate as T
from paper_1710_08332_gb300.codegen import typecheck as TC

PROGRAMS = {
    "dot_partials": lambda: PR.dot_partials(1 << 12, 1 << 10, 64),
    "dot_partials_contig": lambda: PR.dot_partials(1 << 12, 1 << 10, 64, thread_map="contig"),
    "dot_partials_V4": lambda: PR.dot_partials(1 << 12, 1 << 10, 64, V=4),
    "asum_partials_V4": lambda: PR.asum_partials(1 << 12, 1 << 10, 64, V=4),
    "fold_all": lambda: PR.fold_all(256),
    "fold_rows": lambda: PR.fold_rows(64, 32),
    "fold_cols": lambda: PR.fold_cols(64, 32),
    "scal": lambda: PR.scal(1024, 1.5),
    "scal_V4": lambda: PR.scal(1024, 1.5, V=4),
    "gemv_partials": lambda: PR.gemv_partials(64, 256, 32),
    "gemv_partials_V4": lambda: PR.gemv_partials(64, 256, 16, V=4),
    "dot_K1": lambda: PR.dot_K1(512),
    "gemv_bwd_dA": lambda: PR.gemv_bwd_dA(64, 128),
    "gemv_bwd_dx_partials": lambda: PR.gemv_bwd_dx_partials(64, 128, 16),
    "gemv_bwd_dx_fold": lambda: PR.gemv_bwd_dx_fold(4, 128),
    "dot_partials_kahan": lambda: PR.dot_partials_kahan(1 << 12, 1 << 10, 64),
    "fold_pairs_rows": lambda: PR.fold_pairs_rows(16, 8),
    "fold_pairs_all": lambda: PR.fold_pairs_all(16),
    "dot_R": lambda: PR.dot_R(1 << 14, 1 << 11, 128, 4, "interleaved", "tree", 8),
    "dot_R_seq_contig": lambda: PR.dot_R(1 << 13, 1 << 10, 64, 1, "contig", "seq", 1),
    "asum_R": lambda: PR.asum_R(1 << 14, 1 << 11, 256, 4, "interleaved", "tree", 8),
    "gemv_R": lambda: PR.gemv_R(16, 512, 64, 4),
    "gemv_R_warp": lambda: PR.gemv_R_warp(16, 512, 4, 4),
    "dot_bwd": lambda: PR.dot_bwd(1024),
    "dot_bwd_V4": lambda: PR.dot_bwd(1024, 4),
    "gemm": lambda: PR.gemm(24, 40, 12),
    "gemm_V4": lambda: PR.gemm(24, 40, 12, 4),
    "gemm_tA_tB": lambda: PR.gemm(24, 40, 12, 1, True, True),
    "gemm_tA_V4": lambda: PR.gemm(24, 40, 12, 4, True, False),
    "dot_R_kahan": lambda: PR.dot_R_kahan(1 << 14, 1 << 11, 128, 4, "interleaved", "tree", 8),
    "asum_R_kahan_seq": lambda: PR.asum_R_kahan(1 << 13, 1 << 10, 64, 1, "contig", "seq", 1),
    "gemm_tiled": lambda: PR.gemm_tiled(16, 32, 12, 4, 8, 4),
    "gemm_tiled_KV4": lambda: PR.gemm_tiled(16, 32, 12, 4, 8, 4, 4),
    "gemm_tiled_tA_tB": lambda: PR.gemm_tiled(16, 32, 12, 4, 4, 1, 1, True, True),
}


@pytest.mark.parametrize("name", sorted(PROGRAMS))
def test_every_program_is_well_typed(name):
    e, _ = PROGRAMS[name]()
    c, out = T.translate(e)
    TC.typecheck(c, out)


def test_temporaries_and_explored_pipelines_are_well_typed():
    n = 1 << 14
    x = P.inp("x", P.arr(n, P.F32))
    for space, wrap in (("local", P.to_local), ("private", P.to_private), ("global", P.to_global)):
        e = P.join(P.mapWorkgroup(lambda ch: P.mapLocal(
            lambda col: P.reduceSeq(lambda v, a: P.add(a, v), 0.0, col),
            P.split(8, wrap(P.mapLocal(lambda v: P.mul(v, v), ch)))), P.split(1024, x)))
        c, out = T.translate(e)
        TC.typecheck(c, out)
    for d in RW.derivations(n, splits=(1 << 12,), threads=(64,), widths=(1, 4)):
        for _, ph, _ in RW.lower("dot", d, n):
            c, out = T.translate(ph)
            TC.typecheck(c, out)


F = P.F32


def _out(t, name="out"):
    return T.AOut(name, t)


def _lit():
    return P.Lit(1.0)


def test_assignment_of_the_wrong_type():
    with pytest.raises(TC.TypeCheckError, match="types differ"):
        TC.typecheck(T.Assign(_out(P.Arr(4, F)), _lit()))
    with pytest.raises(TC.TypeCheckError, match="types differ"):
        TC.typecheck(T.Assign(_out(F), P.Lit(1.0, P.I32)))


def test_views_have_their_types():
    o = _out(P.Arr(2, P.Arr(4, F)))
    assert TC.acc_type(T.ASplit(4, o)) == P.Arr(8, F)
    assert TC.acc_type(T.AJoin(4, _out(P.Arr(8, F)))) == P.Arr(2, P.Arr(4, F))
    assert TC.acc_type(T.ATranspose(o)) == P.Arr(4, P.Arr(2, F))
    assert TC.acc_type(T.AAsScalar(4, _out(P.Arr(8, F)))) == P.Arr(2, P.VecT(4, F))
    assert TC.acc_type(T.AProj(1, _out(P.PairT(F, P.I32)))) == P.I32
    with pytest.raises(TC.TypeCheckError, match="split acceptor"):
        TC.acc_type(T.ASplit(3, o))
    with pytest.raises(TC.TypeCheckError, match="join acceptor"):
        TC.acc_type(T.AJoin(3, _out(P.Arr(8, F))))
    with pytest.raises(TC.TypeCheckError, match="element acceptor"):
        TC.acc_type(T.AIdx(_out(F), T.IConst(0)))


def test_a_parallel_loop_writes_only_its_own_element():
    i, j = T.IVar("i1"), T.IVar("i2")
    # each iteration writes element i of out, through a split view: well typed
    ok = T.For(i, 8, "global", T.Assign(T.AIdx(T.ASplit(4, _out(P.Arr(2, P.Arr(4, F)))), i), _lit()))
    TC.typecheck(ok)
    CK.check(ok)
    # every iteration writes the same scalar
    shared = T.For(i, 8, "global", T.Assign(_out(F, "s"), _lit()))
    with pytest.raises(TC.TypeCheckError, match="outside its own element acceptor"):
        TC.typecheck(shared)
    with pytest.raises(CK.RaceError):
        CK.check(shared)
    # every iteration writes element j of a sequential loop inside it
    wrong = T.For(i, 8, "global", T.For(j, 4, "seq", T.Assign(T.AIdx(_out(P.Arr(4, F)), j), _lit())))
    with pytest.raises(TC.TypeCheckError, match="outside its own element acceptor"):
        TC.typecheck(wrong)
    with pytest.raises(CK.RaceError):
        CK.check(wrong)
    # a workgroup loop's local loop writes inside the workgroup's element: both own it
    nested = T.For(i, 4, "workgroup", T.For(j, 8, "local", T.Assign(
        T.AIdx(T.AIdx(_out(P.Arr(4, P.Arr(8, F))), i), j), _lit())))
    TC.typecheck(nested)
    # the local loop forgets its index: every thread of a workgroup writes one element
    lost = T.For(i, 4, "workgroup", T.For(j, 8, "local", T.Assign(T.AIdx(_out(P.Arr(4, F)), i), _lit())))
    with pytest.raises(TC.TypeCheckError, match="local loop over i2"):
        TC.typecheck(lost)
    with pytest.raises(CK.RaceError):
        CK.check(lost)


def test_iteration_temporaries_are_private_to_the_iteration():
    i, r = T.IVar("i1"), T.IVar("r2")
    t = T.Temp("t3", F, "private")
    acc = T.AOut(t.name, F, t)
    tv = P.Ident(t.name, F, temp="private")
    body = T.New(t, T.Seq([T.Assign(acc, _lit()),
                           T.For(r, 4, "seq", T.Assign(acc, P.Bin("+", tv, _lit()))),
                           T.Assign(T.AIdx(_out(P.Arr(8, F)), i), tv)]))
    TC.typecheck(T.For(i, 8, "global", body))
    # the same accumulator declared outside the parallel loop is shared by its iterations
    hoisted = T.New(t, T.For(i, 8, "global", T.Seq([
        T.Assign(acc, _lit()), T.Assign(T.AIdx(_out(P.Arr(8, F)), i), tv)])))
    with pytest.raises(TC.TypeCheckError):
        TC.typecheck(hoisted)


def test_a_parallel_loop_may_not_read_what_it_writes():
    i = T.IVar("i1")
    t = T.Temp("t2", P.Arr(8, F), "global")
    tv = P.Ident(t.name, t.type, temp="global")
    # iteration i writes t[i] and reads t[(i + 1) % 8]: the acceptor and the expression of t interfere
    c = T.New(t, T.For(i, 8, "global", T.Assign(T.AIdx(T.AOut(t.name, t.type, t), i),
                                                P.Idx(tv, T.IOp("%", T.IOp("+", i, T.IConst(1)), T.IConst(8))))))
    with pytest.raises(TC.TypeCheckError, match="interference"):
        TC.typecheck(c)
    CK.check(c)  # the write pattern alone is disjoint: only the types see the conflict
    # writing t in one parallel loop and reading it in the next is fine
    j = T.IVar("i3")
    ok = T.New(t, T.Seq([T.For(i, 8, "global", T.Assign(T.AIdx(T.AOut(t.name, t.type, t), i), _lit())),
                         T.For(j, 8, "global", T.Assign(T.AIdx(_out(P.Arr(8, F)), j), P.Idx(tv, j)))]))
    TC.typecheck(ok)


@pytest.mark.parametrize("outer,inner", [("local", "workgroup"), ("workgroup", "workgroup"),
                                         ("global", "local"), ("seq", "global"), ("seq", "local"),
                                         ("local", "local")])
def test_illegal_nestings(outer, inner):
    i, j = T.IVar("i1"), T.IVar("i2")
    out = _out(P.Arr(4, P.Arr(4, F)))
    c = T.For(i, 4, outer, T.For(j, 4, inner, T.Assign(T.AIdx(T.AIdx(out, i), j), _lit())))
    with pytest.raises(TC.TypeCheckError, match="strictly finer"):
        TC.typecheck(c)


@pytest.mark.parametrize("outer,inner", [("workgroup", "local"), ("workgroup", "seq"), ("local", "seq"),
                                         ("global", "seq"), ("seq", "seq")])
def test_legal_nestings(outer, inner):
    i, j = T.IVar("i1"), T.IVar("i2")
    out = _out(P.Arr(4, P.Arr(4, F)))
    TC.typecheck(T.For(i, 4, outer, T.For(j, 4, inner, T.Assign(T.AIdx(T.AIdx(out, i), j), _lit()))))


def _parallel_writes(c, par=(), out=None):
    """(assignment, element acceptor) pairs whose element index is the variable
    of an enclosing parallel loop."""
    out = [] if out is None else out
    if isinstance(c, T.Seq):
        for x in c.cs:
            _parallel_writes(x, par, out)
    elif isinstance(c, T.New):
        _parallel_writes(c.body, par, out)
    elif isinstance(c, T.TreeReduce):
        _parallel_writes(c.fill, par, out)
    elif isinstance(c, T.LastBlock):
        _parallel_writes(c.body, (), out)
    elif isinstance(c, T.For):
        _parallel_writes(c.body, par + ((c.var.name,) if c.level != "seq" else ()), out)
    elif isinstance(c, T.Assign):
        a = c.acc
        while not isinstance(a, T.AOut):
            if isinstance(a, T.AIdx) and isinstance(a.i, T.IVar) and a.i.name in par:
                out.append((c, a))
            a = a.acc
    return out


@pytest.mark.parametrize("name", sorted(PROGRAMS))
def test_every_planted_shared_write_is_rejected(name):
    """Mutation test: each element acceptor a parallel loop writes through,
    in turn indexed by a constant instead of the loop's variable (so that all
    iterations write one element), makes the program ill typed -- and racy
    for the index-arithmetic checker too."""
    e, _ = PROGRAMS[name]()
    c, out = T.translate(e)
    sites = _parallel_writes(c)
    assert sites or name in ("fold_all", "fold_pairs_all", "dot_K1")
    for _, a in sites:
        keep = a.i
        a.i = T.IConst(0)
        try:
            with pytest.raises(TC.TypeCheckError):
                TC.typecheck(c, out)
            with pytest.raises(CK.RaceError):
                CK.check(c)
        finally:
            a.i = keep
    TC.typecheck(c, out)
    CK.check(c)


def test_loop_longer_than_the_array_it_indexes_is_rejected():
    """A parfor over n hands its iterations the n elements of its acceptor: a
    loop of 64 iterations writing element i of a 4-element output (or reading
    element i of a 4-element input) is out of bounds, and both checkers say so."""
    i = T.IVar("i")
    out = T.AOut("out", P.arr(4, P.F32))
    bad = T.For(i, 64, "global", T.Assign(T.AIdx(out, i), P.lit(1.0)))
    with pytest.raises(TC.TypeCheckError, match="past the 4 elements"):
        TC.typecheck(bad, out)
    with pytest.raises(CK.RaceError, match="outside"):
        CK.check(bad)
    with pytest.raises(TC.TypeCheckError, match="past the 4 elements"):
        TC.typecheck(T.For(i, 8, "seq", T.Assign(T.AIdx(out, T.IConst(5)), P.lit(1.0))), out)
    x = P.inp("x", P.arr(4, P.F32))
    big = T.AOut("out", P.arr(64, P.F32))
    with pytest.raises(TC.TypeCheckError, match="read of an element"):
        TC.typecheck(T.For(i, 64, "global", T.Assign(T.AIdx(big, i), P.Idx(x, i))), big)
    # the same loops within bounds pass
    ok = T.For(i, 4, "global", T.Assign(T.AIdx(out, i), P.Idx(x, i)))
    TC.typecheck(ok, out)
    CK.check(ok)


def test_write_to_something_other_than_the_output_is_rejected():
    i = T.IVar("i")
    out = T.AOut("out", P.arr(4, P.F32))
    stray = T.AOut("stray", P.arr(4, P.F32))
    c = T.For(i, 4, "global", T.Assign(T.AIdx(stray, i), P.lit(1.0)))
    with pytest.raises(TC.TypeCheckError, match="neither its output"):
        TC.typecheck(c, out)
    TC.typecheck(c, stray)
