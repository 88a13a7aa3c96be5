"""The strategy-preserving code generator, checked on the host.

Each program is a phrase over the paper's primitives; the generator's C
backend compiles the loop nest it derives, and the result must be
bit-identical to the oracle's evaluation of the same phrase written with the
oracle's own primitives (c1). The CUDA source of every program must compile
for sm_103a. Illegal level nestings and a kernel reading what other blocks
of the same kernel wrote are rejected.
"""
import shutil
import subprocess

import numpy as np
import pytest

from oracle import patterns as c1
from paper_1710_08332_gb300 import codegen as G
from paper_1710_08332_gb300.codegen import build as B
from paper_1710_08332_gb300.codegen import emit as E
from paper_1710_08332_gb300.codegen import programs as PR
from paper_1710_08332_gb300.codegen import translate as T

F = c1.F32


def bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


def uniform(n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, n).astype(np.float32)


def cols(chunk, Tn, thread_map):
    return c1.transpose(c1.split(Tn, chunk)) if thread_map == "interleaved" else c1.split(len(chunk) // Tn, chunk)


def oracle_dot_partials(x, y, s, Tn, thread_map):
    return c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: F.add(a, F.mul(p[0], p[1])), F.zero, col),
                               cols(ch, Tn, thread_map)),
        c1.split(s, c1.zip_(list(x), list(y)))))


def oracle_fold(p):
    return c1.reduce_(lambda v, a: F.add(a, v), F.zero, list(p))


@pytest.mark.parametrize("thread_map", ["interleaved", "contig"])
@pytest.mark.parametrize("n,s,Tn", [(4096, 512, 32), (6144, 2048, 64), (256, 256, 1)])
def test_dot_two_kernels_match_oracle(c_build, n, s, Tn, thread_map):
    x, y = uniform(n, 1), uniform(n, 2)
    e, ins = PR.dot_partials(n, s, Tn, thread_map)
    part = np.zeros(n // s * Tn, np.float32)
    G.compile_c("dotp", e, ins).run(x, y, part)
    want = oracle_dot_partials(x, y, s, Tn, thread_map)
    assert np.array_equal(bits(part), bits(want))
    e2, ins2 = PR.fold_all(part.size)
    out = np.zeros(1, np.float32)
    G.compile_c("fold", e2, ins2).run(part, out)
    assert bits(out)[0] == bits([oracle_fold(want)])[0]


def test_dot_K1_is_the_sequential_loop(c_build):
    x, y = uniform(1000, 3), uniform(1000, 4)
    e, ins = PR.dot_K1(1000)
    out = np.zeros(1, np.float32)
    G.compile_c("k1", e, ins).run(x, y, out)
    acc = np.float32(0)
    for a, b in zip(x, y):
        acc = np.float32(acc + np.float32(a * b))
    assert bits(out)[0] == bits([acc])[0]


def test_asum_scal_gemv_match_oracle(c_build):
    n, s, Tn = 8192, 1024, 64
    x = uniform(n, 5)
    x[::7] = -x[::7]
    e, ins = PR.asum_partials(n, s, Tn, "contig")
    part = np.zeros(n // s * Tn, np.float32)
    G.compile_c("asump", e, ins).run(x, part)
    want = c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda v, a: F.add(a, F.abs(v)), F.zero, col),
                               cols(ch, Tn, "contig")), c1.split(s, list(x))))
    assert np.array_equal(bits(part), bits(want))

    e, ins = PR.scal(n, 1.5)
    out = np.zeros(n, np.float32)
    G.compile_c("scal", e, ins).run(x, out)
    assert np.array_equal(bits(out), bits([F.mul(F.lit(1.5), v) for v in x]))

    M, N, Tn = 37, 512, 32
    A = uniform(M * N, 6)
    xv = uniform(N, 7)
    e, ins = PR.gemv_partials(M, N, Tn)
    part = np.zeros(M * Tn, np.float32)
    G.compile_c("gemvp", e, ins).run(A, xv, part)
    rows = c1.split(N, list(A))
    want = c1.join(c1.mapWorkgroup(
        lambda row: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: F.add(a, F.mul(p[0], p[1])), F.zero, col),
                                cols(c1.zip_(row, list(xv)), Tn, "interleaved")), rows))
    assert np.array_equal(bits(part), bits(want))
    e, ins = PR.fold_rows(M, Tn)
    y = np.zeros(M, np.float32)
    G.compile_c("rows", e, ins).run(part, y)
    assert np.array_equal(bits(y), bits([oracle_fold(r) for r in c1.split(Tn, want)]))


@pytest.mark.parametrize("space", ["global", "private", "local"])
def test_temporaries_in_each_address_space(c_build, space):
    """A map's output consumed inside a workgroup loop becomes a temporary in
    the annotated space; a global one is hoisted out of the parallel loop with
    one slice per iteration (Section 6.4)."""
    n, s = 2048, 256
    x, y = uniform(n, 8), uniform(n, 9)
    X, Y = G.inp("x", G.arr(n, G.F32)), G.inp("y", G.arr(n, G.F32))
    wrap = {"global": lambda e: e, "private": G.to_private, "local": G.to_local}[space]
    e = G.mapWorkgroup(
        lambda ch: G.reduceSeq(lambda v, a: G.add(a, v), 0.0,
                               wrap(G.mapSeq(lambda p: G.mul(G.fst(p), G.snd(p)), ch))),
        G.split(s, G.zip_(X, Y)))
    f = G.compile_c("tmp_" + space, e, [X, Y])
    temps = f.temps_like()
    assert len(temps) == (1 if space == "global" else 0)
    if space == "global":
        assert temps[0].size == n  # 8 workgroups x 256
    out = np.zeros(n // s, np.float32)
    f.run(x, y, out, *temps)
    want = c1.map_(lambda ch: oracle_fold(c1.map_(lambda p: F.mul(p[0], p[1]), ch)),
                   c1.split(s, c1.zip_(list(x), list(y))))
    assert np.array_equal(bits(out), bits(want))


@pytest.fixture(params=["serial", "openmp"])
def c_build(request, monkeypatch):
    """Run a test's host builds serially and again with the outermost parallel
    loop on OpenMP threads (the paper's multicore target): both must equal the
    oracle."""
    if request.param == "openmp":
        orig = G.compile_c
        monkeypatch.setattr(G, "compile_c", lambda *a, **k: orig(*a, **{**k, "openmp": True}))
    return request.param


def test_openmp_marks_only_parallel_loops():
    """Only the outermost work-group or global loop runs on OpenMP threads: a
    program whose top loop is a sequential fold (or the second level after the
    work-group loop) keeps it on one thread."""
    e, ins = PR.dot_partials(1 << 12, 512, 32)
    assert G.compile_c("dotp", e, ins, openmp=True).source.count("#pragma omp parallel for") == 1
    e, ins = PR.fold_all(256)
    assert "#pragma omp" not in G.compile_c("fold", e, ins, openmp=True).source
    e, ins = PR.dot_R(1 << 12, 512, 32, 4, "interleaved", "tree", 8)
    src = G.compile_c("dR", e, ins, openmp=True).source
    assert src.count("#pragma omp parallel for") == 1
    assert src.index("#pragma omp") < src.index("for (long long i")


def test_loop_nest_levels_follow_the_strategy():
    e, ins = PR.dot_partials(4096, 512, 32)
    comm, _ = T.translate(e)
    levels = []

    def walk(c):
        if isinstance(c, T.For):
            levels.append((c.level, c.n))
            walk(c.body)
        elif isinstance(c, T.Seq):
            for x in c.cs:
                walk(x)
        elif isinstance(c, T.New):
            assert c.temp.space == "private"  # reduceI's accumulator
            walk(c.body)

    walk(comm)
    assert levels == [("workgroup", 8), ("local", 32), ("seq", 16)]


def test_illegal_nestings_are_rejected():
    x = G.inp("x", G.arr(1024, G.F32))
    inner = lambda ch: G.mapWorkgroup(lambda v: G.mul(v, v), ch)
    with pytest.raises(T.TranslationError, match="illegal nesting"):
        T.translate(G.mapLocal(inner, G.split(32, x)))
    with pytest.raises(T.TranslationError, match="illegal nesting"):
        T.translate(G.mapGlobal(lambda ch: G.mapGlobal(lambda v: v, ch), G.split(32, x)))
    with pytest.raises(T.TranslationError, match="illegal nesting"):
        T.translate(G.mapWorkgroup(lambda ch: G.mapWorkgroup(lambda v: v, ch), G.split(32, x)))


def test_cross_block_consumption_needs_a_kernel_boundary():
    x = G.inp("x", G.arr(1024, G.F32))
    e = G.reduceSeq(lambda v, a: G.add(a, v), 0.0,
                    G.join(G.mapWorkgroup(lambda ch: G.mapLocal(lambda v: G.mul(v, v), ch), G.split(32, x))))
    with pytest.raises(T.TranslationError, match="kernel"):
        T.translate(e)


def test_type_errors():
    x = G.inp("x", G.arr(1000, G.F32))
    with pytest.raises(TypeError):
        G.split(3, x)
    with pytest.raises(TypeError):
        G.zip_(x, G.inp("y", G.arr(999, G.F32)))
    with pytest.raises(TypeError):
        G.join(x)


@pytest.mark.skipif(not shutil.which("nvcc"), reason="nvcc not installed")
def test_cuda_sources_compile_for_sm103a(tmp_path):
    progs = {"dotp": PR.dot_partials(1 << 20, 8192, 256), "asump": PR.asum_partials(1 << 20, 8192, 256, "contig"),
             "fold": PR.fold_all(4096), "scal": PR.scal(1 << 20, 1.5), "gemvp": PR.gemv_partials(512, 1024, 128),
             "rows": PR.fold_rows(512, 128), "k1": PR.dot_K1(4096), "gemm4": PR.gemm(256, 512, 128, 4),
             "gemm_tt": PR.gemm(256, 512, 128, 1, True, True), "dotbwd4": PR.dot_bwd(1 << 20, 4)}
    for name, (e, ins) in progs.items():
        src = B.cuda_source(E.generate(name, e, ins, "cuda"))
        assert "__fadd_rn" in src or "__fmul_rn" in src
        path = tmp_path / f"{name}.cu"
        path.write_text(src)
        r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-c",
                            str(path), "-o", str(tmp_path / f"{name}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def vadd(a, b):
    return tuple(F.add(p, q) for p, q in zip(a, b))


def vmul(a, b):
    return tuple(F.mul(p, q) for p, q in zip(a, b))


def oracle_dot_partials_vec(x, y, s, Tn, thread_map, V=4):
    zero = tuple(F.zero for _ in range(V))
    return c1.asScalar(c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: vadd(a, vmul(p[0], p[1])), zero, col),
                               cols(ch, Tn, thread_map)),
        c1.split(s // V, c1.zip_(c1.asVector(V, list(x)), c1.asVector(V, list(y)))))))


@pytest.mark.parametrize("thread_map", ["interleaved", "contig"])
def test_vector_dot_scal_gemv_match_oracle(c_build, thread_map):
    """asVector 4 streams, lane-wise folds, un-reduced lane partials (Section 6's float4 kernel)."""
    n, s, Tn = 8192, 2048, 64
    x, y = uniform(n, 12), uniform(n, 13)
    e, ins = PR.dot_partials(n, s, Tn, thread_map, V=4)
    part = np.zeros(n // s * Tn * 4, np.float32)
    G.compile_c("dotv", e, ins).run(x, y, part)
    assert np.array_equal(bits(part), bits(oracle_dot_partials_vec(x, y, s, Tn, thread_map)))

    e, ins = PR.scal(n, 1.5, V=4)
    out = np.zeros(n, np.float32)
    G.compile_c("scalv", e, ins).run(x, out)
    want = c1.asScalar(c1.map_(lambda v: vmul((F.lit(1.5),) * 4, v), c1.asVector(4, list(x))))
    assert np.array_equal(bits(out), bits(want))

    M, N, Tn = 24, 1024, 64
    A, xv = uniform(M * N, 14), uniform(N, 15)
    e, ins = PR.gemv_partials(M, N, Tn, thread_map, V=4)
    part = np.zeros(M * Tn * 4, np.float32)
    G.compile_c("gemvv", e, ins).run(A, xv, part)
    zero = (F.zero,) * 4
    want = c1.asScalar(c1.join(c1.mapWorkgroup(
        lambda row: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: vadd(a, vmul(p[0], p[1])), zero, col),
                                cols(c1.zip_(c1.asVector(4, row), c1.asVector(4, list(xv))), Tn, thread_map)),
        c1.split(N, list(A)))))
    assert np.array_equal(bits(part), bits(want))


def test_vector_views_must_keep_lanes_adjacent():
    """asVector reads V adjacent numbers at an offset that is a multiple of V:
    rows of an array qualify, columns (a transposed view) do not."""
    A = G.inp("A", G.arr(8, 6, G.F32))  # rows of 6: row i starts at 6i
    e = G.mapGlobal(lambda row: G.reduceSeq(lambda v, a: G.add(a, v), G.vlit(0.0, 2), G.asVector(2, row)), A)
    src = E.generate("ok2", e, [A], "cuda")["source"]
    assert "float2" in src
    B = G.inp("B", G.arr(8, 8, G.F32))
    e = G.mapGlobal(lambda col: G.reduceSeq(lambda v, a: G.add(a, v), G.vlit(0.0, 4), G.asVector(4, col)),
                    G.transpose(B))
    with pytest.raises(E.EmitError, match="adjacent"):
        E.generate("bad4", e, [B], "cuda")
    assert not E.divisible(T.iadd(T.imul(T.IVar("i"), 6), T.IConst(0)), 4)
    assert E.divisible(T.iadd(T.imul(T.IVar("i"), 8), T.imul(T.IVar("j"), 4)), 4)


# --------------------------------------------------------------------------
# race freedom of loop nests (the property the paper's type system gives)
# --------------------------------------------------------------------------

from paper_1710_08332_gb300.codegen import check as CK  # noqa: E402


def _assign(acc):
    return T.Assign(acc, G.lit(1.0))


def test_checker_accepts_every_program():
    progs = [PR.dot_partials(4096, 512, 32), PR.dot_partials(4096, 512, 32, "contig", V=4),
             PR.asum_partials(4096, 512, 32), PR.scal(4096, 2.0, V=4), PR.gemv_partials(64, 512, 32),
             PR.fold_rows(64, 32), PR.fold_all(64), PR.dot_K1(64)]
    for e, _ in progs:
        comm, _ = T.translate(e)
        CK.check(comm)


def test_checker_rejects_racy_loop_nests():
    i, j = T.IVar("i"), T.IVar("j")
    out1 = T.AOut("out", G.arr(32, G.F32))
    # every local iteration writes out[0]
    with pytest.raises(CK.RaceError):
        CK.check(T.For(i, 32, "local", _assign(T.AIdx(out1, T.IConst(0)))))
    # the workgroup index is ignored: workgroups overwrite each other
    with pytest.raises(CK.RaceError):
        CK.check(T.For(i, 4, "workgroup", T.For(j, 32, "local", _assign(T.AIdx(out1, j)))))
    # out[i + j]: neighbouring iterations overlap
    out2 = T.AOut("out", G.arr(64, G.F32))
    with pytest.raises(CK.RaceError):
        CK.check(T.For(i, 4, "global", T.For(j, 32, "seq", _assign(T.AIdx(out2, T.iadd(i, j))))))
    # a private variable declared outside a thread-level loop is not per iteration
    t = T.Temp("acc", G.F32, "private")
    with pytest.raises(CK.RaceError):
        CK.check(T.New(t, T.For(i, 32, "local", _assign(T.AOut("acc", G.F32, t)))))


def test_checker_accepts_transposed_and_split_writes():
    i, j = T.IVar("i"), T.IVar("j")
    out = T.AOut("out", G.arr(32, 4, G.F32))
    # out[j][i] = offset j*4 + i: a mixed-radix numbering, injective
    CK.check(T.For(i, 4, "workgroup", T.For(j, 32, "local", _assign(T.AIdx(T.AIdx(T.ATranspose(out), i), j)))))
    # a value split 8 written element q -> out[q / 8][q % 8] = q
    flat = T.AOut("out", G.arr(16, 8, G.F32))
    CK.check(T.For(i, 128, "global", _assign(T.AIdx(T.ASplit(8, flat), i))))
    assert CK.linear_form(T.iadd(T.imul(T.idiv(i, 8), 8), T.imod(i, 8))) == ({"i": 1}, 0)
    assert CK.injective({"a": 1, "b": 32}, {"a": 32, "b": 4})
    assert not CK.injective({"a": 1, "b": 31}, {"a": 32, "b": 4})


# --------------------------------------------------------------------------
# rewrite-based strategy exploration
# --------------------------------------------------------------------------

from paper_1710_08332_gb300.codegen import rewrite as RW  # noqa: E402


def test_rewrite_rules_check_their_shapes():
    with pytest.raises(RW.RuleError):
        RW.rewrite("dot", RW.Derivation([RW.Rule("columns", (32, "interleaved"))]))
    with pytest.raises(RW.RuleError):
        RW.rewrite("dot", RW.Derivation([RW.Rule("split", (100,)), RW.Rule("vectorize", (8,))]))
    e = RW.rewrite("asum", RW.Derivation([RW.Rule("split", (512,)), RW.Rule("columns", (32, "contig"))]))
    assert e == RW.Reduce(RW.Each(RW.Reduce(RW.Each(RW.Reduce(RW.Map("abs", RW.HOLE)),
                                                    RW.Columns(32, "contig", RW.HOLE))),
                                  RW.Split(512, RW.Input("asum"))))
    ds = RW.derivations(1 << 16, splits=(4096,), threads=(128,), maps=("interleaved",), widths=(1, 4))
    assert [str(d) for d in ds] == ["split(4096) ; columns(128, interleaved) ; fuse ; lower",
                                    "split(4096) ; columns(128, interleaved) ; vectorize(4) ; fuse ; lower"]


@pytest.mark.parametrize("kind", ["dot", "asum"])
@pytest.mark.parametrize("tm,V", [("interleaved", 1), ("contig", 4)])
def test_derived_pipelines_match_oracle(c_build, kind, tm, V):
    """Every kernel of a derivation, run on the host, equals the oracle's
    evaluation of the same tree: per-thread folds (lanes with V), then the
    folding stages in order."""
    n, s, Tn = 1 << 14, 2048, 32
    d = RW.Derivation([RW.Rule("split", (s,)), RW.Rule("columns", (Tn, tm))]
                      + ([RW.Rule("vectorize", (V,))] if V > 1 else []) + [RW.Rule("fuse"), RW.Rule("lower")])
    x, y = uniform(n, 40), uniform(n, 41)
    cur = [x, y] if kind == "dot" else [x]
    for name, ph, ins in RW.lower(kind, d, n):
        f = G.compile_c("k_" + name, ph, ins)
        count = next(c for (_, _, c, role) in f.params if role == "out")
        out = np.zeros(count, np.float32)
        f.run(*cur, out, *f.temps_like())
        cur = [out]
    # the oracle's tree: lane folds per thread column, then the fold plan's strided stages
    if kind == "dot":
        items = c1.zip_(list(x), list(y)) if V == 1 else c1.zip_(c1.asVector(V, list(x)), c1.asVector(V, list(y)))
        g = (lambda p: F.mul(p[0], p[1])) if V == 1 else (lambda p: vmul(p[0], p[1]))
    else:
        items = list(x) if V == 1 else c1.asVector(V, list(x))
        g = F.abs if V == 1 else (lambda v: tuple(F.abs(q) for q in v))
    add = F.add if V == 1 else vadd
    zero = F.zero if V == 1 else (F.zero,) * V
    parts = c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda v, a: add(a, g(v)), zero, col), cols(ch, Tn, tm)),
        c1.split(s // V, items)))
    vals = parts if V == 1 else c1.asScalar(parts)
    for grp in RW.fold_plan(len(vals)):  # the derivation's folding stages, in order
        rows = len(vals) // grp  # output j folds vals[j], vals[rows + j], ... (strided groups)
        vals = [oracle_fold(vals[j::rows]) for j in range(rows)]
    assert len(vals) == 1 and bits(cur[0])[0] == bits(vals)[0]
    assert RW.fold_plan(1 << 19) == [128, 128, 32] and RW.fold_plan(96) == [96]
    assert RW.fold_plan(1 << 21) == [128, 128, 128] and RW.fold_plan(3 * 257) == [3 * 257]


def test_gemv_backward_programs_match_the_library_trees(c_build):
    """The generated dx (row chunks of R, then the chunk fold) computes the same
    tree as the library's dx kernel: equal to the loop-nest oracle of that
    kernel; dA = dy x^T exactly."""
    from oracle import loopnest

    M, N, R = 96, 72, 32
    A = np.random.default_rng(50).standard_normal((M, N)).astype(np.float32)
    dy, x = uniform(M, 51), uniform(N, 52)
    e, ins = PR.gemv_bwd_dx_partials(M, N, R)
    part = np.zeros(M // R * N, np.float32)
    G.compile_c("dxp", e, ins).run(A.ravel().copy(), dy, part)
    e, ins = PR.gemv_bwd_dx_fold(M // R, N)
    dx = np.zeros(N, np.float32)
    G.compile_c("dxf", e, ins).run(part, dx)
    assert np.array_equal(bits(dx), bits(loopnest.gemv_bwd_dx_f32(A, dy, R)))
    e, ins = PR.gemv_bwd_dA(M, N)
    dA = np.zeros(M * N, np.float32)
    G.compile_c("dA", e, ins).run(dy, x, dA)
    assert np.array_equal(bits(dA.reshape(M, N)), bits(loopnest.gemv_bwd_dA_f32(x, dy)))


@pytest.mark.parametrize("transA,transB,V", [(False, False, 1), (False, False, 4), (True, False, 4),
                                          (False, True, 1), (True, True, 1), (False, False, 2)])
@pytest.mark.parametrize("M,N,K", [(5, 12, 7), (33, 40, 65), (1, 4, 1)])
def test_gemm_matches_oracle(c_build, M, N, K, transA, transB, V):
    """The generated GEMM (a workgroup per row of C, columns over its threads,
    V adjacent columns per thread as a vector) folds every C_ij over k in
    order from +0, the product and the sum rounded separately: equal to the
    loop-nest oracle with contraction off, in all four operand layouts."""
    from oracle import loopnest

    rng = np.random.default_rng(60 + M + K)
    A = rng.uniform(-1, 1, (K, M) if transA else (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K) if transB else (K, N)).astype(np.float32)
    e, ins = PR.gemm(M, N, K, V, transA, transB)
    C = np.zeros((M, N), np.float32)
    G.compile_c(f"gemm_{M}_{N}_{K}_{int(transA)}{int(transB)}{V}", e, ins).run(A, B, C)
    want = loopnest.gemm_f32(A, B, transA, transB, contract_fma=False)
    assert np.array_equal(bits(C), bits(want))


@pytest.mark.parametrize("R,Cn,V,KV,transA,transB", [
    (4, 8, 4, 1, False, False), (8, 8, 4, 4, False, False), (2, 8, 2, 2, False, False),
    (4, 4, 1, 4, False, True), (8, 4, 4, 1, True, False), (4, 4, 1, 1, True, True), (1, 4, 4, 4, False, False)])
def test_gemm_tiled_matches_oracle(c_build, R, Cn, V, KV, transA, transB):
    """The register-tiled GEMM (a private R x Cn accumulator array per thread,
    A read as vectors along k when KV > 1, the group's KV steps an inner fold)
    still folds every C_ij over k in order from +0: equal to the loop-nest
    oracle with contraction off."""
    from oracle import loopnest

    M, N, K = 24, 40, 36
    rng = np.random.default_rng(100 + R + Cn + KV)
    A = rng.uniform(-1, 1, (K, M) if transA else (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K) if transB else (K, N)).astype(np.float32)
    e, ins = PR.gemm_tiled(M, N, K, R, Cn, V, KV, transA, transB)
    C = np.zeros(M * N, np.float32)
    G.compile_c(f"gemm_tiled_{R}{Cn}{V}{KV}{int(transA)}{int(transB)}", e, ins).run(A, B, C)
    want = loopnest.gemm_f32(A, B, transA, transB, contract_fma=False)
    assert np.array_equal(bits(C.reshape(M, N)), bits(want))


@pytest.mark.parametrize("R,Cn,V,KV,transA,transB", [(8, 8, 4, 4, False, False), (4, 4, 1, 1, True, True),
                                                   (4, 8, 4, 1, True, False), (2, 4, 1, 2, False, True)])
def test_gemm_tiled_fma_matches_oracle(c_build, R, Cn, V, KV, transA, transB):
    """With the contraction declared, every step is fma(a_ik, b_kj, c_ij) (one
    rounding, fmaf on the host): equal to the oracle's fold with fmaf, and not
    to the fold that rounds the product and the sum separately."""
    from oracle import loopnest

    M, N, K = 24, 40, 36
    rng = np.random.default_rng(140 + R + KV)
    A = rng.uniform(-1, 1, (K, M) if transA else (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K) if transB else (K, N)).astype(np.float32)
    e, ins = PR.gemm_tiled(M, N, K, R, Cn, V, KV, transA, transB, "fma")
    C = np.zeros(M * N, np.float32)
    G.compile_c(f"gemm_tiled_fma_{R}{Cn}{V}{KV}{int(transA)}{int(transB)}", e, ins).run(A, B, C)
    want = loopnest.gemm_f32(A, B, transA, transB, contract_fma=True)
    assert np.array_equal(bits(C.reshape(M, N)), bits(want))
    assert not np.array_equal(bits(C.reshape(M, N)), bits(loopnest.gemm_f32(A, B, transA, transB, contract_fma=False)))


def test_fma_phrase_types():
    x = G.inp("x", G.arr(8, G.F32))
    with pytest.raises(TypeError):
        G.fma(G.lit(1.0), G.vlit(1.0, 4), G.lit(0.0))
    with pytest.raises(ValueError):
        PR.gemm_tiled(8, 8, 8, 4, 4, 1, 1, False, False, "fast")
    e = G.mapGlobal(lambda v: G.fma(v, v, G.lit(1.0)), x)
    out = np.zeros(8, np.float32)
    xs = (np.arange(-4, 4) * 0.75).astype(np.float32)  # v * v + 1 exact: one rounding or two agree
    G.compile_c("fma_map", e, [x]).run(xs, out)
    want = (xs.astype(np.float64) ** 2 + 1.0).astype(np.float32)
    assert np.array_equal(bits(out), bits(want))


def test_gemm_derivations_match_oracle(c_build):
    """Every GEMM derivation (vector columns, register tiles, A along k) keeps
    each C_ij the same fold over k: all of them equal the oracle's fold."""
    from oracle import loopnest
    from paper_1710_08332_gb300.codegen import rewrite as RW

    M, N, K = 32, 32, 16
    rng = np.random.default_rng(160)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (K, N)).astype(np.float32)
    want = bits(loopnest.gemm_f32(A, B, False, False, contract_fma=False))
    ds = RW.gemm_derivations(M, N, K)
    assert len(ds) >= 12 and any("tile" in str(d) and "vectorize_k" in str(d) for d in ds)
    for d in ds:
        C = np.zeros(M * N, np.float32)
        tag = "_".join(str(a) for r in d.rules for a in r.args) or "plain"
        G.compile_c(f"gemm_deriv_{tag}", *RW.lower_gemm(d, M, N, K)).run(A, B, C)
        assert np.array_equal(bits(C.reshape(M, N)), want), str(d)
    with pytest.raises(RW.RuleError):
        RW.lower_gemm(RW.Derivation([RW.Rule("vectorize_k", (4,))]), M, N, K)
    with pytest.raises(RW.RuleError):
        RW.lower_gemm(RW.Derivation([RW.Rule("split", (4,))]), M, N, K)


def test_gemv_dx_derivations_match_oracle(c_build):
    """Every dx derivation (row chunks of R, columns as vectors or not) equals the
    oracle's dx for its own R: the chunk partials folded in chunk order."""
    from oracle import loopnest
    from paper_1710_08332_gb300.codegen import rewrite as RW

    M, N = 128, 72
    A = np.random.default_rng(180).standard_normal((M, N)).astype(np.float32)
    dy = uniform(M, 181)
    ds = RW.gemv_dx_derivations(M, N, row_splits=(16, 32, 64), widths=(1, 4))
    assert len(ds) == 6
    for d in ds:
        R = d.rules[0].args[0]
        cur = [A.ravel().copy(), dy]
        for name, ph, ins in RW.lower("gemv_dx", d, N, M):
            out = np.zeros(P_count(ph), np.float32)
            tag = "_".join(str(a) for r in d.rules for a in r.args)
            G.compile_c(f"dx_{name}_{tag}", ph, ins).run(*cur, out)
            cur = [out]
        assert np.array_equal(bits(cur[0]), bits(loopnest.gemv_bwd_dx_f32(A, dy, R))), str(d)
    with pytest.raises(RW.RuleError):
        RW.lower_gemv_dx(RW.Derivation([RW.Rule("vectorize", (4,))]), M, N)


def P_count(ph):
    from paper_1710_08332_gb300.codegen import phrase as PP

    return PP.scalar_count(ph.type) if isinstance(ph.type, PP.Arr) else 1


def test_array_accumulators_are_checked():
    """A reduce may accumulate an array of numbers (or vectors) only; the tiled
    GEMM rejects shapes that do not divide and vector loads across a transpose."""
    x = G.inp("x", G.arr(16, G.F32))
    with pytest.raises(TypeError):
        G.alit(0.0, G.F32)
    with pytest.raises(TypeError):  # the step must return the accumulator's type
        G.reduceSeq(lambda v, acc: v, G.alit(0.0, G.arr(4, G.F32)), x)
    for bad in ((24, 40, 36, 5, 8, 4, 1), (24, 40, 36, 4, 8, 3, 1), (24, 40, 36, 4, 8, 4, 5)):
        with pytest.raises(ValueError):
            PR.gemm_tiled(*bad)
    with pytest.raises(ValueError):
        PR.gemm_tiled(24, 40, 36, 4, 8, 4, 4, True, False)
    with pytest.raises(ValueError):
        PR.gemm_tiled(24, 40, 36, 4, 8, 4, 1, False, True)


def test_gemm_vector_columns_need_a_row_major_B():
    with pytest.raises(ValueError):
        PR.gemm(8, 16, 8, 4, False, True)
    with pytest.raises(ValueError):
        PR.gemm(8, 18, 8, 4)
    with pytest.raises(TypeError):
        G.splat(4, G.vlit(1.0, 4))


@pytest.mark.parametrize("V", [1, 4])
def test_dot_backward_matches_oracle(c_build, V):
    """dx = g y and dy = g x, the generated map applied to each stream."""
    from oracle import loopnest

    n = 4096 + 8
    x, y = uniform(n, 70), uniform(n, 71)
    g = np.array([-0.8125], np.float32)
    e, ins = PR.dot_bwd(n, V)
    f = G.compile_c(f"dot_bwd_{V}", e, ins)
    dx, dy = np.zeros(n, np.float32), np.zeros(n, np.float32)
    f.run(g, y, dx)
    f.run(g, x, dy)
    wx, wy = loopnest.dot_bwd_f32(x, y, float(g[0]))
    assert np.array_equal(bits(dx), bits(wx)) and np.array_equal(bits(dy), bits(wy))


def test_local_temporaries_are_bounded():
    X = G.inp("x", G.arr(1 << 16, G.F32))
    e = G.mapWorkgroup(lambda ch: G.reduceSeq(lambda v, a: G.add(a, v), 0.0,
                                              G.to_local(G.mapLocal(lambda v: G.mul(v, v), ch))),
                       G.split(1 << 14, X))  # 64 KiB of shared memory per block
    with pytest.raises(E.EmitError, match="48 KiB"):
        E.generate("big_local", e, [X], "cuda")


def test_input_names_must_not_clash_with_generated_names():
    for bad in ("t3", "out", "i1", "2x", "dpia_lane4"):
        X = G.inp(bad, G.arr(64, G.F32))
        with pytest.raises(E.EmitError):
            E.generate("k", G.mapGlobal(lambda v: G.mul(v, v), X), [X], "cuda")


def test_random_dot_strategies_match_oracle(c_build):
    """Thirty random derivations (split, threads, thread map, width) on random
    lengths: every generated pipeline equals the oracle's evaluation of its tree."""
    rng = np.random.default_rng(60)
    done = 0
    while done < 30:
        V = int(rng.choice([1, 2, 4]))
        Tn = int(rng.choice([1, 2, 8, 32, 64]))
        R = int(rng.integers(1, 6))
        s = Tn * V * R
        C = int(rng.integers(1, 5))
        n = s * C
        tm = str(rng.choice(["interleaved", "contig"]))
        x, y = uniform(n, 100 + done), uniform(n, 200 + done)
        e, ins = PR.dot_partials(n, s, Tn, tm, V=V)
        out = np.zeros(C * Tn * V, np.float32)
        G.compile_c(f"rd{done}", e, ins).run(x, y, out)
        if V == 1:
            want = oracle_dot_partials(x, y, s, Tn, tm)
        else:
            want = oracle_dot_partials_vec(x, y, s, Tn, tm, V)
        assert np.array_equal(bits(out), bits(want)), (n, s, Tn, tm, V)
        done += 1


@pytest.mark.parametrize("tm", ["interleaved", "contig"])
def test_compensated_pipeline_matches_oracle(c_build, tm):
    """Kahan pairs as the fold's accumulator: per-thread compensated sums, then
    group merges and the final merge, each equal to the oracle's kahan_step /
    kahan_combine evaluation of the same tree."""
    n, s, Tn, g = 1 << 13, 1024, 32, 16
    x, y = uniform(n, 70), uniform(n, 71)
    e, ins = PR.dot_partials_kahan(n, s, Tn, tm)
    part = np.zeros(2 * n // s * Tn, np.float32)
    G.compile_c("dk", e, ins).run(x, y, part)
    want = c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: c1.kahan_step(F, a, F.mul(p[0], p[1])),
                                                      (F.zero, F.zero), col), cols(ch, Tn, tm)),
        c1.split(s, c1.zip_(list(x), list(y)))))
    assert np.array_equal(bits(part), bits([v for pr in want for v in pr]))
    m = len(want)
    e, ins = PR.fold_pairs_rows(m // g, g)
    grp = np.zeros(2 * (m // g), np.float32)
    G.compile_c("kg", e, ins).run(part, grp)
    merged = [c1.reduce_(lambda pr, a: c1.kahan_combine(F, a, pr), (F.zero, F.zero), r) for r in c1.split(g, want)]
    assert np.array_equal(bits(grp), bits([v for pr in merged for v in pr]))
    e, ins = PR.fold_pairs_all(len(merged))
    out = np.zeros(1, np.float32)
    G.compile_c("kf", e, ins).run(grp, out)
    final = c1.reduce_(lambda pr, a: c1.kahan_combine(F, a, pr), (F.zero, F.zero), merged)
    assert bits(out)[0] == bits([final[0]])[0]


@pytest.mark.parametrize("rows,g", [(1, 7), (5, 128), (64, 3), (300, 32)])
def test_fold_cols_folds_strided_groups_in_order(c_build, rows, g):
    """fold_cols(rows, g): output j is the sequential f32 fold of p[j],
    p[rows + j], ..., p[(g - 1) rows + j] from +0 -- the transpose of split
    rows -- and its threads' reads are p[i], p[i + 1], ... for consecutive j."""
    p = np.random.default_rng(rows * 1000 + g).standard_normal(rows * g).astype(np.float32)
    out = np.zeros(rows, np.float32)
    e, ins = PR.fold_cols(rows, g)
    G.compile_c("fcols", e, ins).run(p, out)
    want = np.zeros(rows, np.float32)
    for j in range(rows):
        acc = np.float32(0.0)
        for k in range(g):
            acc = np.float32(acc + p[k * rows + j])
        want[j] = acc
    assert out.tobytes() == want.tobytes()
    src = B.cuda_source(E.generate("fcols", e, ins, backend="cuda"))
    assert "blockIdx" in src and "__global__" in src


# --------------------------------------------------------------------------
# the whole strategy in one kernel: lane trees, the block tree, the second
# level in the last work-group
# --------------------------------------------------------------------------


@pytest.mark.parametrize("n,s,T,V,tm,second,T2", [
    (1 << 14, 2048, 64, 4, "interleaved", "tree", 8), (1 << 14, 1024, 32, 1, "contig", "seq", 1),
    (1 << 15, 4096, 128, 4, "contig", "tree", 8), (4096, 512, 128, 4, "interleaved", "seq", 1),
    (1 << 13, 1024, 256, 2, "interleaved", "tree", 4), (1 << 12, 256, 8, 4, "interleaved", "tree", 16)])
def test_single_launch_reductions_match_oracle(c_build, n, s, T, V, tm, second, T2):
    """dot_R and asum_R (thread folds, lane trees within warps and over the warp
    sums, the second level) run as C equal the oracle's loop nest of the same
    strategy bit for bit."""
    from oracle import loopnest

    x, y = uniform(n, 80 + T), uniform(n, 81 + V)
    st = c1.Strategy(s=s, T=T, V=V, thread_map=tm, second=second, T2=max(T2, 1))
    e, ins = PR.dot_R(n, s, T, V, tm, second, T2)
    f = G.compile_c("dR", e, ins)
    out = np.zeros(1, np.float32)
    f.run(x, y, out, *f.temps_like())
    assert bits(out)[0] == bits([loopnest.dot_f32(x, y, st)])[0]
    e, ins = PR.asum_R(n, s, T, V, tm, second, T2)
    f = G.compile_c("aR", e, ins)
    f.run(x, out, *f.temps_like())
    assert bits(out)[0] == bits([loopnest.asum_f32(x, st)])[0]


def test_single_launch_gemv_matches_oracle(c_build):
    from oracle import loopnest

    rng = np.random.default_rng(90)
    M, N = 37, 1024
    A = rng.standard_normal((M, N)).astype(np.float32)
    xv = uniform(N, 91)
    for T, V in ((64, 4), (256, 1), (32, 4)):
        e, ins = PR.gemv_R(M, N, T, V)
        f = G.compile_c("gR", e, ins)
        y = np.zeros(M, np.float32)
        f.run(A.ravel().copy(), xv, y, *f.temps_like())
        assert np.array_equal(bits(y), bits(loopnest.gemv_f32(A, xv, c1.Strategy(s=N, T=T, V=V))))
    A2 = rng.standard_normal((40, N)).astype(np.float32)
    e, ins = PR.gemv_R_warp(40, N, 8, 4)
    f = G.compile_c("gRw", e, ins)
    y = np.zeros(40, np.float32)
    f.run(A2.ravel().copy(), xv, y, *f.temps_like())
    assert np.array_equal(bits(y), bits(loopnest.gemv_f32(A2, xv, c1.Strategy(s=N, T=32, V=4))))


def test_lane_trees_and_second_level_are_checked():
    """A lane tree needs a warp map around it, a warp map a work-group map, and
    the second level is a kernel's whole expression."""
    x = G.inp("x", G.arr(1024, G.F32))
    plus = lambda a, b: G.add(a, b)
    with pytest.raises(T.TranslationError, match="warp map"):
        T.translate(G.mapWorkgroup(lambda ch: G.reduceTree(plus, ch), G.split(32, x)))
    with pytest.raises(T.TranslationError, match="illegal nesting"):
        T.translate(G.mapWarp(lambda ch: G.reduceTree(plus, ch), G.split(32, x)))
    with pytest.raises(T.TranslationError, match="illegal nesting"):
        T.translate(G.mapWorkgroup(lambda ch: G.mapLane(lambda v: v, ch), G.split(32, x)))
    with pytest.raises(TypeError, match="power-of-two"):
        G.reduceTree(plus, G.inp("z", G.arr(24, G.F32)))
    parts = G.join(G.mapWorkgroup(lambda ch: G.mapWarp(lambda g: G.reduceTree(plus, g), G.split(32, ch)),
                                  G.split(64, x)))
    sl = G.secondLevel(parts, lambda p: G.reduceSeq(lambda v, a: G.add(a, v), 0.0, p))
    with pytest.raises(T.TranslationError, match="second level"):
        T.translate(G.add(sl, sl))
    comm, out = T.translate(sl)
    CK.check(comm)
    from paper_1710_08332_gb300.codegen import typecheck as TC

    TC.typecheck(comm, out)


@pytest.mark.skipif(not shutil.which("nvcc"), reason="nvcc not installed")
@pytest.mark.parametrize("n,s,T,V,tm,second,T2", [
    (1 << 14, 2048, 128, 4, "interleaved", "tree", 8), (1 << 14, 2048, 128, 4, "contig", "seq", 1),
    (1 << 13, 1024, 64, 1, "interleaved", "tree", 8), (1 << 12, 512, 32, 2, "interleaved", "seq", 1),
    (1 << 12, 256, 8, 4, "interleaved", "tree", 16)])
def test_compensated_single_launch_matches_oracle(c_build, n, s, T, V, tm, second, T2):
    """The compensated one-kernel dot and asum (lane-wise Kahan folds, lane pairs
    merged in lane order, trees and second level over (s, c) pairs, the final s)
    equal the oracle's compensated loop nest of the same strategy, and differ
    from the plain one."""
    from oracle import loopnest

    x, y = uniform(n, 90 + T), uniform(n, 91 + V)
    st = c1.Strategy(s=s, T=T, V=V, thread_map=tm, second=second, T2=max(T2, 1), compensated=True)
    out = np.zeros(1, np.float32)
    f = G.compile_c(f"dRk_{n}_{s}_{T}_{V}_{tm}_{second}", *PR.dot_R_kahan(n, s, T, V, tm, second, T2))
    f.run(x, y, out, *f.temps_like())
    assert bits(out)[0] == bits([loopnest.dot_f32(x, y, st)])[0]
    f = G.compile_c(f"aRk_{n}_{s}_{T}_{V}_{tm}_{second}", *PR.asum_R_kahan(n, s, T, V, tm, second, T2))
    f.run(x, out, *f.temps_like())
    assert bits(out)[0] == bits([loopnest.asum_f32(x, st)])[0]


def test_single_launch_sources_compile_for_sm103a(tmp_path):
    progs = {"dotR": PR.dot_R(1 << 20, 8192, 256, 4, "interleaved", "tree", 128),
             "dotRk": PR.dot_R_kahan(1 << 20, 8192, 256, 4, "interleaved", "tree", 128),
             "asumRk": PR.asum_R_kahan(1 << 20, 8192, 256, 4, "contig", "seq", 1),
             "asumR": PR.asum_R(1 << 20, 8192, 256, 4, "contig", "seq", 1),
             "gemvR": PR.gemv_R(512, 1024, 128, 4), "gemvRw": PR.gemv_R_warp(512, 1024, 8, 4)}
    for name, (e, ins) in progs.items():
        src = B.cuda_source(E.generate(name, e, ins, "cuda", unroll=4))
        assert "__shfl_down_sync" in src
        path = tmp_path / f"{name}.cu"
        path.write_text(src)
        r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-c",
                            str(path), "-o", str(tmp_path / f"{name}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


# --------------------------------------------------------------------------
# exploration beyond the reduce family: the one-kernel form, GEMV's row map,
# map fusion across kernels
# --------------------------------------------------------------------------


def _oracle_of_derivation(kind, d, x, y=None, A=None):
    """The oracle's value of a derivation's tree: c2 for the strategy's first
    level (or the whole one-kernel strategy), c1 for the folding stages."""
    from oracle import loopnest

    args = {r.name: r.args for r in d.rules}
    if kind == "gemv":
        if "rows" in args:  # a warp per row: 32 interleaved lanes, then the lane tree
            return loopnest.gemv_f32(A, x, c1.Strategy(s=A.shape[1], T=32, V=args.get("vectorize", (1,))[0]))
        T, tm = args["columns"]
        V = args.get("vectorize", (1,))[0]
        st = c1.Strategy(s=A.shape[1], T=T, V=V, thread_map=tm)
        if "tree" in args:
            return loopnest.gemv_f32(A, x, st)
        return np.array([oracle_fold(list(loopnest.lane_partials_f32("dot", row, x, st))) for row in A], np.float32)
    s, (T, tm), V = args["split"][0], args["columns"], args.get("vectorize", (1,))[0]
    src = loopnest.scal_f32(RW.SCALE, x) if kind == "asum_scal" else x
    k = "dot" if kind == "dot" else "asum"
    if "second" in args:
        kind2, T2 = args["second"]
        return np.float32((loopnest.dot_f32(src, y, c1.Strategy(s=s, T=T, V=V, thread_map=tm, second=kind2, T2=T2))
                           if k == "dot" else
                           loopnest.asum_f32(src, c1.Strategy(s=s, T=T, V=V, thread_map=tm, second=kind2, T2=T2))))
    vals = list(loopnest.lane_partials_f32(k, src, y, c1.Strategy(s=s, T=T, V=V, thread_map=tm)))
    for grp in RW.fold_plan(len(vals)):
        rows = len(vals) // grp
        vals = [oracle_fold(vals[j::rows]) for j in range(rows)]
    return np.float32(vals[0])


def _run_host(kind, d, inputs, n, M=0):
    cur = list(inputs)
    for name, ph, ins in RW.lower(kind, d, n, M):
        f = G.compile_c("h_" + name, ph, ins)
        count = next(c for (_, _, c, role) in f.params if role == "out")
        out = np.zeros(count, np.float32)
        f.run(*cur, out, *f.temps_like())
        cur = [out]
    return cur[0]


def test_rewrite_rules_for_one_kernel_rows_and_fusion():
    with pytest.raises(RW.RuleError, match="tree results"):
        RW.rewrite("dot", RW.Derivation([RW.Rule("split", (512,)), RW.Rule("columns", (32, "contig")),
                                         RW.Rule("second", ("tree", 8))]))
    with pytest.raises(RW.RuleError, match="Map f \\(Map g X\\)"):
        RW.rewrite("dot", RW.Derivation([RW.Rule("fuse_maps")]))
    with pytest.raises(RW.RuleError, match="32 lanes"):
        RW.rewrite("gemv", RW.Derivation([RW.Rule("rows", ("warp",)), RW.Rule("columns", (64, "interleaved"))]))
    e = RW.rewrite("asum_scal", RW.Derivation([RW.Rule("fuse_maps"), RW.Rule("split", (512,)),
                                               RW.Rule("columns", (32, "interleaved")), RW.Rule("tree"),
                                               RW.Rule("second", ("seq", 1))]))
    assert e == RW.Last("seq", 1, RW.Each(RW.Tree(RW.Each(RW.Reduce(RW.Map("abs.scale", RW.HOLE)),
                                                           RW.Columns(32, "interleaved", RW.HOLE))),
                                          RW.Split(512, RW.Input("asum_scal"))))
    n = 1 << 14
    d_un = RW.Derivation([RW.Rule("split", (1024,)), RW.Rule("columns", (64, "interleaved")), RW.Rule("tree"),
                          RW.Rule("second", ("tree", 16))])
    d_fu = RW.Derivation([RW.Rule("fuse_maps")] + d_un.rules)
    assert [k for k, _, _ in RW.lower("asum_scal", d_un, n)] == ["map_scale", "one_kernel"]
    assert [k for k, _, _ in RW.lower("asum_scal", d_fu, n)] == ["one_kernel"]
    assert len(RW.derivations(n, splits=(1024,), threads=(64,), maps=("contig",), widths=(4,),
                              forms=("paper", "single"), kind="asum_scal")) == 4


@pytest.mark.parametrize("form", ["paper", "single"])
def test_dot_and_asum_scal_derivations_match_oracle(c_build, form):
    """Every derivation (both thread maps, widths 1 and 4; for asum_scal with and
    without fuse_maps) equals the oracle's evaluation of its tree; fusing the
    maps changes no bit."""
    n = 1 << 14
    x, y = uniform(n, 400), uniform(n, 401)
    for kind in ("dot", "asum_scal"):
        got = {}
        for d in RW.derivations(n, splits=(2048,), threads=(64,), maps=("interleaved", "contig"), widths=(1, 4),
                                forms=(form,), kind=kind):
            v = _run_host(kind, d, [x, y] if kind == "dot" else [x], n)
            assert bits(v)[0] == bits([_oracle_of_derivation(kind, d, x, y)])[0], str(d)
            got.setdefault(str(d).replace("fuse_maps ; ", ""), set()).add(bits(v)[0])
        assert all(len(b) == 1 for b in got.values())


def test_gemv_derivations_match_oracle(c_build):
    """Rows at block level (one kernel with the row's tree, or partials and row
    folds) and at warp level, each equal to the oracle's evaluation of its tree."""
    rng = np.random.default_rng(402)
    M, N = 24, 512
    A = rng.standard_normal((M, N)).astype(np.float32)
    xv = uniform(N, 403)
    ds = RW.gemv_derivations(M, N, threads=(32, 128), widths=(1, 4))
    assert any(r.name == "rows" for d in ds for r in d.rules)
    for d in ds:
        got = _run_host("gemv", d, [A.ravel().copy(), xv], N, M)
        assert np.array_equal(bits(got), bits(_oracle_of_derivation("gemv", d, xv, A=A))), str(d)
