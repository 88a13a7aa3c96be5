"""Generated CUDA kernels on the GPU: bit-identical to the oracle's evaluation
of the same phrase (c1), for every level mapping, thread mapping and address
space the generator handles, and under launch shapes other than the default
(the grid-stride loops make the result independent of them)."""
import numpy as np
import pytest
import torch

from oracle import patterns as c1
from paper_1710_08332_gb300 import codegen as G
from paper_1710_08332_gb300.codegen import programs as PR
from tests.test_codegen_host import bits, cols, oracle_dot_partials, oracle_fold, uniform

pytestmark = pytest.mark.gpu
F = c1.F32


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(kernel, *arrays, out_count, grid=None, block=None):
    out = torch.full((out_count,), float("nan"), device="cuda")
    kernel.run(*arrays, out, *kernel.temps_like(), grid=grid, block=block)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("thread_map", ["interleaved", "contig"])
def test_dot_two_kernels(cuda_device, thread_map):
    n, s, Tn = 1 << 16, 4096, 128
    x, y = uniform(n, 21), uniform(n, 22)
    e, ins = PR.dot_partials(n, s, Tn, thread_map)
    k = G.compile_cuda("dotp", e, ins)
    part = run(k, dev(x), dev(y), out_count=n // s * Tn)
    want = oracle_dot_partials(x, y, s, Tn, thread_map)
    assert np.array_equal(bits(part), bits(want))
    # other launch shapes: fewer blocks than chunks, fewer threads than columns
    for grid, block in ((3, 128), (16, 32), (64, 96)):
        again = run(k, dev(x), dev(y), out_count=n // s * Tn, grid=grid, block=block)
        assert np.array_equal(bits(again), bits(want))
    e2, ins2 = PR.fold_all(part.size)
    out = run(G.compile_cuda("fold", e2, ins2), dev(part), out_count=1)
    assert bits(out)[0] == bits([oracle_fold(want)])[0]


def test_asum_scal_gemv_k1(cuda_device):
    n, s, Tn = 1 << 15, 2048, 64
    x = uniform(n, 23)
    e, ins = PR.asum_partials(n, s, Tn, "interleaved")
    part = run(G.compile_cuda("asump", e, ins), dev(x), out_count=n // s * Tn)
    want = c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda v, a: F.add(a, F.abs(v)), F.zero, col),
                               cols(ch, Tn, "interleaved")), c1.split(s, list(x))))
    assert np.array_equal(bits(part), bits(want))

    e, ins = PR.scal(n, 1.5)
    out = run(G.compile_cuda("scal", e, ins), dev(x), out_count=n)
    assert np.array_equal(bits(out), bits(np.float32(1.5) * x))

    M, N, Tn = 300, 1024, 128
    A, xv = uniform(M * N, 24), uniform(N, 25)
    e, ins = PR.gemv_partials(M, N, Tn, "contig")
    part = run(G.compile_cuda("gemvp", e, ins), dev(A), dev(xv), out_count=M * Tn)
    want = c1.join(c1.mapWorkgroup(
        lambda row: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: F.add(a, F.mul(p[0], p[1])), F.zero, col),
                                cols(c1.zip_(row, list(xv)), Tn, "contig")), c1.split(N, list(A))))
    assert np.array_equal(bits(part), bits(want))
    e, ins = PR.fold_rows(M, Tn)
    y = run(G.compile_cuda("rows", e, ins), dev(part), out_count=M)
    assert np.array_equal(bits(y), bits([oracle_fold(r) for r in c1.split(Tn, want)]))

    x1, y1 = uniform(3000, 26), uniform(3000, 27)
    e, ins = PR.dot_K1(3000)
    out = run(G.compile_cuda("k1", e, ins), dev(x1), dev(y1), out_count=1)
    assert bits(out)[0] == bits([oracle_fold([F.mul(a, b) for a, b in zip(x1, y1)])])[0]


@pytest.mark.parametrize("space", ["global", "private", "local"])
def test_temporaries(cuda_device, space):
    n, s = 1 << 14, 512
    x, y = uniform(n, 28), uniform(n, 29)
    X, Y = G.inp("x", G.arr(n, G.F32)), G.inp("y", G.arr(n, G.F32))
    wrap = {"global": lambda e: e, "private": G.to_private, "local": G.to_local}[space]
    level = G.mapLocal if space == "local" else G.mapSeq
    e = G.mapWorkgroup(
        lambda ch: G.reduceSeq(lambda v, a: G.add(a, v), 0.0, wrap(level(lambda p: G.mul(G.fst(p), G.snd(p)), ch))),
        G.split(s, G.zip_(X, Y)))
    k = G.compile_cuda("tmp_" + space, e, [X, Y])
    want = c1.map_(lambda ch: oracle_fold(c1.map_(lambda p: F.mul(p[0], p[1]), ch)),
                   c1.split(s, c1.zip_(list(x), list(y))))
    for grid, block in ((None, 128), (5, 64)):
        out = run(k, dev(x), dev(y), out_count=n // s, grid=grid, block=block)
        assert np.array_equal(bits(out), bits(want))


@pytest.mark.parametrize("tm,V", [("interleaved", 1), ("interleaved", 4), ("contig", 4)])
def test_generated_dot_at_size_matches_oracle(cuda_device, tm, V):
    """n = 2^22: the generated partials kernel against the oracle's lane
    partials of the same strategy (c2), element by element, then the fold plan's
    stages against the oracle's strided folds of those partials (c1)."""
    from oracle import loopnest
    from oracle import patterns as P_
    from paper_1710_08332_gb300.codegen import rewrite as RW

    n, s, Tn = 1 << 22, 16384, 256
    x, y = uniform(n, 30), uniform(n, 31)
    e, ins = PR.dot_partials(n, s, Tn, tm, V=V)
    part = run(G.compile_cuda("dotp", e, ins, unroll=4), dev(x), dev(y), out_count=n // s * Tn * V)
    want = loopnest.lane_partials_f32("dot", x, y, P_.Strategy(s=s, T=Tn, V=V, thread_map=tm))
    assert np.array_equal(bits(part), bits(want))
    vals = list(want)
    cur = dev(part)
    for grp in RW.fold_plan(len(vals)):
        rows = len(vals) // grp
        ph, i2 = PR.fold_cols(rows, grp) if grp < len(vals) else PR.fold_all(len(vals))
        got = run(G.compile_cuda(f"fold{grp}_{rows}", ph, i2, unroll=64), cur, out_count=rows,
                  grid=max(1, rows // 64), block=min(64, rows))
        vals = [oracle_fold(vals[j::rows]) for j in range(rows)]
        assert np.array_equal(bits(got), bits(vals))
        cur = dev(got)


@pytest.mark.parametrize("thread_map", ["interleaved", "contig"])
def test_vector_kernels(cuda_device, thread_map):
    from tests.test_codegen_host import oracle_dot_partials_vec, vmul, vadd

    n, s, Tn = 1 << 16, 4096, 128
    x, y = uniform(n, 32), uniform(n, 33)
    e, ins = PR.dot_partials(n, s, Tn, thread_map, V=4)
    want = oracle_dot_partials_vec(x, y, s, Tn, thread_map)
    for unroll in (1, 4, 16):  # unrolling reorders no step of a sequential loop
        part = run(G.compile_cuda("dotv", e, ins, unroll=unroll), dev(x), dev(y), out_count=n // s * Tn * 4)
        assert np.array_equal(bits(part), bits(want))
    e2, ins2 = PR.fold_rows(part.size // 64, 64)
    folded = run(G.compile_cuda("fold64", e2, ins2, unroll=16), dev(part), out_count=part.size // 64,
                 grid=max(1, part.size // 64 // 256), block=256)
    assert np.array_equal(bits(folded), bits([oracle_fold(r) for r in c1.split(64, list(want))]))

    e, ins = PR.asum_partials(n, s, Tn, thread_map, V=4)
    part = run(G.compile_cuda("asumv", e, ins), dev(x), out_count=n // s * Tn * 4)
    zero = (F.zero,) * 4
    want = c1.asScalar(c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda v, a: vadd(a, tuple(F.abs(q) for q in v)), zero, col),
                               cols(ch, Tn, thread_map)), c1.split(s // 4, c1.asVector(4, list(x))))))
    assert np.array_equal(bits(part), bits(want))

    e, ins = PR.scal(n, 1.5, V=4)
    out = run(G.compile_cuda("scalv", e, ins), dev(x), out_count=n, grid=37, block=128)
    assert np.array_equal(bits(out), bits(np.float32(1.5) * x))

    M, N, Tn = 200, 2048, 128
    A, xv = uniform(M * N, 34), uniform(N, 35)
    e, ins = PR.gemv_partials(M, N, Tn, thread_map, V=4)
    part = run(G.compile_cuda("gemvv", e, ins), dev(A), dev(xv), out_count=M * Tn * 4)
    want = c1.asScalar(c1.join(c1.mapWorkgroup(
        lambda row: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: vadd(a, vmul(p[0], p[1])), zero, col),
                                cols(c1.zip_(c1.asVector(4, row), c1.asVector(4, list(xv))), Tn, thread_map)),
        c1.split(N, list(A)))))
    assert np.array_equal(bits(part), bits(want))


@pytest.mark.parametrize("kind", ["dot", "asum_scal"])
def test_exploration_ranks_derivations_and_each_is_exact_for_its_tree(cuda_device, kind):
    """The explored derivations -- the paper's form (partials, then folding
    kernels) and the one-kernel form (the chunk tree and the second level in
    the last block), for asum_scal with and without fusing the maps -- are
    ranked by time; the fastest three and slowest two each equal the oracle's
    evaluation of their own tree and lie within the normwise bound of the exact
    result (the bench compares the forms' times at the full size)."""
    from oracle import naive64
    from paper_1710_08332_gb300.codegen import rewrite as RW
    from tests.test_codegen_host import _oracle_of_derivation

    n = 1 << 22
    x, y = uniform(n, 42), uniform(n, 43)
    dx, dy = dev(x), dev(y)
    ins = [dx, dy] if kind == "dot" else [dx]
    derivs = RW.derivations(n, splits=(1 << 14, 1 << 15), threads=(128, 256),
                            maps=("interleaved", "contig"), widths=(1, 4), forms=("paper", "single"), kind=kind)
    ranked = RW.explore(kind, ins, n, derivs, reps=3)
    assert len(ranked) == len(derivs) and ranked[0][0] <= ranked[-1][0]
    if kind == "dot":
        exact, scale = naive64.dot_exact(x, y), naive64.abs_dot_f64(x, y)
    else:
        xs = np.float32(RW.SCALE) * x
        exact, scale = naive64.asum_exact(xs), naive64.asum_exact(xs)
    for _, d in ranked[:3] + ranked[-2:]:
        got = RW.run_pipeline(RW.compile_pipeline(kind, d, n), ins)
        torch.cuda.synchronize()
        want = _oracle_of_derivation(kind, d, x, y)
        assert bits(got.cpu().numpy())[0] == bits([want])[0], str(d)
        assert abs(float(want) - exact) <= 1e-5 * scale



def test_gemv_exploration_each_is_exact_for_its_tree(cuda_device):
    """GEMV derivations (rows at block level, one kernel or partials and row
    folds; rows at warp level) ranked on 8192 x 8192; the fastest and the
    slowest equal the oracle's evaluation of their trees on every row."""
    from paper_1710_08332_gb300.codegen import rewrite as RW
    from synth import workloads as W
    from tests.test_codegen_host import _oracle_of_derivation

    A, xv, _ = W.gemv("cuda")
    M, N = A.shape
    derivs = RW.gemv_derivations(M, N, threads=(128, 256), widths=(4,))
    ranked = RW.explore("gemv", [A, xv], N, derivs, reps=3, M=M)
    hA, hx = A.cpu().numpy(), xv.cpu().numpy()
    for _, d in ranked[:2] + ranked[-1:]:
        got = RW.run_pipeline(RW.compile_pipeline("gemv", d, N, M), [A, xv])
        torch.cuda.synchronize()
        assert np.array_equal(bits(got.cpu().numpy()), bits(_oracle_of_derivation("gemv", d, hx, A=hA))), str(d)


def test_generated_gemv_backward(cuda_device):
    from oracle import loopnest

    M, N, R = 512, 1000, 32
    A = np.random.default_rng(53).standard_normal((M, N)).astype(np.float32)
    dy, x = uniform(M, 54), uniform(N, 55)
    e, ins = PR.gemv_bwd_dx_partials(M, N, R)
    part = run(G.compile_cuda("dxp", e, ins, unroll=8), dev(A.ravel()), dev(dy), out_count=M // R * N)
    e, ins = PR.gemv_bwd_dx_fold(M // R, N)
    dx = run(G.compile_cuda("dxf", e, ins, unroll=8), dev(part), out_count=N, grid=4, block=256)
    assert np.array_equal(bits(dx), bits(loopnest.gemv_bwd_dx_f32(A, dy, R)))
    e, ins = PR.gemv_bwd_dA(M, N)
    dA = run(G.compile_cuda("dA", e, ins), dev(dy), dev(x), out_count=M * N)
    assert np.array_equal(bits(dA.reshape(M, N)), bits(loopnest.gemv_bwd_dA_f32(x, dy)))


def test_generated_compensated_dot(cuda_device):
    from tests.test_codegen_host import cols

    n, s, Tn = 1 << 16, 4096, 128
    x, y = uniform(n, 72), uniform(n, 73)
    e, ins = PR.dot_partials_kahan(n, s, Tn)
    part = run(G.compile_cuda("dk", e, ins, unroll=4), dev(x), dev(y), out_count=2 * n // s * Tn)
    want = c1.join(c1.mapWorkgroup(
        lambda ch: c1.mapLocal(lambda col: c1.reduce_(lambda p, a: c1.kahan_step(F, a, F.mul(p[0], p[1])),
                                                      (F.zero, F.zero), col), cols(ch, Tn, "interleaved")),
        c1.split(s, c1.zip_(list(x), list(y)))))
    assert np.array_equal(bits(part), bits([v for pr in want for v in pr]))
    e, ins = PR.fold_pairs_all(len(want))
    out = run(G.compile_cuda("kf", e, ins), dev(part), out_count=1)
    final = c1.reduce_(lambda pr, a: c1.kahan_combine(F, a, pr), (F.zero, F.zero), want)
    assert bits(out)[0] == bits([final[0]])[0]


# --------------------------------------------------------------------------
# the whole strategy in one generated kernel
# --------------------------------------------------------------------------


@pytest.mark.parametrize("n,s,T,V,tm,second,T2", [
    (1 << 20, 8192, 256, 4, "interleaved", "tree", 128), (1 << 20, 8192, 256, 4, "interleaved", "seq", 1),
    (1 << 20, 16384, 512, 4, "contig", "tree", 64), (1 << 18, 4096, 1024, 1, "interleaved", "tree", 64),
    (1 << 18, 2048, 64, 2, "contig", "seq", 1), (1 << 16, 512, 32, 4, "interleaved", "tree", 128)])
def test_single_launch_reductions_match_oracle_gpu(cuda_device, n, s, T, V, tm, second, T2):
    """dot_R / asum_R generated as one kernel each (thread folds, lane trees,
    the second level in the last block) equal the oracle's loop nest of the
    same strategy bit for bit, on consecutive launches (the ticket counter is
    back at zero after each) and under a smaller persistent grid."""
    from oracle import loopnest
    from oracle import patterns as P_

    x, y = uniform(n, 300 + T), uniform(n, 301 + V)
    st = P_.Strategy(s=s, T=T, V=V, thread_map=tm, second=second, T2=max(T2, 1))
    want_d, want_a = loopnest.dot_f32(x, y, st), loopnest.asum_f32(x, st)
    e, ins = PR.dot_R(n, s, T, V, tm, second, T2)
    kd = G.compile_cuda("dotR", e, ins, unroll=4)
    e, ins = PR.asum_R(n, s, T, V, tm, second, T2)
    ka = G.compile_cuda("asumR", e, ins, unroll=4)
    dx, dy = dev(x), dev(y)
    temps_d, temps_a = kd.temps_like(), ka.temps_like()
    for grid in (None, None, 37):
        out = torch.full((1,), float("nan"), device="cuda")
        kd.run(dx, dy, out, *temps_d, grid=grid)
        torch.cuda.synchronize()
        assert bits(out.cpu().numpy())[0] == bits([want_d])[0], grid
        ka.run(dx, out, *temps_a, grid=grid)
        torch.cuda.synchronize()
        assert bits(out.cpu().numpy())[0] == bits([want_a])[0], grid
    assert int(temps_d[-1].item()) == 0 and int(temps_a[-1].item()) == 0


def test_single_launch_dot_at_size_matches_oracle(cuda_device):
    """The bandwidth workload's dot (n = 2^26) as one generated kernel with the
    strategy the library's tuner picks most often (split 65536, 256 threads,
    float4 lanes, a tree second level over the 1024 chunk results): bit for
    bit the oracle's dot of the same strategy."""
    from oracle import loopnest
    from oracle import patterns as P_
    from synth import workloads as W

    x, y = W.bandwidth("cuda")
    n, s, T, V, T2 = x.numel(), 65536, 256, 4, 256
    e, ins = PR.dot_R(n, s, T, V, "interleaved", "tree", T2)
    k = G.compile_cuda("dotR26", e, ins, unroll=4)
    out = torch.empty(1, device="cuda")
    k.run(x, y, out, *k.temps_like())
    torch.cuda.synchronize()
    want = loopnest.dot_f32(x.cpu().numpy(), y.cpu().numpy(), P_.Strategy(s=s, T=T, V=V, second="tree", T2=T2))
    assert bits(out.cpu().numpy())[0] == bits([want])[0]


@pytest.mark.parametrize("M,N,T,V", [(8192, 8192, 128, 4), (300, 1024, 256, 1), (64, 4096, 1024, 4)])
def test_single_launch_gemv_matches_oracle_gpu(cuda_device, M, N, T, V):
    """gemv_R (a block per row) and gemv_R_warp (a warp per row) against the
    oracle's GEMV of the same strategy, every row."""
    from oracle import loopnest
    from oracle import patterns as P_

    rng = np.random.default_rng(M + N)
    A = (rng.standard_normal((M, N)) / np.sqrt(N)).astype(np.float32)
    xv = uniform(N, 310)
    dA, dxv = dev(A.ravel()), dev(xv)
    e, ins = PR.gemv_R(M, N, T, V)
    got = run(G.compile_cuda("gemvR", e, ins, unroll=4), dA, dxv, out_count=M)
    assert np.array_equal(bits(got), bits(loopnest.gemv_f32(A, xv, P_.Strategy(s=N, T=T, V=V))))
    if M % 8 == 0:
        e, ins = PR.gemv_R_warp(M, N, 8, 4)
        got = run(G.compile_cuda("gemvRw", e, ins, unroll=4), dA, dxv, out_count=M)
        assert np.array_equal(bits(got), bits(loopnest.gemv_f32(A, xv, P_.Strategy(s=N, T=32, V=4))))


@pytest.mark.parametrize("transA,transB,V", [(False, False, 4), (True, False, 4), (False, True, 1),
                                          (True, True, 1), (False, False, 1)])
def test_generated_gemm_matches_oracle(cuda_device, transA, transB, V):
    """The generated GEMM, every C_ij one fold over k from +0 (product and sum
    rounded separately), in all four operand layouts: equal to the loop-nest
    oracle with contraction off, under the default launch and smaller grids
    and blocks (row and column loops stride over what the launch covers)."""
    from oracle import loopnest

    M, N, K = 130, 264, 77
    rng = np.random.default_rng(80 + 2 * transA + transB)
    A = rng.standard_normal((K, M) if transA else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if transB else (K, N)).astype(np.float32)
    k = G.compile_cuda(f"gemm_{int(transA)}{int(transB)}_{V}", *PR.gemm(M, N, K, V, transA, transB), unroll=4)
    want = loopnest.gemm_f32(A, B, transA, transB, contract_fma=False)
    for grid, block in ((None, None), (7, 64), (200, 32)):
        got = run(k, dev(A), dev(B), out_count=M * N, grid=grid, block=block).reshape(M, N)
        assert np.array_equal(bits(got), bits(want)), (grid, block)


@pytest.mark.parametrize("R,Cn,V,KV,transA,transB,contract", [
    (4, 8, 4, 1, False, False, "off"), (8, 8, 4, 4, False, False, "off"), (4, 4, 1, 4, False, True, "off"),
    (8, 4, 4, 1, True, False, "off"), (4, 4, 1, 1, True, True, "off"), (8, 8, 4, 4, False, False, "fma"),
    (4, 4, 1, 1, True, True, "fma")])
def test_generated_tiled_gemm_matches_oracle(cuda_device, R, Cn, V, KV, transA, transB, contract):
    """The register-tiled GEMM (private accumulator arrays, A read along k as
    vectors when KV > 1) in every operand layout, under the default launch and
    smaller ones: equal to the loop-nest oracle with contraction off."""
    from oracle import loopnest

    M, N, K = 136, 264, 76
    rng = np.random.default_rng(120 + R + KV)
    A = rng.standard_normal((K, M) if transA else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if transB else (K, N)).astype(np.float32)
    k = G.compile_cuda(f"gemm_tiled_{R}{Cn}{V}{KV}{int(transA)}{int(transB)}_{contract}",
                       *PR.gemm_tiled(M, N, K, R, Cn, V, KV, transA, transB, contract))
    want = loopnest.gemm_f32(A, B, transA, transB, contract_fma=contract == "fma")
    for grid, block in ((None, None), (5, 32), (40, 128)):
        got = run(k, dev(A), dev(B), out_count=M * N, grid=grid, block=block).reshape(M, N)
        assert np.array_equal(bits(got), bits(want)), (grid, block)


@pytest.mark.parametrize("form", ["columns", "tiled", "tiled_fma"])
def test_generated_gemm_4096(cuda_device, form):
    """At 4096^3 (the float4-column form, the register-tiled form with 8 x 8
    tiles and A read along k, and a 16 x 8 tiled form with the contraction
    declared): every element equal to the library's FP32 fold with the same
    contraction (the same fold per element), and 96 full rows equal to the
    oracle's fold."""
    from oracle import loopnest
    from synth import workloads as W
    from tests.test_gpu_gemm import _f32_rows_4096

    import paper_1710_08332_gb300 as dpia

    n = W.GEMM_MNK
    A, B, _ = W.gemm("cuda")
    contract = "fma" if form == "tiled_fma" else "off"
    if form == "columns":
        k, block = G.compile_cuda("gemm_4096_v4", *PR.gemm(n, n, n, 4), unroll=4), None
    elif form == "tiled":
        k, block = G.compile_cuda("gemm_4096_tiled", *PR.gemm_tiled(n, n, n, 8, 8, 4, 4)), 128
    else:
        k, block = G.compile_cuda("gemm_4096_tiled_fma", *PR.gemm_tiled(n, n, n, 16, 8, 4, 4, contract="fma")), 128
    C = torch.empty(n * n, device="cuda")
    k.run(A, B, C, block=block)
    lib = torch.empty(n, n, device="cuda")
    dpia.dpia_gemm_f32(A, B, lib, n, n, n, n, n, n, 0, 0, contract)
    torch.cuda.synchronize()
    got = C.view(n, n)
    assert torch.equal(got.view(torch.int32), lib.view(torch.int32))
    rows = _f32_rows_4096(n)
    want = loopnest.gemm_f32_sample(A.cpu().numpy(), B.cpu().numpy(), False, False, contract == "fma", rows,
                                    np.arange(n))
    assert np.array_equal(bits(got.cpu().numpy()[rows]), bits(want))


@pytest.mark.parametrize("V", [1, 4])
def test_generated_dot_backward(cuda_device, V):
    """dx = g y, dy = g x from the generated map: equal to the oracle and to the
    library's dot backward."""
    from oracle import loopnest

    import paper_1710_08332_gb300 as dpia

    n = (1 << 20) + 4 * 7
    x, y = uniform(n, 90), uniform(n, 91)
    g = np.array([1.375], np.float32)
    k = G.compile_cuda(f"dot_bwd_{V}", *PR.dot_bwd(n, V))
    dx = run(k, dev(g), dev(y), out_count=n)
    dy = run(k, dev(g), dev(x), out_count=n)
    wx, wy = loopnest.dot_bwd_f32(x, y, float(g[0]))
    assert np.array_equal(bits(dx), bits(wx)) and np.array_equal(bits(dy), bits(wy))
    lx, ly = dpia.dot_bwd(dev(x), dev(y), dev(g))
    assert np.array_equal(bits(lx.cpu().numpy()), bits(dx)) and np.array_equal(bits(ly.cpu().numpy()), bits(dy))


def test_gemm_exploration_ranks_derivations_that_match_oracle(cuda_device):
    """The GEMM derivations on the GPU at 512^3: each one's output equals the
    oracle's fold, and the exploration ranks every (derivation, block) pair."""
    from oracle import loopnest
    from paper_1710_08332_gb300.codegen import rewrite as RW

    n = 512
    rng = np.random.default_rng(170)
    hA = rng.standard_normal((n, n)).astype(np.float32)
    hB = rng.standard_normal((n, n)).astype(np.float32)
    want = bits(loopnest.gemm_f32(hA, hB, False, False, contract_fma=False))
    A, B = dev(hA), dev(hB)
    ds = RW.gemm_derivations(n, n, n)
    for d in ds:
        tag = "_".join(str(a) for r in d.rules for a in r.args) or "plain"
        k = G.compile_cuda(f"xgemm_{n}_{n}_{n}_{tag}", *RW.lower_gemm(d, n, n, n),
                           unroll=1 if "tile" in str(d) else 4)
        got = run(k, A, B, out_count=n * n, block=128 if "tile" in str(d) else None)
        assert np.array_equal(bits(got.reshape(n, n)), want), str(d)
    ranked = RW.explore_gemm(A, B, n, n, n, ds, reps=2)
    assert len(ranked) == sum(2 if "tile" in str(d) else 1 for d in ds)
    assert [t[0] for t in ranked] == sorted(t[0] for t in ranked)


@pytest.mark.parametrize("n,s,second,T2", [(1 << 20, 8192, "seq", 1), (1 << 22, 16384, "tree", 256),
                                           (1 << 26, 16384, "tree", 256)])
def test_generated_compensated_dot_matches_oracle_and_library(cuda_device, n, s, second, T2):
    """The compensated one-kernel dot (Kahan at every level, trees over (s, c)
    pairs by shuffles) equals the oracle's compensated loop nest and the
    library's compensated dot, on two consecutive launches (the ticket resets)."""
    from oracle import loopnest
    from synth import workloads as W

    import paper_1710_08332_gb300 as dpia

    x, y = W.bandwidth("cuda", n=n)
    k = G.compile_cuda(f"dot_R_kahan_{n}_{s}_{second}", *PR.dot_R_kahan(n, s, 256, 4, "interleaved", second, T2),
                       unroll=4)
    temps = k.temps_like()
    outs = []
    for _ in range(2):
        out = torch.full((1,), float("nan"), device="cuda")
        k.run(x, y, out, *temps)
        outs.append(out)
    st = dpia.ReduceStrategy(split=s, threads=256, vec=4, second=second, threads2=T2, compensated=True)
    lib = torch.empty(1, device="cuda")
    dpia.dpia_dot_f32(x, y, n, st, lib, dpia.workspace(dpia.dpia_dot_workspace_size(n, st), "cuda"))
    torch.cuda.synchronize()
    want = loopnest.dot_f32(x.cpu().numpy(), y.cpu().numpy(),
                            c1.Strategy(s=s, T=256, V=4, second=second, T2=T2, compensated=True))
    for out in outs:
        assert bits(out.cpu().numpy())[0] == bits([want])[0]
    assert bits(lib.cpu().numpy())[0] == bits([want])[0]


def test_gemv_dx_exploration_matches_oracle(cuda_device):
    """GEMV dx derivations at 8192^2 on the GPU: the ranked pipelines, each run
    again, equal the oracle's dx for their own row split."""
    from oracle import loopnest
    from paper_1710_08332_gb300.codegen import rewrite as RW
    from synth import workloads as W

    A, _, dy = W.gemv("cuda")
    M, N = A.shape
    hA, hdy = A.cpu().numpy(), dy.cpu().numpy()
    ranked = RW.explore("gemv_dx", [A, dy], N, RW.gemv_dx_derivations(M, N), reps=2, M=M)
    assert len(ranked) == 12 and [t[0] for t in ranked] == sorted(t[0] for t in ranked)
    for _, d in (ranked[0], ranked[-1]):
        R = d.rules[0].args[0]
        pipe = RW.compile_pipeline("gemv_dx", d, N, M)
        got = RW.run_pipeline(pipe, [A, dy])
        torch.cuda.synchronize()
        assert np.array_equal(bits(got.cpu().numpy()), bits(loopnest.gemv_bwd_dx_f32(hA, hdy, R))), str(d)
