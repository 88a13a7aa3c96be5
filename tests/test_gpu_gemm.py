"""GPU parity of the GEMM instances.

FP32 fold: bit-identical to the oracle's sequential k loop (both contractions,
all four operand layouts, ragged shapes, and 96 full rows of C at 4096^3).
BF16 tensor cores: the cast is bit-exact against round-to-nearest-even; the
product is checked against FP64 of the bf16-rounded inputs (||C - C64||_F /
||C64||_F <= 1e-4, and per element within the f32 accumulation bound) and
against FP64 of the original FP32 inputs (<= 2e-2); at 4096^3 every element of
the forward and both backward products.
"""
import numpy as np
import pytest
import torch

import paper_1710_08332_gb300 as dpia
from oracle import loopnest, naive64
from synth import workloads as W
from tests.helpers import assert_bits_equal, host

pytestmark = pytest.mark.gpu


def _store(op, trans):
    """The stored matrix whose op() is `op` (row-major)."""
    return np.ascontiguousarray(op.T) if trans else np.ascontiguousarray(op)


@pytest.mark.parametrize("contract", ["fma", "off"])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(256, 384, 80), (300, 257, 70), (1, 129, 3), (128, 128, 16), (260, 132, 84),
                                   (200, 264, 36), (384, 256, 4)])
def test_gemm_f32_bits(cuda_device, contract, tA, tB, M, N, K):
    """Every layout and both contractions; shapes whose rows are 16-byte multiples
    (with the declared contraction and B not transposed: the TMA-staged kernel,
    including ragged M and N and a k tail) and shapes that are not (the
    register-staged kernel)."""
    g = torch.Generator().manual_seed(M * 7 + N + K)
    opA = torch.randn(M, K, generator=g).numpy()
    opB = torch.randn(K, N, generator=g).numpy()
    A, B = _store(opA, tA), _store(opB, tB)
    C = torch.full((M, N), float("nan"), device="cuda")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dpia.dpia_gemm_f32(Ad, Bd, C, M, N, K, A.shape[1], B.shape[1], N, tA, tB, contract)
    want = loopnest.gemm_f32(A, B, bool(tA), bool(tB), contract == "fma")
    assert_bits_equal(host(C), want, f"gemm f32 {contract} tA={tA} tB={tB} {M}x{N}x{K}")


def test_gemm_f32_unaligned_leading_dims(cuda_device):
    M, N, K = 70, 90, 33
    g = torch.Generator().manual_seed(3)
    A = torch.randn(M, K + 3, generator=g)
    B = torch.randn(K, N + 1, generator=g)
    C = torch.zeros(M, N + 2, device="cuda")
    dpia.dpia_gemm_f32(A.cuda(), B.cuda(), C, M, N, K, K + 3, N + 1, N + 2, 0, 0, "fma")
    want = loopnest.gemm_f32(A[:, :K].contiguous().numpy(), B[:, :N].contiguous().numpy(), False, False, True)
    assert_bits_equal(host(C)[:, :N], want, "unaligned")


@pytest.fixture(scope="module")
def gemm_inputs():
    A, B, dC = W.gemm("cuda")
    return A, B, dC


def _f32_rows_4096(n):
    """Rows of C checked at 4096^3: two in every 128-row tile row (at offsets that
    vary from tile to tile) and every 16th row of the last 512 -- 96 rows, all
    columns."""
    rows = set()
    for t in range(n // 128):
        rows.add(t * 128 + (t * 41) % 128)
        rows.add(t * 128 + 127 - (t * 23) % 128)
    rows.update(range(n - 512, n, 16))
    return np.array(sorted(rows))


def test_gemm_f32_4096_rows(cuda_device, gemm_inputs):
    """The FP32 fold at 4096^3 (the automatic schedule: one launch) against the
    oracle's fold, bit for bit, on 96 full rows of C (every tile row), and
    within the summation bound of FP64 there; all of C is the same bits under
    the half-tile and k-range piece schedules."""
    A, B, _ = gemm_inputs
    n = W.GEMM_MNK
    C = torch.empty(n, n, device="cuda")
    dpia.dpia_gemm_f32(A, B, C, n, n, n, n, n, n, 0, 0, "fma")
    for sched in (2, 3):
        C2 = torch.empty(n, n, device="cuda")
        dpia.dpia_gemm_f32(A, B, C2, n, n, n, n, n, n, 0, 0, "fma", schedule=sched)
        assert torch.equal(C2.view(torch.int32), C.view(torch.int32)), f"schedule {sched}"
        del C2
    rows = _f32_rows_4096(n)
    assert rows.size >= 64
    hA, hB = host(A), host(B)
    want = loopnest.gemm_f32_sample(hA, hB, False, False, True, rows, np.arange(n))
    got = host(C)[rows]
    assert_bits_equal(got, want, "gemm f32 4096 rows")
    ref = hA[rows].astype(np.float64) @ hB.astype(np.float64)
    scale = np.abs(hA[rows]).astype(np.float64) @ np.abs(hB).astype(np.float64)
    assert np.all(np.abs(got - ref) <= (n + 1) * 2.0 ** -24 * scale)


def test_cast_bf16_exact(cuda_device):
    x = torch.randn(1 << 20, device="cuda") * 3
    x[:6] = torch.tensor([0.0, -0.0, 1e-40, -3e38, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8])
    y = torch.empty(x.numel() + 3, dtype=torch.bfloat16, device="cuda")[:x.numel()]
    dpia.dpia_cast_f32_bf16(x, y, x.numel())
    want = naive64.bf16_round(host(x))
    assert np.array_equal(host(y.float()).astype(np.float64), want)
    assert np.array_equal(np.signbit(host(y.float())), np.signbit(want))


class Bf16Ref:
    """FP64 references of op(A) op(B) for the BF16 GEMM's tolerance checks: the
    product of the bf16-rounded operands, its f32 accumulation bound
    (K + 2) 2^-23 (|A16| |B16|)_ij, and the product of the original f32
    operands. Computed once, for checks of several kernels on one product."""

    def __init__(self, opA, opB):
        a16 = naive64.bf16_round(opA)
        b16 = naive64.bf16_round(opB)
        self.ref16 = a16 @ b16
        self.bound = (opA.shape[1] + 2) * 2.0 ** -23 * (np.abs(a16) @ np.abs(b16)) + 1e-30
        self.ref32 = opA.astype(np.float64) @ opB.astype(np.float64)

    def check(self, C, what):
        rel = np.linalg.norm(C - self.ref16) / np.linalg.norm(self.ref16)
        assert rel <= 1e-4, f"{what}: rel err vs bf16 inputs {rel}"
        worst = np.max(np.abs(C - self.ref16) / self.bound)
        assert worst <= 1.0, f"{what}: elementwise error {worst} x the f32 accumulation bound"
        rel32 = np.linalg.norm(C - self.ref32) / np.linalg.norm(self.ref32)
        assert rel32 <= 2e-2, f"{what}: rel err vs f32 inputs {rel32}"
        return rel, rel32


def _bf16_check(C, opA, opB, what):
    """C against FP64 of the bf16-rounded operands (tight) and of the f32 ones (loose)."""
    return Bf16Ref(opA, opB).check(C, what)


@pytest.mark.parametrize("tile_n", [0, 128, 224, 256])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(256, 512, 256), (200, 300, 136), (384, 256, 64), (128, 768, 1024),
                                   (520, 900, 200)])
def test_gemm_bf16_tolerance(cuda_device, tA, tB, M, N, K, tile_n):
    g = torch.Generator().manual_seed(M + 3 * N + 7 * K + tA + 2 * tB)
    opA = torch.randn(M, K, generator=g).numpy()
    opB = torch.randn(K, N, generator=g).numpy()
    A, B = _store(opA, tA), _store(opB, tB)
    # leading dimensions padded to multiples of 8 elements (16 bytes), as TMA requires
    lda = (A.shape[1] + 7) // 8 * 8
    ldb = (B.shape[1] + 7) // 8 * 8
    Ad = torch.zeros(A.shape[0], lda, device="cuda")
    Ad[:, :A.shape[1]] = torch.from_numpy(A)
    Bd = torch.zeros(B.shape[0], ldb, device="cuda")
    Bd[:, :B.shape[1]] = torch.from_numpy(B)
    Ab, Bb = dpia.to_bf16(Ad), dpia.to_bf16(Bd)
    C = torch.full((M, N), float("nan"), device="cuda")
    dpia.dpia_gemm_bf16(Ab, Bb, C, M, N, K, lda, ldb, N, tA, tB, tile_n=tile_n)
    torch.cuda.synchronize()
    _bf16_check(host(C).astype(np.float64), opA, opB, f"bf16 tA={tA} tB={tB} {M}x{N}x{K} tile_n={tile_n}")
    assert dpia.dpia_poll_device_status() == 0


@pytest.mark.parametrize("cluster,tile_m", [(1, 0), (2, 256), (2, 512)])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K,tile_n", [(768, 448, 192, 224), (520, 300, 136, 0), (1024, 256, 64, 128),
                                          (100, 520, 320, 160), (384, 200, 72, 256), (1280, 96, 128, 128),
                                          (600, 301, 64, 0)])
def test_gemm_bf16_cta_pairs(cuda_device, tA, tB, M, N, K, tile_n, cluster, tile_m):
    """One CTA per 256-row tile (cluster 1) or a CTA pair (cluster 2: each CTA
    stages 128 rows of every 256-row block of A and half of B's columns, one
    M=256 MMA per block across both; tile_m 512 = two blocks per tile):
    ragged M, N and K, tiles whose later blocks lie past M (M = 100, 384, 520,
    768 with 512-row tiles), odd halves of B (tile_n 160: 80 columns per CTA),
    N below one tile, C rows not a multiple of 16 bytes apart (N = 301: no
    tensor map of C, stored element by element), and a small persistent grid
    (several tiles per pair, both accumulator sets of each CTA in turn)."""
    g = torch.Generator().manual_seed(11 * M + 5 * N + K + tA + 2 * tB)
    opA = torch.randn(M, K, generator=g).numpy()
    opB = torch.randn(K, N, generator=g).numpy()
    A, B = _store(opA, tA), _store(opB, tB)
    lda = (A.shape[1] + 7) // 8 * 8
    ldb = (B.shape[1] + 7) // 8 * 8
    Ad = torch.zeros(A.shape[0], lda, device="cuda")
    Ad[:, :A.shape[1]] = torch.from_numpy(A)
    Bd = torch.zeros(B.shape[0], ldb, device="cuda")
    Bd[:, :B.shape[1]] = torch.from_numpy(B)
    Ab, Bb = dpia.to_bf16(Ad), dpia.to_bf16(Bd)
    for grid in (0, 2):
        C = torch.full((M, N), float("nan"), device="cuda")
        dpia.dpia_gemm_bf16(Ab, Bb, C, M, N, K, lda, ldb, N, tA, tB, grid=grid, tile_m=tile_m, tile_n=tile_n,
                            cluster=cluster)
        torch.cuda.synchronize()
        _bf16_check(host(C).astype(np.float64), opA, opB,
                    f"bf16 cluster={cluster} tile_m={tile_m} grid={grid} tA={tA} tB={tB} {M}x{N}x{K}")
        assert dpia.dpia_poll_device_status() == 0


@pytest.mark.parametrize("cluster,tile_m", [(1, 0), (2, 256), (2, 512)])
@pytest.mark.parametrize("offset", [4, 1])
def test_gemm_bf16_strided_c_untouched_outside(cuda_device, cluster, tile_m, offset):
    """C as a column window of a wider matrix (ldc > N): with a 16-byte aligned
    window (offset 4) C is written through its tensor map, whose bounds clip
    the ragged tiles; with offset 1 element by element. Either way exactly the
    M x N window changes: the columns beside it keep their NaNs."""
    M, N, K = 700, 296, 200  # K and N multiples of 8: A's and B's rows 16-byte aligned, as TMA needs
    g = torch.Generator().manual_seed(99 + offset + cluster)
    opA = torch.randn(M, K, generator=g).numpy()
    opB = torch.randn(K, N, generator=g).numpy()
    Ab = dpia.to_bf16(torch.from_numpy(opA).cuda())
    Bb = dpia.to_bf16(torch.from_numpy(opB).cuda())
    ldc = N + 20
    big = torch.full((M, ldc), float("nan"), device="cuda")
    C = big[:, offset:offset + N]
    dpia.dpia_gemm_bf16(Ab, Bb, C, M, N, K, K, N, ldc, 0, 0, tile_m=tile_m, cluster=cluster)
    torch.cuda.synchronize()
    assert dpia.dpia_poll_device_status() == 0
    _bf16_check(host(C).astype(np.float64), opA, opB, f"strided C offset={offset} cluster={cluster}")
    hb = host(big)
    assert np.isnan(hb[:, :offset]).all() and np.isnan(hb[:, offset + N:]).all()


@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0)])
def test_gemm_bf16_variants_4096(cuda_device, gemm_inputs, tA, tB):
    """At 4096^3, in the three operand layouts of the forward and backward
    products, every kernel variant -- one CTA per 256-row tile, CTA pairs with
    256- and 512-row tiles -- computes every element of C within the f32
    accumulation bound of the FP64 product of the bf16-rounded operands (and
    the Frobenius bounds); the variants agree to a few f32 ulps."""
    A, B, _ = gemm_inputs
    n = W.GEMM_MNK
    Ab, Bb = dpia.to_bf16(A), dpia.to_bf16(B)
    out = []
    for cluster, tile_m in ((1, 0), (2, 256), (2, 512)):
        C = torch.empty(n, n, device="cuda")
        dpia.dpia_gemm_bf16(Ab, Bb, C, n, n, n, n, n, n, tA, tB, tile_m=tile_m, tile_n=224, cluster=cluster)
        out.append(C)
    torch.cuda.synchronize()
    assert dpia.dpia_poll_device_status() == 0
    hA, hB = host(A), host(B)
    ref = Bf16Ref(hA.T if tA else hA, hB.T if tB else hB)
    for C, label in zip(out, ("one SM", "pair 256", "pair 512")):
        ref.check(host(C).astype(np.float64), f"4096^3 {label} tA={tA} tB={tB}")
    scale = out[0].abs().max().item()
    for C in out[1:]:
        d = (out[0] - C).abs().max().item()
        assert d <= 1e-5 * scale, (d, scale)


def test_gemm_bf16_4096(cuda_device, gemm_inputs):
    """The GEMM workload (4096^3) with the default kernel choice: forward and
    both backward products, every element checked."""
    A, B, dC = gemm_inputs
    n = W.GEMM_MNK
    Ab, Bb, dCb = dpia.to_bf16(A), dpia.to_bf16(B), dpia.to_bf16(dC)
    hA, hB, hdC = host(A), host(B), host(dC)
    C = torch.empty(n, n, device="cuda")
    dpia.dpia_gemm_bf16(Ab, Bb, C, n, n, n, n, n, n, 0, 0)            # C = A B
    _bf16_check(host(C).astype(np.float64), hA, hB, "C = A B")
    dA = torch.empty(n, n, device="cuda")
    dpia.dpia_gemm_bf16(dCb, Bb, dA, n, n, n, n, n, n, 0, 1)          # dA = dC B^T
    _bf16_check(host(dA).astype(np.float64), hdC, hB.T, "dA = dC B^T")
    dB = torch.empty(n, n, device="cuda")
    dpia.dpia_gemm_bf16(Ab, dCb, dB, n, n, n, n, n, n, 1, 0)          # dB = A^T dC
    _bf16_check(host(dB).astype(np.float64), hA.T, hdC, "dB = A^T dC")
    assert dpia.dpia_poll_device_status() == 0


def test_gemm_validation(cuda_device):
    A = torch.zeros(64, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, 64, device="cuda")
    with pytest.raises(dpia.DPIAError, match="ALIGN"):
        dpia.dpia_gemm_bf16(A, A, C, 60, 60, 60, 60, 64, 64, 0, 0)  # lda not a multiple of 8
    with pytest.raises(dpia.DPIAError, match="ALIAS"):
        dpia.dpia_gemm_f32(C, C, C, 64, 64, 64, 64, 64, 64, 0, 0)
    with pytest.raises(dpia.DPIAError, match="SHAPE"):
        dpia.dpia_gemm_f32(C, C, torch.zeros(4, device="cuda"), 64, 64, 64, 32, 64, 64, 0, 0)


@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1)])
def test_gemm_f32_tail_rows_as_half_tiles(cuda_device, tA, tB):
    """Schedule 2: 2560 x 2048 tiles fill more than the SMs hold with a small last wave: the
    last tile row runs as half-height tiles in a second launch; every element
    is still the oracle's fold."""
    M, N, K = 2560, 2048, 64
    A = (torch.randn(K, M) if tA else torch.randn(M, K)).numpy()
    B = (torch.randn(N, K) if tB else torch.randn(K, N)).numpy()
    C = torch.full((M, N), float("nan"), device="cuda")
    dpia.dpia_gemm_f32(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, M, N, K, A.shape[1], B.shape[1],
                       N, tA, tB, "fma", schedule=2)
    torch.cuda.synchronize()
    rows = np.r_[0:8, 2300:2560]
    want = loopnest.gemm_f32_sample(A, B, bool(tA), bool(tB), True, rows, np.arange(N))
    assert_bits_equal(host(C)[rows], want, f"tail tA={tA} tB={tB}")


def _two_rows_per_tile_row(M):
    rows = set()
    for t in range((M + 127) // 128):
        lo, hi = t * 128, min(M, t * 128 + 128)
        rows.add(lo + (t * 37) % (hi - lo))
        rows.add(hi - 1 - (t * 11) % (hi - lo))
    return np.array(sorted(rows))


@pytest.mark.parametrize("contract", ["fma", "off"])
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(3500, 3490, 300), (3584, 3584, 40), (3584, 3584, 48)])
def test_gemm_f32_pieces_bits(cuda_device, contract, tA, tB, M, N, K):
    """k-range pieces (schedule 3): 784 tiles, each CTA's range cut at k-slices
    that differ from tile to tile (ragged M and N, a k tail of 12 or 8; or
    every tile interior with K a multiple of 16, the EXACT instances), the
    cut tiles' folds carried through C from the first launch to the second.
    All of C is the same bits under schedules 1, 2, 3 and 0, and two rows of
    every tile row are the oracle's fold."""
    g = torch.Generator().manual_seed(M + 3 * N + K)
    opA = torch.randn(M, K, generator=g).numpy()
    opB = torch.randn(K, N, generator=g).numpy()
    A, B = _store(opA, tA), _store(opB, tB)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = {}
    for sched in (3, 1, 2, 0):
        C = torch.full((M, N), float("nan"), device="cuda")
        dpia.dpia_gemm_f32(Ad, Bd, C, M, N, K, A.shape[1], B.shape[1], N, tA, tB, contract, schedule=sched)
        out[sched] = C
    torch.cuda.synchronize()
    for sched in (1, 2, 0):
        assert torch.equal(out[sched].view(torch.int32), out[3].view(torch.int32)), f"schedule {sched} vs 3"
    rows = _two_rows_per_tile_row(M)
    want = loopnest.gemm_f32_sample(A, B, bool(tA), bool(tB), contract == "fma", rows, np.arange(N))
    assert_bits_equal(host(out[3])[rows], want, f"pieces {contract} tA={tA} tB={tB} {M}x{N}x{K}")


def test_gemm_f32_pieces_refused_when_they_do_not_fit(cuda_device):
    """Schedule 3 needs at least two tiles' k-slices per resident CTA: 4 x 4
    tiles are refused with a strategy error, before any launch."""
    A = torch.zeros(512, 512, device="cuda")
    C = torch.zeros(512, 512, device="cuda")
    with pytest.raises(dpia.DPIAError, match="STRATEGY"):
        dpia.dpia_gemm_f32(A, A.clone(), C, 512, 512, 512, 512, 512, 512, 0, 0, "fma", schedule=3)
