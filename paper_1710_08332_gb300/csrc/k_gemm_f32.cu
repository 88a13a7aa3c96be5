// FP32 GEMM on the CUDA cores: C = op(A) op(B) as
//   map (lambda a. map (lambda b. fold_k (a_k * b_k)) (transpose B)) A,
// each C_ij folded over k = 0..K-1 in order from +0, either with fmaf (the
// contraction declared) or with a separately rounded multiply and add.
//
// The map over C is split into 128 x 128 tiles (a block each; with the
// declared FMA, at most 128 registers so that two blocks share an SM); inside a
// tile, 256 threads own 8 x 8 elements each. k advances in slices of 16 staged in
// shared memory (double-buffered, the next slice prefetched through registers
// while the current one is consumed). Every element's fold stays one
// sequential chain in k, so the result is bit-identical to the oracle's loop.
// Interior-only shapes run an EXACT instance without edge cases. A partly
// empty last wave of tiles can be run as one launch, as half-height tiles in a
// second launch, or as k-range pieces over two launches (the cut folds carried
// through C); every schedule gives the same bits.
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

int resident_blocks(const void *kernel, int threads);

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

template <bool FMA>
__device__ __forceinline__ float madd(float a, float b, float acc) {
  if constexpr (FMA) return __fmaf_rn(a, b, acc);
  else return __fadd_rn(acc, __fmul_rn(a, b));
}

struct GemmArgs {
  const float *A, *B;
  float *C;
  int64_t M, N, K, lda, ldb, ldc;
};

// op(A)[m][k] and op(B)[k][n] element loads with bounds (0 outside).
template <bool TA>
__device__ __forceinline__ float a_at(const GemmArgs &g, int64_t m, int64_t k) {
  if (m >= g.M || k >= g.K) return 0.0f;
  return TA ? g.A[k * g.lda + m] : g.A[m * g.lda + k];
}
template <bool TB>
__device__ __forceinline__ float b_at(const GemmArgs &g, int64_t k, int64_t n) {
  if (k >= g.K || n >= g.N) return 0.0f;
  return TB ? g.B[n * g.ldb + k] : g.B[k * g.ldb + n];
}

// Load the (m0, k0) A slice and (k0, n0) B slice into registers: 8 + 8 floats
// per thread; `vec` selects 128-bit loads (interior, aligned tiles).
template <bool TA, bool TB>
__device__ __forceinline__ void load_slices(const GemmArgs &g, int64_t m0, int64_t n0, int64_t k0,
                                            bool vec, float (&ra)[8], float (&rb)[8]) {
  const int tid = threadIdx.x;
  if (vec) {
    if (!TA) {  // A[m][k]: thread -> row m = tid/2, k = (tid%2)*8 .. +7
      const float *p = g.A + (m0 + tid / 2) * g.lda + k0 + (tid % 2) * 8;
      float4 u = __ldg(reinterpret_cast<const float4 *>(p)), v = __ldg(reinterpret_cast<const float4 *>(p + 4));
      ra[0] = u.x; ra[1] = u.y; ra[2] = u.z; ra[3] = u.w; ra[4] = v.x; ra[5] = v.y; ra[6] = v.z; ra[7] = v.w;
    } else {  // A[k][m]: thread -> k = tid/16, m = (tid%16)*8 .. +7
      const float *p = g.A + (k0 + tid / 16) * g.lda + m0 + (tid % 16) * 8;
      float4 u = __ldg(reinterpret_cast<const float4 *>(p)), v = __ldg(reinterpret_cast<const float4 *>(p + 4));
      ra[0] = u.x; ra[1] = u.y; ra[2] = u.z; ra[3] = u.w; ra[4] = v.x; ra[5] = v.y; ra[6] = v.z; ra[7] = v.w;
    }
    if (!TB) {  // B[k][n]: thread -> k = tid/16, n = (tid%16)*8 .. +7
      const float *p = g.B + (k0 + tid / 16) * g.ldb + n0 + (tid % 16) * 8;
      float4 u = __ldg(reinterpret_cast<const float4 *>(p)), v = __ldg(reinterpret_cast<const float4 *>(p + 4));
      rb[0] = u.x; rb[1] = u.y; rb[2] = u.z; rb[3] = u.w; rb[4] = v.x; rb[5] = v.y; rb[6] = v.z; rb[7] = v.w;
    } else {  // B[n][k]: thread -> n = tid/2, k = (tid%2)*8 .. +7
      const float *p = g.B + (n0 + tid / 2) * g.ldb + k0 + (tid % 2) * 8;
      float4 u = __ldg(reinterpret_cast<const float4 *>(p)), v = __ldg(reinterpret_cast<const float4 *>(p + 4));
      rb[0] = u.x; rb[1] = u.y; rb[2] = u.z; rb[3] = u.w; rb[4] = v.x; rb[5] = v.y; rb[6] = v.z; rb[7] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!TA) ra[j] = a_at<TA>(g, m0 + tid / 2, k0 + (tid % 2) * 8 + j);
      else ra[j] = a_at<TA>(g, m0 + (tid % 16) * 8 + j, k0 + tid / 16);
      if (!TB) rb[j] = b_at<TB>(g, k0 + tid / 16, n0 + (tid % 16) * 8 + j);
      else rb[j] = b_at<TB>(g, k0 + (tid % 2) * 8 + j, n0 + tid / 2);
    }
  }
}

// Registers -> shared slices As[k][m], Bs[k][n].
template <bool TA, bool TB>
__device__ __forceinline__ void store_slices(float (*As)[BM], float (*Bs)[BN], const float (&ra)[8],
                                             const float (&rb)[8]) {
  const int tid = threadIdx.x;
  if (!TA) {
#pragma unroll
    for (int j = 0; j < 8; ++j) As[(tid % 2) * 8 + j][tid / 2] = ra[j];
  } else {
    *reinterpret_cast<float4 *>(&As[tid / 16][(tid % 16) * 8]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    *reinterpret_cast<float4 *>(&As[tid / 16][(tid % 16) * 8 + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
  }
  if (!TB) {
    *reinterpret_cast<float4 *>(&Bs[tid / 16][(tid % 16) * 8]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    *reinterpret_cast<float4 *>(&Bs[tid / 16][(tid % 16) * 8 + 4]) = make_float4(rb[4], rb[5], rb[6], rb[7]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) Bs[(tid % 2) * 8 + j][tid / 2] = rb[j];
  }
}

// Element (i, j) of a thread's 8 x 8 micro-tile: row m0 + ty*4 + i (i < 4) or
// m0 + 64 + ty*4 + (i-4); column n0 + h*64 + tx*4 + jj for j = 4h + jj.
template <bool EXACT>
__device__ __forceinline__ void load_c(const GemmArgs &g, int vec_ok, int64_t m0, int64_t n0, float (&acc)[8][8]) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (EXACT || (m < g.M && vec_ok && n + 4 <= g.N)) {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(g.C + m * g.ldc + n));
        acc[i][4 * h] = v.x; acc[i][4 * h + 1] = v.y; acc[i][4 * h + 2] = v.z; acc[i][4 * h + 3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][4 * h + j] = m < g.M && n + j < g.N ? __ldcg(g.C + m * g.ldc + n + j) : 0.0f;
      }
    }
  }
}

template <bool EXACT>
__device__ __forceinline__ void store_c(const GemmArgs &g, int vec_ok, int64_t m0, int64_t n0,
                                        const float (&acc)[8][8]) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (!EXACT && m >= g.M) continue;
    float *crow = g.C + m * g.ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (EXACT || (vec_ok && n + 4 <= g.N)) {
        *reinterpret_cast<float4 *>(crow + n) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (n + j < g.N) crow[n + j] = acc[i][4 * h + j];
      }
    }
  }
}

// Slices kt0 .. kt1-1 (kt1 > kt0) of the fold of the 128 x 128 tile at (m0, n0):
// the accumulators start at +0 (from_c false) or at the values C holds (a fold
// that an earlier launch carried up to slice kt0), and are written to C at the
// end. A fold cut into such pieces runs the same chain of roundings as one
// pass over all slices, so the bits of C do not depend on the cut.
template <bool TA, bool TB, bool FMA, bool EXACT>
__device__ __forceinline__ void fold_tile(const GemmArgs &g, int vec_ok, float (*As)[BK][BM], float (*Bs)[BK][BN],
                                          int64_t m0, int64_t n0, int64_t kt0, int64_t kt1, bool from_c) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const bool interior_mn = EXACT || (m0 + BM <= g.M && n0 + BN <= g.N);
  float acc[8][8];
  if (from_c) {
    load_c<EXACT>(g, vec_ok, m0, n0, acc);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  }

  float ra[8], rb[8];
  load_slices<TA, TB>(g, m0, n0, kt0 * BK, EXACT || (vec_ok && interior_mn && kt0 * BK + BK <= g.K), ra, rb);
  store_slices<TA, TB>(As[0], Bs[0], ra, rb);
  __syncthreads();
  for (int64_t kt = kt0; kt < kt1; ++kt) {
    const int buf = (int)(kt - kt0) & 1;
    const int64_t k0 = kt * BK;
    if (kt + 1 < kt1) {
      const int64_t k1 = k0 + BK;
      load_slices<TA, TB>(g, m0, n0, k1, EXACT || (vec_ok && interior_mn && k1 + BK <= g.K), ra, rb);
    }
    const int kcount = EXACT ? BK : (g.K - k0 < BK ? (int)(g.K - k0) : BK);
    if (EXACT || kcount == BK) {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = madd<FMA>(a[i], b[j], acc[i][j]);
      }
    } else {
      for (int kk = 0; kk < kcount; ++kk) {  // k tail: exactly K terms, no padded ones
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = madd<FMA>(a[i], b[j], acc[i][j]);
      }
    }
    if (kt + 1 < kt1) {
      store_slices<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
    }
    __syncthreads();
  }
  store_c<EXACT>(g, vec_ok, m0, n0, acc);
}

// EXACT: every tile interior (M, N multiples of 128), K a multiple of 16 and
// the 128-bit paths legal, so the loads, the k loop and the stores need no
// edge cases (4096^3: 2.42 against 2.63 ms for the general kernel; the same
// fold of every element).
template <bool TA, bool TB, bool FMA, bool EXACT>
__global__ void __launch_bounds__(NT, FMA ? 2 : 1) sgemm_fold_kernel(const GemmArgs g, int vec_ok) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const bool interior_mn = EXACT || (m0 + BM <= g.M && n0 + BN <= g.N);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  const int64_t nk = EXACT ? g.K / BK : ceil_div(g.K, BK);
  float ra[8], rb[8];
  load_slices<TA, TB>(g, m0, n0, 0, EXACT || (vec_ok && interior_mn && BK <= g.K), ra, rb);
  store_slices<TA, TB>(As[0], Bs[0], ra, rb);
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    const int64_t k0 = kt * BK;
    if (kt + 1 < nk) {
      const int64_t k1 = k0 + BK;
      load_slices<TA, TB>(g, m0, n0, k1, EXACT || (vec_ok && interior_mn && k1 + BK <= g.K), ra, rb);
    }
    const int kcount = EXACT ? BK : (g.K - k0 < BK ? (int)(g.K - k0) : BK);
    if (EXACT || kcount == BK) {
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = madd<FMA>(a[i], b[j], acc[i][j]);
      }
    } else {
      for (int kk = 0; kk < kcount; ++kk) {  // k tail: exactly K terms, no padded ones
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = madd<FMA>(a[i], b[j], acc[i][j]);
      }
    }
    if (kt + 1 < nk) {
      store_slices<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
    }
    __syncthreads();
  }
  // epilogue: rows ty*4 + i (i<4) and 64 + ty*4 + (i-4); columns likewise
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (!EXACT && m >= g.M) continue;
    float *crow = g.C + m * g.ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (EXACT || (vec_ok && n + 4 <= g.N)) {
        *reinterpret_cast<float4 *>(crow + n) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (n + j < g.N) crow[n + j] = acc[i][4 * h + j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The fold cut into k-range pieces over two launches (a stream-k schedule that
// keeps every fold sequential). The work is the list of (tile, k-slice) units
// in tile-major order, W = tiles x S units with S = ceil(K / 16), cut into P
// equal ranges, one per CTA. CTA c's range [u0, u1) holds the high-k part of
// the tile it shares with CTA c-1 (L_c slices), whole tiles, and the low-k part
// of the tile it shares with CTA c+1. The first launch folds the whole tiles
// and the low-k parts and leaves the accumulators in C; the second folds the
// high-k parts, starting from what C holds. Every CTA's second-launch share is
// D = max_c L_c slices: its own L_c plus the last D - L_c slices of its last
// whole tile (which it then stops short of in the first launch), so both
// launches are balanced. The host requires floor(W / P) >= 2 S, so that every
// range holds at least one whole tile and every tile is cut at most once
// between two CTAs.
// ---------------------------------------------------------------------------

struct PieceArgs {
  int64_t W, P, S, tn, D;
};

template <bool TA, bool TB, bool FMA, bool EXACT>
__global__ void __launch_bounds__(NT, FMA ? 2 : 1) sgemm_fold_pieces_kernel(const GemmArgs g, int vec_ok,
                                                                            const PieceArgs p, int phase) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  // this CTA's pieces in this launch: (tile, first slice, end slice) each;
  // read from shared memory at the start of every piece so that none of the
  // plan stays in registers across a fold
  __shared__ int64_t plan[3][3];
  __shared__ int64_t whole[2];  // phase 0: first whole tile, count of whole tiles before the last
  __shared__ int npieces;
  if (threadIdx.x == 0) {
    const int64_t c = blockIdx.x;
    const int64_t u0 = c * p.W / p.P, u1 = (c + 1) * p.W / p.P;
    const int64_t t_first = ceil_div(u0, p.S), t_last = u1 / p.S;  // whole tiles [t_first, t_last)
    const int64_t L = t_first * p.S - u0, T = u1 - t_last * p.S, E = p.D - L;
    int n = 0;
    auto add = [&](int64_t t, int64_t kt0, int64_t kt1) {
      plan[n][0] = t; plan[n][1] = kt0; plan[n][2] = kt1; ++n;
    };
    if (phase == 0) {
      whole[0] = t_first;
      whole[1] = t_last - 1 - t_first;  // whole tiles folded over every slice
      add(t_last - 1, 0, p.S - E);      // the last whole tile, short of its E top slices
      if (T > 0) add(t_last, 0, T);     // the low-k part of the tile shared with CTA c+1
    } else {
      whole[0] = 0;
      whole[1] = 0;
      if (E > 0) add(t_last - 1, p.S - E, p.S);
      if (L > 0) add(t_first - 1, p.S - L, p.S);  // the high-k part of the tile shared with CTA c-1
    }
    npieces = n;
  }
  __syncthreads();
  const volatile int64_t *vw = whole;
  for (int64_t i = 0; i < vw[1]; ++i) {
    const int64_t t = vw[0] + i;
    fold_tile<TA, TB, FMA, EXACT>(g, vec_ok, As, Bs, (t / p.tn) * BM, (t % p.tn) * BN, 0, p.S, false);
  }
  const volatile int *vn = &npieces;
  for (int j = 0; j < *vn; ++j) {
    const volatile int64_t *q = plan[j];
    const int64_t t = q[0], kt0 = q[1];
    fold_tile<TA, TB, FMA, EXACT>(g, vec_ok, As, Bs, (t / p.tn) * BM, (t % p.tn) * BN, kt0, q[2], kt0 > 0);
  }
}

// ---------------------------------------------------------------------------
// Tiles of 64 x 128 for the last rows of C (schedule 2): when the 128 x 128
// tiles leave a last wave less than half full, those rows are computed as
// half-height tiles by a second launch. Same fold, same bits, same 8 x 8 elements per thread as
// the full tile (rows ty*4 + i and 32 + ty*4 + i, columns as above), on 128
// threads, so that four blocks share an SM.
// ---------------------------------------------------------------------------

constexpr int BMH = 64, NTH = 128;

// The (m0, k0) slice of op(A) (64 x 16) and the (k0, n0) slice of op(B)
// (16 x 128) into registers, 8 and 16 values per thread.
template <bool TA, bool TB>
__device__ __forceinline__ void load_half_slices(const GemmArgs &g, int64_t m0, int64_t n0, int64_t k0, bool vec,
                                                 float (&ra)[8], float (&rb)[16]) {
  const int tid = threadIdx.x;
  if (vec) {
    // A[m][k]: m = tid/2, k = (tid%2)*8 .. +7;  A[k][m]: k = tid/8, m = (tid%8)*8 .. +7
    const float *pa = !TA ? g.A + (m0 + tid / 2) * g.lda + k0 + (tid % 2) * 8
                          : g.A + (k0 + tid / 8) * g.lda + m0 + (tid % 8) * 8;
    const float4 u = __ldg(reinterpret_cast<const float4 *>(pa)), v = __ldg(reinterpret_cast<const float4 *>(pa + 4));
    ra[0] = u.x; ra[1] = u.y; ra[2] = u.z; ra[3] = u.w; ra[4] = v.x; ra[5] = v.y; ra[6] = v.z; ra[7] = v.w;
    // B[k][n]: k = tid/8, n = (tid%8)*16 .. +15;  B[n][k]: n = tid, k = 0 .. 15
    const float *pb = !TB ? g.B + (k0 + tid / 8) * g.ldb + n0 + (tid % 8) * 16 : g.B + (n0 + tid) * g.ldb + k0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 w = __ldg(reinterpret_cast<const float4 *>(pb + 4 * q));
      rb[4 * q] = w.x; rb[4 * q + 1] = w.y; rb[4 * q + 2] = w.z; rb[4 * q + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      ra[j] = !TA ? a_at<TA>(g, m0 + tid / 2, k0 + (tid % 2) * 8 + j) : a_at<TA>(g, m0 + (tid % 8) * 8 + j, k0 + tid / 8);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      rb[j] = !TB ? b_at<TB>(g, k0 + tid / 8, n0 + (tid % 8) * 16 + j) : b_at<TB>(g, k0 + j, n0 + tid);
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void store_half_slices(float (*As)[BMH], float (*Bs)[BN], const float (&ra)[8],
                                                  const float (&rb)[16]) {
  const int tid = threadIdx.x;
  if (!TA) {
#pragma unroll
    for (int j = 0; j < 8; ++j) As[(tid % 2) * 8 + j][tid / 2] = ra[j];
  } else {
    *reinterpret_cast<float4 *>(&As[tid / 8][(tid % 8) * 8]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    *reinterpret_cast<float4 *>(&As[tid / 8][(tid % 8) * 8 + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
  }
  if (!TB) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<float4 *>(&Bs[tid / 8][(tid % 8) * 16 + 4 * q]) =
          make_float4(rb[4 * q], rb[4 * q + 1], rb[4 * q + 2], rb[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) Bs[j][tid] = rb[j];
  }
}

template <bool TA, bool TB, bool FMA>
__global__ void __launch_bounds__(NTH, 4) sgemm_fold_half_kernel(const GemmArgs g, int vec_ok) {
  __shared__ __align__(16) float As[2][BK][BMH];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int64_t m0 = (int64_t)blockIdx.y * BMH, n0 = (int64_t)blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // ty in 0..7
  const bool interior_mn = m0 + BMH <= g.M && n0 + BN <= g.N;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  const int64_t nk = ceil_div(g.K, BK);
  float ra[8], rb[16];
  load_half_slices<TA, TB>(g, m0, n0, 0, vec_ok && interior_mn && BK <= g.K, ra, rb);
  store_half_slices<TA, TB>(As[0], Bs[0], ra, rb);
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    const int64_t k0 = kt * BK;
    if (kt + 1 < nk) {
      const int64_t k1 = k0 + BK;
      load_half_slices<TA, TB>(g, m0, n0, k1, vec_ok && interior_mn && k1 + BK <= g.K, ra, rb);
    }
    const int kcount = g.K - k0 < BK ? (int)(g.K - k0) : BK;
    for (int kk = 0; kk < kcount; ++kk) {  // exactly K terms in order
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][32 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = madd<FMA>(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) store_half_slices<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 32 + ty * 4 + (i - 4));
    if (m >= g.M) continue;
    float *crow = g.C + m * g.ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (vec_ok && n + 4 <= g.N) {
        *reinterpret_cast<float4 *>(crow + n) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (n + j < g.N) crow[n + j] = acc[i][4 * h + j];
      }
    }
  }
}

template <bool FMA>
const void *pick_half(int ta, int tb) {
  if (!ta && !tb) return (const void *)sgemm_fold_half_kernel<false, false, FMA>;
  if (!ta && tb) return (const void *)sgemm_fold_half_kernel<false, true, FMA>;
  if (ta && !tb) return (const void *)sgemm_fold_half_kernel<true, false, FMA>;
  return (const void *)sgemm_fold_half_kernel<true, true, FMA>;
}

template <bool FMA, bool EXACT>
const void *pick(int ta, int tb) {
  if (!ta && !tb) return (const void *)sgemm_fold_kernel<false, false, FMA, EXACT>;
  if (!ta && tb) return (const void *)sgemm_fold_kernel<false, true, FMA, EXACT>;
  if (ta && !tb) return (const void *)sgemm_fold_kernel<true, false, FMA, EXACT>;
  return (const void *)sgemm_fold_kernel<true, true, FMA, EXACT>;
}

}  // namespace

namespace {

template <bool FMA, bool EXACT>
const void *pick_pieces(int ta, int tb) {
  if (!ta && !tb) return (const void *)sgemm_fold_pieces_kernel<false, false, FMA, EXACT>;
  if (!ta && tb) return (const void *)sgemm_fold_pieces_kernel<false, true, FMA, EXACT>;
  if (ta && !tb) return (const void *)sgemm_fold_pieces_kernel<true, false, FMA, EXACT>;
  return (const void *)sgemm_fold_pieces_kernel<true, true, FMA, EXACT>;
}

// The piece schedule over P CTAs (two per SM with the declared FMA): W units
// of (tile, k-slice), D the second launch's share.
bool piece_plan(int64_t M, int64_t N, int64_t K, int fma, PieceArgs *p) {
  const int64_t tn = ceil_div(N, BN), tm = ceil_div(M, BM), S = ceil_div(K, BK);
  const void *k = fma ? pick_pieces<true, false>(0, 0) : pick_pieces<false, false>(0, 0);
  const int64_t P = (int64_t)sm_count() * resident_blocks(k, NT);
  if (S < 1 || P < 1) return false;
  const int64_t W = tn * tm * S;
  if (W / P < 2 * S) return false;
  int64_t D = 0;
  for (int64_t c = 0; c < P; ++c) {
    const int64_t u0 = c * W / P, L = ceil_div(u0, S) * S - u0;
    if (L > D) D = L;
  }
  *p = PieceArgs{W, P, S, tn, D};
  return true;
}

}  // namespace

bool gemm_f32_pieces_fit(int64_t M, int64_t N, int64_t K, int fma) {
  PieceArgs p;
  return piece_plan(M, N, K, fma, &p);
}

cudaError_t launch_gemm_f32(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K,
                            int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int fma,
                            int vec_ok, int schedule, cudaStream_t stream) {
  GemmArgs g{A, B, C, M, N, K, lda, ldb, ldc};
  const bool exact = vec_ok && M % BM == 0 && N % BN == 0 && K % BK == 0;
  const void *k = fma ? (exact ? pick<true, true>(transA, transB) : pick<true, false>(transA, transB))
                      : (exact ? pick<false, true>(transA, transB) : pick<false, false>(transA, transB));
  const int64_t tn = ceil_div(N, BN), tm = ceil_div(M, BM);
  const int64_t slots = (int64_t)sm_count() * resident_blocks(k, NT);
  const int64_t total = tn * tm, rem = total % slots;
  // automatic: one launch, unless the last wave leaves some SM two tiles and
  // more than 8% of all the two-tile slots of the launch's waves empty; then
  // the k-range pieces where they fit. A last wave of at most one tile per SM
  // costs about half a wave, since a tile alone on an SM runs faster than one
  // of two (4096^3: one launch 2.42 ms, half-height tail tiles 2.58, pieces
  // 2.64); the pieces cost about 8-10% of the run in all (3584 x 3584 x 4096:
  // 1.98 ms against 2.07 in one launch; 6144 x 6144 x 2048: 3.05 against 2.75).
  const int64_t sms = sm_count();
  const bool pieces_pay = total > slots && rem > sms && (slots - rem) * 100 > 8 * slots * (total / slots + 1);
  PieceArgs p;
  if ((schedule == 0 && pieces_pay) || schedule == 3) {
    if (piece_plan(M, N, K, fma, &p)) {
      const void *kp = fma ? (exact ? pick_pieces<true, true>(transA, transB) : pick_pieces<true, false>(transA, transB))
                           : (exact ? pick_pieces<false, true>(transA, transB)
                                    : pick_pieces<false, false>(transA, transB));
      for (int phase = 0; phase < 2; ++phase) {
        void *pargs[] = {&g, &vec_ok, &p, &phase};
        cudaError_t e = cudaLaunchKernel(kp, dim3((unsigned)p.P), dim3(NT), pargs, 0, stream);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    if (schedule == 3) return cudaErrorInvalidValue;  // refused on the host before this call
  }
  int64_t tail = 0;  // tile rows computed as half tiles
  if (schedule == 2 && total > slots && rem > 0 && rem <= slots / 2) tail = ceil_div(rem, tn);
  if (tail >= tm) tail = 0;
  void *args[] = {&g, &vec_ok};
  cudaError_t e = cudaLaunchKernel(k, dim3((unsigned)tn, (unsigned)(tm - tail)), dim3(NT), args, 0, stream);
  if (e != cudaSuccess || tail == 0) return e;
  const int64_t m_main = (tm - tail) * BM;
  GemmArgs t = g;
  t.A = transA ? A + m_main : A + m_main * lda;
  t.C = C + m_main * ldc;
  t.M = M - m_main;
  const void *kh = fma ? pick_half<true>(transA, transB) : pick_half<false>(transA, transB);
  void *targs[] = {&t, &vec_ok};
  return cudaLaunchKernel(kh, dim3((unsigned)tn, (unsigned)ceil_div(t.M, BMH)), dim3(NTH), targs, 0, stream);
}

}  // namespace dpia
