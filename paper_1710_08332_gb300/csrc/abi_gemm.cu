// C ABI of the GEMM instances (FP32 fold, BF16 tensor cores), the bf16 cast
// and the device status poll. Validation happens on the host before launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/dpia.h"
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {
cudaError_t launch_gemm_f32(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K,
                            int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int fma, int vec_ok,
                            int schedule, cudaStream_t stream);
bool gemm_f32_pieces_fit(int64_t M, int64_t N, int64_t K, int fma);
cudaError_t launch_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int64_t M, int64_t N, int64_t K,
                             int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int grid, int tile_m,
                             int tile_n, int cluster, int vec_ok, cudaStream_t stream);
cudaError_t poll_device_status(unsigned *out);
cudaError_t launch_bounded_wait_probe(uint64_t timeout_ns, cudaStream_t stream);
int resident_blocks(const void *kernel, int threads);
}  // namespace dpia

using namespace dpia;

namespace {

bool aligned(const void *p, int64_t a) { return (reinterpret_cast<uintptr_t>(p) % (uintptr_t)a) == 0; }

bool overlap(const void *a, int64_t na, const void *b, int64_t nb) {
  if (!a || !b || na <= 0 || nb <= 0) return false;
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + (uintptr_t)nb && y < x + (uintptr_t)na;
}

// bytes spanned by a row-major rows x cols matrix with leading dimension ld
int64_t span(int64_t rows, int64_t cols, int64_t ld, int64_t esize) {
  return rows > 0 && cols > 0 ? ((rows - 1) * ld + cols) * esize : 0;
}

dpia_status cuda_status(cudaError_t e, const char *fn) {
  if (e == cudaSuccess) return DPIA_OK;
  set_last_error("%s: CUDA error %d (%s)", fn, (int)e, cudaGetErrorString(e));
  return DPIA_ERR_CUDA;
}

// Shared checks of the two GEMMs; op(A) is M x K, op(B) is K x N.
dpia_status check_gemm(const char *fn, const void *A, const void *B, const float *C, int64_t M, int64_t N,
                       int64_t K, int64_t lda, int64_t ldb, int64_t ldc, int transA, int transB, int64_t esize,
                       int64_t *abytes, int64_t *bbytes) {
  if (M < 0 || N < 0 || K < 0) {
    set_last_error("%s: negative shape", fn);
    return DPIA_ERR_SHAPE;
  }
  if ((transA != 0 && transA != 1) || (transB != 0 && transB != 1)) {
    set_last_error("%s: transA/transB must be 0 or 1", fn);
    return DPIA_ERR_SHAPE;
  }
  const int64_t a_rows = transA ? K : M, a_cols = transA ? M : K;
  const int64_t b_rows = transB ? N : K, b_cols = transB ? K : N;
  if (lda < (a_cols > 1 ? a_cols : 1) || ldb < (b_cols > 1 ? b_cols : 1) || ldc < (N > 1 ? N : 1)) {
    set_last_error("%s: leading dimension smaller than the stored row length", fn);
    return DPIA_ERR_SHAPE;
  }
  if (M == 0 || N == 0) return DPIA_OK;
  if (!C || (K > 0 && (!A || !B))) {
    set_last_error("%s: NULL matrix", fn);
    return DPIA_ERR_NULL;
  }
  *abytes = span(a_rows, a_cols, lda, esize);
  *bbytes = span(b_rows, b_cols, ldb, esize);
  const int64_t cbytes = span(M, N, ldc, 4);
  if (overlap(C, cbytes, A, *abytes) || overlap(C, cbytes, B, *bbytes)) {
    set_last_error("%s: C overlaps A or B", fn);
    return DPIA_ERR_ALIAS;
  }
  if (!aligned(C, 4)) {
    set_last_error("%s: C must be 4-byte aligned", fn);
    return DPIA_ERR_ALIGN;
  }
  return DPIA_OK;
}

__global__ void cast_bf16_kernel(const float *x, uint16_t *y, int64_t n) {
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x;
  const int64_t nv = n / 4;
  for (int64_t i = g0; i < nv; i += ng) {
    float4 v = ld_stream_v4(x + 4 * i);
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t *>(&lo);
    o.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(y + 4 * i) = o;
  }
  for (int64_t e = nv * 4 + g0; e < n; e += ng) {
    __nv_bfloat16 b = __float2bfloat16_rn(x[e]);
    y[e] = *reinterpret_cast<uint16_t *>(&b);
  }
}

}  // namespace

extern "C" {

dpia_status dpia_gemm_f32(const float *A, const float *B, float *C, int64_t M, int64_t N, int64_t K, int64_t lda,
                          int64_t ldb, int64_t ldc, int32_t transA, int32_t transB, const dpia_gemm_strategy *st,
                          dpia_stream_t stream) {
  const char *fn = "dpia_gemm_f32";
  set_last_error("");
  if (!st) {
    set_last_error("%s: strategy is NULL", fn);
    return DPIA_ERR_NULL;
  }
  if (st->contract != DPIA_CONTRACT_OFF && st->contract != DPIA_CONTRACT_FMA) {
    set_last_error("%s: contract=%d", fn, st->contract);
    return DPIA_ERR_STRATEGY;
  }
  if ((st->tile_m && st->tile_m != 128) || (st->tile_n && st->tile_n != 128) || (st->tile_k && st->tile_k != 16)) {
    set_last_error("%s: only 128 x 128 x 16 tiles are implemented for the FP32 fold", fn);
    return DPIA_ERR_UNSUPPORTED;
  }
  if (st->schedule < 0 || st->schedule > 3) {
    set_last_error("%s: schedule=%d (0 automatic, 1 tiles, 2 half-height tail tiles, 3 k-range pieces)", fn,
                   st->schedule);
    return DPIA_ERR_STRATEGY;
  }
  int64_t ab = 0, bb = 0;
  dpia_status rc = check_gemm(fn, A, B, C, M, N, K, lda, ldb, ldc, transA, transB, 4, &ab, &bb);
  if (rc || M == 0 || N == 0) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (K == 0) return cuda_status(cudaMemset2DAsync(C, ldc * 4, 0, N * 4, M, s), fn);
  if (st->schedule == 3 && !gemm_f32_pieces_fit(M, N, K, st->contract)) {
    set_last_error("%s: schedule 3 needs at least two tiles' k-slices per CTA of the device", fn);
    return DPIA_ERR_STRATEGY;
  }
  if (!aligned(A, 4) || !aligned(B, 4)) {
    set_last_error("%s: A and B must be 4-byte aligned", fn);
    return DPIA_ERR_ALIGN;
  }
  const int vec_ok = aligned(A, 16) && aligned(B, 16) && aligned(C, 16) && lda % 4 == 0 && ldb % 4 == 0 &&
                     ldc % 4 == 0;
  return cuda_status(
      launch_gemm_f32(A, B, C, M, N, K, lda, ldb, ldc, transA, transB, st->contract, vec_ok, st->schedule, s), fn);
}

dpia_status dpia_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int64_t M, int64_t N, int64_t K,
                           int64_t lda, int64_t ldb, int64_t ldc, int32_t transA, int32_t transB,
                           const dpia_gemm_strategy *st, dpia_stream_t stream) {
  const char *fn = "dpia_gemm_bf16";
  set_last_error("");
  if (!st) {
    set_last_error("%s: strategy is NULL", fn);
    return DPIA_ERR_NULL;
  }
  if ((st->tile_m && st->tile_m != 256 && !(st->tile_m == 512 && st->cluster == 2)) ||
      (st->tile_k && st->tile_k != 64) ||
      (st->tile_n && (st->tile_n < 128 || st->tile_n > 256 || st->tile_n % 32 != 0))) {
    set_last_error("%s: tiles are tile_m x tile_n x 64 with tile_m 256 (512 on a CTA pair, cluster = 2) and "
                   "tile_n in {128, 160, ..., 256} (0 = chosen per shape)", fn);
    return DPIA_ERR_UNSUPPORTED;
  }
  if (st->grid < 0) {
    set_last_error("%s: grid=%d", fn, st->grid);
    return DPIA_ERR_STRATEGY;
  }
  if (st->cluster != 0 && st->cluster != 1 && st->cluster != 2) {
    set_last_error("%s: cluster=%d (0 = chosen per shape, 1 = one CTA per tile, 2 = a CTA pair)", fn, st->cluster);
    return DPIA_ERR_STRATEGY;
  }
  int64_t ab = 0, bb = 0;
  dpia_status rc = check_gemm(fn, A, B, C, M, N, K, lda, ldb, ldc, transA, transB, 2, &ab, &bb);
  if (rc || M == 0 || N == 0) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (K == 0) return cuda_status(cudaMemset2DAsync(C, ldc * 4, 0, N * 4, M, s), fn);
  if (!aligned(A, 16) || !aligned(B, 16) || lda % 8 != 0 || ldb % 8 != 0) {
    set_last_error("%s: A and B must be 16-byte aligned with leading dimensions a multiple of 8 (TMA)", fn);
    return DPIA_ERR_ALIGN;
  }
  if (M > 0x7fffffff || N > 0x7fffffff || K > 0x7fffffff) {
    set_last_error("%s: dimensions beyond 2^31-1", fn);
    return DPIA_ERR_SHAPE;
  }
  const int vec_ok = aligned(C, 16) && ldc % 4 == 0;
  return cuda_status(
      launch_gemm_bf16(A, B, C, M, N, K, lda, ldb, ldc, transA, transB, st->grid, st->tile_m, st->tile_n,
                       st->cluster, vec_ok, s),
      fn);
}

dpia_status dpia_cast_f32_bf16(const float *x, uint16_t *y, int64_t n, dpia_stream_t stream) {
  const char *fn = "dpia_cast_f32_bf16";
  set_last_error("");
  if (n < 0) {
    set_last_error("%s: negative length", fn);
    return DPIA_ERR_SHAPE;
  }
  if (n == 0) return DPIA_OK;
  if (!x || !y) {
    set_last_error("%s: NULL pointer", fn);
    return DPIA_ERR_NULL;
  }
  if (!aligned(x, 16) || !aligned(y, 8)) {
    set_last_error("%s: x must be 16-byte and y 8-byte aligned", fn);
    return DPIA_ERR_ALIGN;
  }
  if (overlap(x, n * 4, y, n * 2)) {
    set_last_error("%s: y overlaps x", fn);
    return DPIA_ERR_ALIAS;
  }
  const int threads = 256;
  int64_t cap = (int64_t)sm_count() * resident_blocks((const void *)cast_bf16_kernel, threads);
  int64_t need = ceil_div(ceil_div(n, 4), threads);
  int64_t grid = need < cap ? need : cap;
  cast_bf16_kernel<<<(unsigned)(grid < 1 ? 1 : grid), threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, y, n);
  return cuda_status(cudaGetLastError(), fn);
}

dpia_status dpia_selftest_bounded_wait(uint32_t timeout_us, dpia_stream_t stream) {
  set_last_error("");
  if (timeout_us < 1 || timeout_us > 2000000u) {
    set_last_error("dpia_selftest_bounded_wait: timeout_us=%u outside 1 .. 2000000", timeout_us);
    return DPIA_ERR_SHAPE;
  }
  cudaError_t e = launch_bounded_wait_probe((uint64_t)timeout_us * 1000ull, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "dpia_selftest_bounded_wait");
  return DPIA_OK;
}

dpia_status dpia_poll_device_status(int32_t *status) {
  set_last_error("");
  if (!status) {
    set_last_error("dpia_poll_device_status: status is NULL");
    return DPIA_ERR_NULL;
  }
  unsigned v = 0;
  cudaError_t e = poll_device_status(&v);
  if (e != cudaSuccess) return cuda_status(e, "dpia_poll_device_status");
  *status = (int32_t)v;
  return DPIA_OK;
}

}  // extern "C"
