// Pure maps: scal (map (a*)), the dot adjoint (two pointwise products with a
// broadcast gradient) and GEMV's dA = dy x^T (a map of maps). Each is a
// parallel map over asVector-V elements (Section 6.2), grid-stride over a
// persistent grid, 128-bit loads and streaming 128-bit stores.
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

int resident_blocks(const void *kernel, int threads);

namespace {

template <int V>
__device__ __forceinline__ void store_vec(float *p, const float (&r)[V]) {
  if constexpr (V == 1) {
    p[0] = r[0];
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(r[0], r[1]);
  } else {
#pragma unroll
    for (int q = 0; q < V / 4; ++q)
      st_stream_v4(p + 4 * q, make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]));
  }
}

// y[i] = a * x[i]; vectors of V, scalar tail.
template <int V>
__global__ void __launch_bounds__(256) scal_kernel(float a, const float *x, float *y, int64_t n) {
  const int64_t nv = n / V;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x;
  constexpr int U = Unroll<V, 2>::value > 4 ? 4 : Unroll<V, 2>::value;
  int64_t i = g0;
  for (; i + (U - 1) * ng < nv; i += U * ng) {
    float r[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u) load_vec<V, false>(x + (i + u * ng) * V, r[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int v = 0; v < V; ++v) r[u][v] = __fmul_rn(a, r[u][v]);
      store_vec<V>(y + (i + u * ng) * V, r[u]);
    }
  }
  for (; i < nv; i += ng) {
    float r[V];
    load_vec<V, false>(x + i * V, r);
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = __fmul_rn(a, r[v]);
    store_vec<V>(y + i * V, r);
  }
  for (int64_t e = nv * V + g0; e < n; e += ng) y[e] = __fmul_rn(a, x[e]);
}

// The same map over contiguous chunks of 256 * U vectors: a block takes chunks
// blockIdx.x, + gridDim.x, ...; in a chunk thread t loads vectors t, t + 256, ...
// (all U loads in flight before the stores), so each block streams one
// contiguous 32 KiB (V = 4, U = 8) piece at a time. A ragged end is left to
// the grid-stride kernel's tail loops (vectors, then scalars).
template <int V, int U>
__global__ void __launch_bounds__(256) scal_chunk_kernel(float a, const float *x, float *y, int64_t n) {
  const int64_t nv = n / V;
  const int64_t chunks = nv / (256 * U);
  for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int64_t base = c * (256 * U) + threadIdx.x;
    float r[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u) load_vec<V, false>(x + (base + u * 256) * V, r[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int v = 0; v < V; ++v) r[u][v] = __fmul_rn(a, r[u][v]);
      store_vec<V>(y + (base + u * 256) * V, r[u]);
    }
  }
  // the vectors past the last whole chunk, then the scalar tail
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = chunks * (256 * U) + g0; i < nv; i += ng) {
    float r[V];
    load_vec<V, false>(x + i * V, r);
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = __fmul_rn(a, r[v]);
    store_vec<V>(y + i * V, r);
  }
  for (int64_t e = nv * V + g0; e < n; e += ng) y[e] = __fmul_rn(a, x[e]);
}

// dx = g*y, dy = g*x with g read from device memory.
__global__ void __launch_bounds__(256) dot_bwd_kernel(const float *x, const float *y, const float *g,
                                                      int64_t n, float *dx, float *dy) {
  const float gv = __ldg(g);
  const int64_t nv = n / 4;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ng = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = g0; i < nv; i += ng) {
    if (dx) {
      float4 b = ld_stream_v4(y + 4 * i);
      st_stream_v4(dx + 4 * i, make_float4(__fmul_rn(gv, b.x), __fmul_rn(gv, b.y), __fmul_rn(gv, b.z),
                                           __fmul_rn(gv, b.w)));
    }
    if (dy) {
      float4 a = ld_stream_v4(x + 4 * i);
      st_stream_v4(dy + 4 * i, make_float4(__fmul_rn(gv, a.x), __fmul_rn(gv, a.y), __fmul_rn(gv, a.z),
                                           __fmul_rn(gv, a.w)));
    }
  }
  for (int64_t e = nv * 4 + g0; e < n; e += ng) {
    if (dx) dx[e] = __fmul_rn(gv, y[e]);
    if (dy) dy[e] = __fmul_rn(gv, x[e]);
  }
}

// dA[i][j] = dy[i] * x[j]: one block per row (grid-stride), x from L1/L2.
__global__ void __launch_bounds__(256) outer_kernel(const float *x, const float *dy, int64_t M,
                                                    int64_t N, float *dA, int64_t ldda, int vec) {
  const int64_t nv = vec ? N / 4 : 0;
  for (int64_t i = blockIdx.x; i < M; i += gridDim.x) {
    const float d = __ldg(dy + i);
    float *row = dA + i * ldda;
    for (int64_t j = threadIdx.x; j < nv; j += blockDim.x) {
      float4 xv = ld_cached_v4(x + 4 * j);
      st_stream_v4(row + 4 * j, make_float4(__fmul_rn(d, xv.x), __fmul_rn(d, xv.y),
                                            __fmul_rn(d, xv.z), __fmul_rn(d, xv.w)));
    }
    for (int64_t j = nv * 4 + threadIdx.x; j < N; j += blockDim.x) row[j] = __fmul_rn(d, __ldg(x + j));
  }
}

int64_t persistent_grid(const void *k, int threads, int64_t work_threads) {
  int64_t cap = (int64_t)sm_count() * resident_blocks(k, threads);
  int64_t need = ceil_div(work_threads, threads);
  int64_t g = need < cap ? need : cap;
  return g < 1 ? 1 : g;
}

}  // namespace

cudaError_t launch_scal(float a, const float *x, float *y, int64_t n, int V, cudaStream_t stream) {
  const void *k = nullptr;
  switch (V) {
    case 1: k = (const void *)scal_kernel<1>; break;
    case 2: k = (const void *)scal_kernel<2>; break;
    case 4: k = (const void *)scal_chunk_kernel<4, 8>; break;
    case 8: k = (const void *)scal_kernel<8>; break;
    case 16: k = (const void *)scal_kernel<16>; break;
    default: return cudaErrorInvalidValue;
  }
  const int threads = 256;
  int64_t grid = persistent_grid(k, threads, ceil_div(n, V));
  void *args[] = {&a, &x, &y, &n};
  return cudaLaunchKernel(k, dim3((unsigned)grid), dim3(threads), args, 0, stream);
}

cudaError_t launch_dot_bwd(const float *x, const float *y, const float *g, int64_t n, float *dx,
                           float *dy, cudaStream_t stream) {
  const int threads = 256;
  int64_t grid = persistent_grid((const void *)dot_bwd_kernel, threads, ceil_div(n, 4));
  dot_bwd_kernel<<<(unsigned)grid, threads, 0, stream>>>(x, y, g, n, dx, dy);
  return cudaGetLastError();
}

cudaError_t launch_outer(const float *x, const float *dy, int64_t M, int64_t N, float *dA,
                         int64_t ldda, int vec, cudaStream_t stream) {
  const int threads = 256;
  int64_t cap = (int64_t)sm_count() * resident_blocks((const void *)outer_kernel, threads);
  int64_t grid = M < cap ? M : cap;
  if (grid < 1) grid = 1;
  outer_kernel<<<(unsigned)grid, threads, 0, stream>>>(x, dy, M, N, dA, ldda, vec);
  return cudaGetLastError();
}

}  // namespace dpia
