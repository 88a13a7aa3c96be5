// GEMV forward and the dx half of its backward.
//
// Forward: y = map (lambda row. R (zip row x)) A. The map over rows runs at
// block level (a block per row, grid-stride) or warp level (a warp per row);
// the row reduce is the strategy reduction of k_reduce.cu restricted to one
// unit: the row is split into chunks of s, each chunk folded by the unit's
// threads and reduced by the halving tree, and the chunk results are folded in
// chunk order by the unit's first thread. A is streamed once; x is re-read by
// every row and stays in L1/L2.
//
// Backward dx = A^T dy: a map over columns of a split-over-rows fold. Block
// (tile, chunk) owns 4*blockDim consecutive columns (4 per thread) and Rs rows;
// each thread folds its four columns down the chunk's rows in row order (8 rows
// of loads in flight), and
// writes the four chunk partials. The last block of each column tile (ticket,
// no waiting) folds the tile's partials in chunk order into dx.
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

int resident_blocks(const void *kernel, int threads);

namespace {

template <class A, int V, int LEVEL>
__global__ void __launch_bounds__(max_threads_for_vec(V)) gemv_kernel(const GemvLaunch p) {
  using acc_t = typename A::acc_t;
  __shared__ acc_t sm[32];
  if constexpr (LEVEL == int(ChunkLevel::Block)) {
    const int t = threadIdx.x;
    for (int64_t i = blockIdx.x; i < p.M; i += gridDim.x) {
      const float *row = p.A + i * p.lda;
      acc_t acc = A::zero();
      for (int64_t c = 0; c < p.Crow; ++c) {
        const bool full = (c + 1) * p.s <= p.N;
        acc_t v = thread_fold<DotF32, A, V, true>(row, p.x, p.N, c * p.s + t * p.tstride, p.Rc,
                                                   p.step, full);
        v = block_tree<A>(v, p.Tc, sm);
        if (t == 0) acc = A::combine(acc, v);
      }
      if (t == 0) p.y[i] = A::result(acc);
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t w0 = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t nw = gridDim.x * wpb;
    for (int64_t i = w0; i < p.M; i += nw) {
      const float *row = p.A + i * p.lda;
      acc_t acc = A::zero();
      for (int64_t c = 0; c < p.Crow; ++c) {
        const bool full = (c + 1) * p.s <= p.N;
        acc_t v = thread_fold<DotF32, A, V, true, 2, true>(row, p.x, p.N, c * p.s + lane * p.tstride, p.Rc,
                                                            p.step, full);
        v = warp_tree<A>(v, 32);
        if (lane == 0) acc = A::combine(acc, v);
      }
      if (lane == 0) p.y[i] = A::result(acc);
    }
  }
}

template <class A, int LEVEL>
const void *gemv_pick_v(int V) {
  switch (V) {
    case 1: return (const void *)gemv_kernel<A, 1, LEVEL>;
    case 2: return (const void *)gemv_kernel<A, 2, LEVEL>;
    case 4: return (const void *)gemv_kernel<A, 4, LEVEL>;
    case 8: return (const void *)gemv_kernel<A, 8, LEVEL>;
    case 16: return (const void *)gemv_kernel<A, 16, LEVEL>;
  }
  return nullptr;
}

constexpr int kBwdThreads = 256;  // 1024 columns per tile
constexpr int kDxRows = 8;        // rows of 128-bit loads in flight per thread

__global__ void __launch_bounds__(kBwdThreads) gemv_bwd_dx_kernel(const GemvBwdLaunch p) {
  __shared__ int is_last;
  const int64_t tile = blockIdx.x;
  const int64_t chunk = blockIdx.y;
  const int64_t j0 = tile * (4 * kBwdThreads) + 4 * threadIdx.x;
  const int64_t r0 = chunk * p.Rs;
  const int64_t r1 = r0 + p.Rs < p.M ? r0 + p.Rs : p.M;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (p.vec && j0 + 4 <= p.N) {
    int64_t i = r0;
    for (; i + kDxRows <= r1; i += kDxRows) {
      float4 a[kDxRows];
      float d[kDxRows];
#pragma unroll
      for (int u = 0; u < kDxRows; ++u) {
        a[u] = ld_stream_v4(p.A + (i + u) * p.lda + j0);
        d[u] = __ldg(p.dy + i + u);
      }
#pragma unroll
      for (int u = 0; u < kDxRows; ++u) {
        acc[0] = __fadd_rn(acc[0], __fmul_rn(a[u].x, d[u]));
        acc[1] = __fadd_rn(acc[1], __fmul_rn(a[u].y, d[u]));
        acc[2] = __fadd_rn(acc[2], __fmul_rn(a[u].z, d[u]));
        acc[3] = __fadd_rn(acc[3], __fmul_rn(a[u].w, d[u]));
      }
    }
    for (; i < r1; ++i) {
      float4 a = ld_stream_v4(p.A + i * p.lda + j0);
      float d = __ldg(p.dy + i);
      acc[0] = __fadd_rn(acc[0], __fmul_rn(a.x, d));
      acc[1] = __fadd_rn(acc[1], __fmul_rn(a.y, d));
      acc[2] = __fadd_rn(acc[2], __fmul_rn(a.z, d));
      acc[3] = __fadd_rn(acc[3], __fmul_rn(a.w, d));
    }
  } else if (j0 < p.N) {  // ragged last columns, or a leading dimension not fit for 128-bit loads
    for (int64_t i = r0; i < r1; ++i) {
      const float d = __ldg(p.dy + i);
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (j0 + v < p.N) acc[v] = __fadd_rn(acc[v], __fmul_rn(p.A[i * p.lda + j0 + v], d));
    }
  }
  float *part = p.partials + chunk * p.Npad;
  if (j0 < p.N) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (j0 + v < p.N) part[j0 + v] = acc[v];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(p.counters + tile, 1u);
    __threadfence();
    is_last = (ticket == gridDim.y - 1);
  }
  __syncthreads();
  if (!is_last) return;
  // fold the tile's partials over the row chunks in chunk order from zero;
  // loads run 8 chunks ahead of the dependent adds
  float res[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (j0 < p.N) {
    const bool full4 = j0 + 4 <= p.N;
    int64_t c = 0;
    for (; c + 8 <= p.Cr; c += 8) {
      float4 b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float *pc = p.partials + (c + u) * p.Npad + j0;
        b[u] = full4 ? __ldcg(reinterpret_cast<const float4 *>(pc))
                     : make_float4(__ldcg(pc), j0 + 1 < p.N ? __ldcg(pc + 1) : 0.0f,
                                   j0 + 2 < p.N ? __ldcg(pc + 2) : 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        res[0] = __fadd_rn(res[0], b[u].x);
        res[1] = __fadd_rn(res[1], b[u].y);
        res[2] = __fadd_rn(res[2], b[u].z);
        res[3] = __fadd_rn(res[3], b[u].w);
      }
    }
    for (; c < p.Cr; ++c) {
      const float *pc = p.partials + c * p.Npad;
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (j0 + v < p.N) res[v] = __fadd_rn(res[v], __ldcg(pc + j0 + v));
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v)
    if (j0 + v < p.N) p.dx[j0 + v] = res[v];
  if (threadIdx.x == 0) p.counters[tile] = 0u;
}

}  // namespace

cudaError_t launch_gemv(bool compensated, int V, ChunkLevel level, int threads, int grid,
                        const GemvLaunch &p, cudaStream_t stream) {
  const void *k = nullptr;
  if (level == ChunkLevel::Block)
    k = compensated ? gemv_pick_v<KahanF32, 1>(V) : gemv_pick_v<SumF32, 1>(V);
  else if (level == ChunkLevel::Warp)
    k = compensated ? gemv_pick_v<KahanF32, 2>(V) : gemv_pick_v<SumF32, 2>(V);
  if (!k) return cudaErrorInvalidValue;
  const int64_t units_per_block = level == ChunkLevel::Block ? 1 : threads / 32;
  if (grid <= 0) {
    int64_t cap = (int64_t)sm_count() * resident_blocks(k, threads);
    int64_t need = ceil_div(p.M, units_per_block);
    grid = (int)(need < cap ? need : cap);
    if (grid < 1) grid = 1;
  }
  void *args[] = {const_cast<GemvLaunch *>(&p)};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, stream);
}

cudaError_t launch_gemv_bwd_dx(const GemvBwdLaunch &p, cudaStream_t stream) {
  const int64_t tiles = ceil_div(p.N, 4 * kBwdThreads);
  if (p.Cr > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)tiles, (unsigned)p.Cr);
  gemv_bwd_dx_kernel<<<grid, kBwdThreads, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace dpia
