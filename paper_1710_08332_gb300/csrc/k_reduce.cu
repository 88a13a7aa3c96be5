// Strategy reduction kernel: dot (f32, int32) and asum.
//
// The split input is mapped chunk by chunk onto the GPU hierarchy the strategy
// names (Section 6.2's mapWorkgroup / mapLocal / mapGlobal levels, with the
// warp as the extra sm_103a level):
//   BLOCK: chunk c -> block (c mod gridDim), Tc = blockDim threads;
//   WARP : chunk c -> warp  (c mod #warps),   Tc = 32 lanes;
//   GRID : chunk c -> thread(c mod #threads), Tc = 1 (a sequential fold).
// Each thread folds its column of the chunk (thread_fold), the Tc results are
// reduced by the halving tree, and the chunk result goes to partials[c] -- the
// hoisted global temporary of Section 6.4. The second-level reduce over the C
// partials runs in the last block to finish: every block fences its partials
// and takes a ticket; the block that draws the last ticket reduces them. No
// block ever waits for another.
#include <type_traits>

#include "../../include/dpia.h"
#include "async_copy.cuh"
#include "device_common.cuh"
#include "kernels.h"

namespace dpia {

namespace {

// Partials written by other blocks are read from L2 (never a stale L1 line).
template <class A>
__device__ __forceinline__ typename A::acc_t load_partial(const typename A::acc_t *p, int64_t i) {
  return __ldcg(p + i);
}

// Partials staged per tile of the sequential second level.
constexpr int kSeqTile = 2048;

// Second level over the C chunk partials, run by the last block.
template <class A>
__device__ void second_level(const ReduceLaunch &p, typename A::acc_t *sm, typename A::acc_t *stage) {
  using acc_t = typename A::acc_t;
  const acc_t *part = static_cast<const acc_t *>(p.partials);
  acc_t res = A::zero();
  if (!p.second_tree) {
    // left fold in chunk order from zero (the final sequential loop): the
    // block stages a tile of partials in shared memory with one parallel load,
    // then thread 0 folds the tile in order
    acc_t acc = A::zero();
    for (int64_t k0 = 0; k0 < p.C; k0 += kSeqTile) {
      const int cnt = p.C - k0 < kSeqTile ? (int)(p.C - k0) : kSeqTile;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) stage[i] = load_partial<A>(part, k0 + i);
      __syncthreads();
      if (threadIdx.x == 0)
        for (int i = 0; i < cnt; ++i) acc = A::combine(acc, stage[i]);
      __syncthreads();
    }
    res = acc;
  } else {
    // thread t folds partials r*T2 + t (identity past C), then the tree
    const int t = threadIdx.x;
    acc_t acc = A::zero();
    if (t < p.T2) {
      const int64_t R2 = ceil_div(p.C, p.T2);
      for (int64_t r = 0; r < R2; ++r) {
        const int64_t i = r * p.T2 + t;
        acc = A::combine(acc, i < p.C ? load_partial<A>(part, i) : A::zero());
      }
    }
    res = block_tree<A>(acc, p.T2, sm);
  }
  if (threadIdx.x == 0) {
    *static_cast<typename A::out_t *>(p.out) = A::result(res);
    *p.counter = 0u;  // leave the workspace counter zero for the next call
  }
}

template <class E, class A, int V, int LEVEL>
__global__ void __launch_bounds__(max_threads_for_vec(V)) reduce_kernel(const ReduceLaunch p) {
  using in_t = typename E::in_t;
  using acc_t = typename A::acc_t;
  __shared__ acc_t sm[32];
  __shared__ acc_t stage[kSeqTile];
  __shared__ int is_last;
  const in_t *x = static_cast<const in_t *>(p.x);
  const in_t *y = static_cast<const in_t *>(p.y);
  acc_t *part = static_cast<acc_t *>(p.partials);

  if constexpr (LEVEL == int(ChunkLevel::Block)) {
    const int t = threadIdx.x;
    for (int64_t c = blockIdx.x; c < p.C; c += gridDim.x) {
      const int64_t base = c * p.s + t * p.tstride;
      const bool full = (c + 1) * p.s <= p.n;
      acc_t v = thread_fold<E, A, V, false>(x, y, p.n, base, p.Rc, p.step, full);
      v = block_tree<A>(v, p.Tc, sm);
      if (t == 0) part[c] = v;
    }
  } else if constexpr (LEVEL == int(ChunkLevel::Warp)) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t w0 = blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t nw = gridDim.x * wpb;
    for (int64_t c = w0; c < p.C; c += nw) {
      const int64_t base = c * p.s + lane * p.tstride;
      const bool full = (c + 1) * p.s <= p.n;
      acc_t v = thread_fold<E, A, V, false>(x, y, p.n, base, p.Rc, p.step, full);
      v = warp_tree<A>(v, 32);
      if (lane == 0) part[c] = v;
    }
  } else {
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ng = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = g0; c < p.C; c += ng) {
      const bool full = (c + 1) * p.s <= p.n;
      part[c] = thread_fold<E, A, V, false>(x, y, p.n, c * p.s, p.Rc, p.step, full);
    }
  }

  // publish this block's partials, then take a ticket
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(p.counter, 1u);
    __threadfence();
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) second_level<A>(p, sm, stage);
}

// ---------------------------------------------------------------------------
// toLocal: chunks staged through shared memory
// ---------------------------------------------------------------------------
//
// The BLOCK/THREAD reduction with the interleaved map and V = 4, where each
// full chunk reaches the threads through shared memory: one thread copies the
// chunk tile by tile (kStages-deep ring; a tile is TR rows, a row the T*4
// consecutive items the block folds in one step) with bulk asynchronous
// copies counted on one mbarrier per stage, and thread t folds items
// (q*T + t)*4 + v of each row q from there -- the same items in the same order
// as the direct loads, so the result is bit-identical. A ragged last chunk
// takes the direct path (identity items past n).

constexpr int kStages = 4;
constexpr int kStageBytes = 16384;  // a stage holds >= 16 KiB of whole rows over all operands

__host__ __device__ constexpr int staged_rows(int threads, int operands) {
  return threads * 16 * operands >= kStageBytes ? 1 : kStageBytes / (threads * 16 * operands);
}

template <class T>
__device__ __forceinline__ void lds4(const T *p, T (&r)[4]) {
  using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
  const V4 a = *reinterpret_cast<const V4 *>(p);
  r[0] = a.x;
  r[1] = a.y;
  r[2] = a.z;
  r[3] = a.w;
}

template <class E, class A>
__global__ void __launch_bounds__(1024) reduce_staged_kernel(const ReduceLaunch p, unsigned *status) {
  using in_t = typename E::in_t;
  using acc_t = typename A::acc_t;
  constexpr int NOP = E::kTwo ? 2 : 1;
  extern __shared__ __align__(128) unsigned char ring[];
  __shared__ acc_t sm[32];
  __shared__ acc_t stage[kSeqTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int is_last, bad;
  const int t = threadIdx.x, T = blockDim.x;
  const int TR = staged_rows(T, NOP);
  const in_t *x = static_cast<const in_t *>(p.x);
  const in_t *y = static_cast<const in_t *>(p.y);
  acc_t *part = static_cast<acc_t *>(p.partials);
  const int64_t row = (int64_t)T * 4;                               // items per row
  const uint32_t op_bytes = (uint32_t)(TR * row * sizeof(in_t));   // one operand's tile
  const int64_t tpc = ceil_div(p.Rc, TR);                          // tiles per chunk
  const int64_t Cfull = p.n / p.s;                                 // chunks without identity items
  const int64_t G = gridDim.x;
  const int64_t mine = (int64_t)blockIdx.x < Cfull ? ceil_div(Cfull - blockIdx.x, G) : 0;
  const int64_t ntiles = mine * tpc;
  if (t == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
    mbar_init_fence();
    bad = 0;
  }
  __syncthreads();
  // tile k of this block: chunk blockIdx.x + (k / tpc) * G, rows (k % tpc) * TR ..
  auto issue = [&](int64_t k) {
    const int st = (int)(k % kStages);
    const int64_t c = blockIdx.x + (k / tpc) * G;
    const int64_t r0 = (k % tpc) * TR;
    const int64_t rows = p.Rc - r0 < TR ? p.Rc - r0 : TR;
    const uint32_t b = (uint32_t)(rows * row * sizeof(in_t));
    const int64_t e0 = c * p.s + r0 * row;
    unsigned char *dst = ring + (size_t)st * NOP * op_bytes;
    fence_proxy_async_smem();
    mbar_expect_tx(&full[st], NOP * b);
    bulk_load(dst, x + e0, b, &full[st]);
    if constexpr (NOP == 2) bulk_load(dst + op_bytes, y + e0, b, &full[st]);
  };
  if (t == 0)
    for (int64_t k = 0; k < kStages && k < ntiles; ++k) issue(k);
  acc_t acc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = A::zero();
  int64_t k = 0;
  for (; k < ntiles; ++k) {
    const int st = (int)(k % kStages);
    if (!mbar_wait_bounded(&full[st], (uint32_t)((k / kStages) & 1))) bad = 1;
    __syncthreads();
    if (bad) break;
    const int64_t tt = k % tpc;
    const int64_t rows = p.Rc - tt * TR < TR ? p.Rc - tt * TR : TR;
    const in_t *bx = reinterpret_cast<const in_t *>(ring + (size_t)st * NOP * op_bytes) + 4 * t;
    const in_t *by = reinterpret_cast<const in_t *>(ring + (size_t)st * NOP * op_bytes + op_bytes) + 4 * t;
    for (int64_t q = 0; q < rows; ++q) {
      in_t xv[4], yv[4];
      lds4(bx + q * row, xv);
      if constexpr (NOP == 2) lds4(by + q * row, yv);
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] = A::step(acc[v], E::elem(xv[v], E::kTwo ? yv[v] : xv[v]));
    }
    if (tt == tpc - 1) {  // the chunk is folded: lanes, then the tree
      acc_t c_acc = A::zero();
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        c_acc = A::combine(c_acc, acc[v]);
        acc[v] = A::zero();
      }
      c_acc = block_tree<A>(c_acc, T, sm);
      if (t == 0) part[blockIdx.x + (k / tpc) * G] = c_acc;
    }
    __syncthreads();  // every thread is done with stage st
    if (t == 0 && k + kStages < ntiles) issue(k + kStages);
  }
  if (bad) {
    // a copy did not complete in time: wait (bounded) for the copies still in
    // flight into this block's ring, record the error, and take the ticket
    // anyway so that the workspace counter returns to zero
    if (t == 0) {
      for (int64_t q = k; q < ntiles && q < k + kStages; ++q)
        mbar_wait_bounded(&full[q % kStages], (uint32_t)((q / kStages) & 1));
      if (status) atomicExch(status, (unsigned)DPIA_ERR_TIMEOUT);
    }
  } else if (Cfull < p.C && (int64_t)blockIdx.x == Cfull % G) {
    const int64_t c = Cfull;  // the ragged last chunk: direct loads
    acc_t v = thread_fold<E, A, 4, false>(x, y, p.n, c * p.s + t * p.tstride, p.Rc, p.step, false);
    v = block_tree<A>(v, T, sm);
    if (t == 0) part[c] = v;
  }

  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned ticket = atomicAdd(p.counter, 1u);
    __threadfence();
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) second_level<A>(p, sm, stage);
}

template <class E, class A>
cudaError_t launch_staged(int threads, int grid, const ReduceLaunch &p, cudaStream_t stream) {
  const void *k = (const void *)reduce_staged_kernel<E, A>;
  constexpr int NOP = E::kTwo ? 2 : 1;
  const size_t ring = (size_t)kStages * NOP * staged_rows(threads, NOP) * threads * 16;
  if (!ensure_dyn_smem(k, ring)) return cudaErrorInvalidConfiguration;
  if (grid <= 0) {
    const int64_t cap = (int64_t)sm_count() * resident_blocks_dyn(k, threads, ring);
    grid = (int)(p.C < cap ? p.C : cap);
    if (grid < 1) grid = 1;
  }
  unsigned *status = device_status_word();
  void *args[] = {const_cast<ReduceLaunch *>(&p), &status};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, ring, stream);
}

// Self-test of the bounded waits: one block waits on an mbarrier that nothing
// completes; the wait gives up after timeout_ns and the block records
// DPIA_ERR_TIMEOUT in the device status word. No copy is in flight.
__global__ void bounded_wait_probe_kernel(uint64_t timeout_ns, unsigned *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool done = mbar_wait_bounded(&bar, 0, timeout_ns);
  if (!done && threadIdx.x == 0 && status) atomicExch(status, (unsigned)DPIA_ERR_TIMEOUT);
}

template <class E, class A, int LEVEL>
const void *pick_v(int V) {
  switch (V) {
    case 1: return (const void *)reduce_kernel<E, A, 1, LEVEL>;
    case 2: return (const void *)reduce_kernel<E, A, 2, LEVEL>;
    case 4: return (const void *)reduce_kernel<E, A, 4, LEVEL>;
    case 8: return (const void *)reduce_kernel<E, A, 8, LEVEL>;
    case 16: return (const void *)reduce_kernel<E, A, 16, LEVEL>;
  }
  return nullptr;
}

template <class E, class A>
const void *pick_level(ChunkLevel level, int V) {
  switch (level) {
    case ChunkLevel::Grid: return pick_v<E, A, 0>(V);
    case ChunkLevel::Block: return pick_v<E, A, 1>(V);
    case ChunkLevel::Warp: return pick_v<E, A, 2>(V);
  }
  return nullptr;
}

}  // namespace

int resident_blocks(const void *kernel, int threads);

cudaError_t launch_bounded_wait_probe(uint64_t timeout_ns, cudaStream_t stream) {
  unsigned *status = device_status_word();
  if (!status) return cudaErrorInvalidSymbol;
  bounded_wait_probe_kernel<<<1, 32, 0, stream>>>(timeout_ns, status);
  return cudaGetLastError();
}

cudaError_t launch_reduce_staged(ReduceOp op, bool compensated, int threads, int grid,
                                 const ReduceLaunch &p, cudaStream_t stream) {
  if (op == ReduceOp::DotF32)
    return compensated ? launch_staged<DotF32, KahanF32>(threads, grid, p, stream)
                       : launch_staged<DotF32, SumF32>(threads, grid, p, stream);
  if (op == ReduceOp::AsumF32)
    return compensated ? launch_staged<AsumF32, KahanF32>(threads, grid, p, stream)
                       : launch_staged<AsumF32, SumF32>(threads, grid, p, stream);
  return launch_staged<DotI32, SumI64>(threads, grid, p, stream);
}

cudaError_t launch_reduce(ReduceOp op, bool compensated, int V, ChunkLevel level, int threads,
                          int grid, const ReduceLaunch &p, cudaStream_t stream) {
  const void *k = nullptr;
  if (op == ReduceOp::DotF32)
    k = compensated ? pick_level<DotF32, KahanF32>(level, V) : pick_level<DotF32, SumF32>(level, V);
  else if (op == ReduceOp::AsumF32)
    k = compensated ? pick_level<AsumF32, KahanF32>(level, V) : pick_level<AsumF32, SumF32>(level, V);
  else
    k = pick_level<DotI32, SumI64>(level, V);
  if (!k) return cudaErrorInvalidValue;
  int64_t units_per_block = level == ChunkLevel::Block ? 1 : level == ChunkLevel::Warp ? threads / 32 : threads;
  int64_t need = ceil_div(p.C, units_per_block);
  if (grid <= 0) {
    int64_t cap = (int64_t)sm_count() * resident_blocks(k, threads);
    grid = (int)(need < cap ? need : cap);
    if (grid < 1) grid = 1;
  }
  void *args[] = {const_cast<ReduceLaunch *>(&p)};
  return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, 0, stream);
}

}  // namespace dpia
