// Host-side launch interface between the C ABI layer (abi.cu) and the kernel
// translation units. Arguments arrive here already validated.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dpia {

enum class ReduceOp { DotF32 = 0, AsumF32 = 1, DotI32 = 2 };
enum class ChunkLevel { Grid = 0, Block = 1, Warp = 2 };

struct ReduceLaunch {
  const void *x;
  const void *y;
  int64_t n;
  int64_t s;        // chunk elements
  int64_t C;        // chunks
  int64_t Rc;       // fold steps per thread per chunk: s / (Tc * V)
  int64_t step;     // elements between a thread's successive fold steps
  int64_t tstride;  // elements between the first items of neighbouring threads
  int Tc;           // threads per chunk
  int second_tree;  // 0 seq, 1 tree
  int T2;           // threads of the tree second level
  void *partials;   // C (or padded) partials
  unsigned *counter;
  void *out;
};

// Launch the reduction; returns cudaSuccess or the launch error. `grid` = 0
// picks a persistent grid.
cudaError_t launch_reduce(ReduceOp op, bool compensated, int V, ChunkLevel level, int threads,
                          int grid, const ReduceLaunch &p, cudaStream_t stream);

// The same reduction (BLOCK/THREAD, V = 4, interleaved map) with each chunk
// staged through shared memory by bulk asynchronous copies (toLocal).
cudaError_t launch_reduce_staged(ReduceOp op, bool compensated, int threads, int grid,
                                 const ReduceLaunch &p, cudaStream_t stream);

// One block that waits timeout_ns on an mbarrier nothing completes, then sets
// the device status word to DPIA_ERR_TIMEOUT.
cudaError_t launch_bounded_wait_probe(uint64_t timeout_ns, cudaStream_t stream);

// Device address of the library's sticky device status word (0 = no error;
// DPIA_ERR_TIMEOUT after a bounded wait ran out), or null.
unsigned *device_status_word();

struct GemvLaunch {
  const float *A;
  int64_t M, N, lda;
  const float *x;
  float *y;
  int64_t s;        // row chunk elements
  int64_t Crow;     // chunks per row
  int64_t Rc;       // fold steps per thread per chunk
  int64_t step;
  int64_t tstride;
  int Tc;
};
cudaError_t launch_gemv(bool compensated, int V, ChunkLevel level, int threads, int grid,
                        const GemvLaunch &p, cudaStream_t stream);

cudaError_t launch_scal(float a, const float *x, float *y, int64_t n, int V, cudaStream_t stream);
cudaError_t launch_dot_bwd(const float *x, const float *y, const float *g, int64_t n, float *dx,
                           float *dy, cudaStream_t stream);
cudaError_t launch_outer(const float *x, const float *dy, int64_t M, int64_t N, float *dA,
                         int64_t ldda, int vec, cudaStream_t stream);

struct GemvBwdLaunch {
  const float *A;
  int64_t M, N, lda;
  const float *dy;
  float *dx;
  int64_t Rs;        // rows per chunk
  int64_t Cr;        // row chunks
  float *partials;   // Cr x Npad
  int64_t Npad;
  unsigned *counters;  // one per column tile
  int vec;             // A 16-byte aligned and lda a multiple of 4: 128-bit loads
};
cudaError_t launch_gemv_bwd_dx(const GemvBwdLaunch &p, cudaStream_t stream);

// Device properties cached per device.
int sm_count();
// Resident blocks per SM of a kernel at a block size and dynamic shared memory.
int resident_blocks_dyn(const void *kernel, int threads, size_t dyn_smem);
// Allow a kernel `bytes` of dynamic shared memory on the current device.
bool ensure_dyn_smem(const void *kernel, size_t bytes);

// Set the calling host thread's dpia_last_error_message() text (printf format).
void set_last_error(const char *fmt, ...);

}  // namespace dpia
