// dpia_dot_f32_noalloc: the dot product with its scratch in a static device
// array, for callers that cannot allocate device memory themselves -- for
// example a plugin hosted by another framework that owns the whole memory
// pool and hands the plugin no allocator, or a latency-critical path where a
// cudaMalloc (which may synchronise the device) is not acceptable. The caller
// still passes the inputs and the output; only the scratch (the per-chunk
// partials and the completion counter) comes from this file.
//
// The scratch lives in a file-scope __device__ array of kNoAllocScratchBytes
// that every GPU loading the library holds until the process exits. Host code
// may not pass the array's name to a kernel (on the host it is only a stand-in
// symbol), so the first call on each device, with that device current, looks
// up its device address with cudaGetSymbolAddress and caches it. That first
// call should therefore come before any stream capture on that device. The
// cached address stays valid only as long as the device's context: after
// cudaDeviceReset the array is unloaded with the rest of the device code, so
// the entry must not be used on a device that has been reset.
//
// All calls share the one array: calls that overlap on the GPU (on different
// streams, or from several host threads without ordering) race on it. The
// completion counter is cleared on every call with cudaMemsetAsync on the
// caller's stream; the partials need no clearing (each is written before it is
// read). No cudaMalloc, cudaFree or other allocating routine is called.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/dpia.h"
#include "kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = DPIA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
dpia_status scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    dpia::set_last_error("dpia_dot_f32_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
    return DPIA_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    dpia::set_last_error("dpia_dot_f32_noalloc: device ordinal %d out of range", dev);
    return DPIA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      dpia::set_last_error("dpia_dot_f32_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                           cudaGetErrorString(e));
      return DPIA_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DPIA_OK;
}

}  // namespace

extern "C" dpia_status dpia_dot_f32_noalloc(const float *x, const float *y, int64_t n,
                                            const dpia_reduce_strategy *st, float *out,
                                            dpia_stream_t stream) {
  const size_t need = dpia_dot_workspace_size(n, st);
  if (need == 0) {
    // the strategy is invalid for n: let the regular entry report why
    return dpia_dot_f32(x, y, n, st, out, nullptr, 0, stream);
  }
  if (need > kNoAllocScratchBytes) {
    dpia::set_last_error(
        "dpia_dot_f32_noalloc: this n and split need %zu bytes of scratch, more than the %zu-byte "
        "static scratch (8 bytes per chunk after a 128-byte counter: at most %zu chunks); use a larger "
        "split or dpia_dot_f32 with a workspace",
        need, kNoAllocScratchBytes, (kNoAllocScratchBytes - 128) / 8);
    return DPIA_ERR_WORKSPACE;
  }
  void *scratch = nullptr;
  dpia_status rc = scratch_for_current_device(&scratch);
  if (rc != DPIA_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 128, s);  // the completion counter starts at zero
  if (e != cudaSuccess) {
    dpia::set_last_error("dpia_dot_f32_noalloc: clearing the counter failed: %s", cudaGetErrorString(e));
    return DPIA_ERR_CUDA;
  }
  return dpia_dot_f32(x, y, n, st, out, scratch, kNoAllocScratchBytes, stream);
}
