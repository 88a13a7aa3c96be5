// Per-device properties and occupancy queries, cached (the first call per
// kernel and block size asks the runtime; later calls are a map lookup), and
// the dynamic shared-memory limit of kernels that need more than 48 KiB.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "kernels.h"

namespace dpia {

namespace {
std::mutex g_mu;
std::map<int, int> g_sms;
std::map<std::tuple<int, const void *, int, size_t>, int> g_resident;
std::map<std::pair<int, const void *>, size_t> g_dyn_set;  // dynamic shared memory allowed per kernel
}  // namespace

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) d = 0;
  return d;
}

int sm_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  g_sms[dev] = v;
  return v;
}

int resident_blocks_dyn(const void *kernel, int threads, size_t dyn_smem) {
  const int dev = current_device();
  auto key = std::make_tuple(dev, kernel, threads, dyn_smem);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_resident.find(key);
    if (it != g_resident.end()) return it->second;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, dyn_smem) != cudaSuccess || nb <= 0)
    nb = 1;
  std::lock_guard<std::mutex> lk(g_mu);
  g_resident[key] = nb;
  return nb;
}

int resident_blocks(const void *kernel, int threads) { return resident_blocks_dyn(kernel, threads, 0); }

bool ensure_dyn_smem(const void *kernel, size_t bytes) {
  const int dev = current_device();
  auto key = std::make_pair(dev, kernel);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dyn_set.find(key);
  if (it != g_dyn_set.end() && it->second >= bytes) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return false;
  g_dyn_set[key] = bytes;
  return true;
}

}  // namespace dpia
