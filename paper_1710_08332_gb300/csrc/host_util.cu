// Per-device properties and occupancy queries, cached (the first call per
// kernel and block size asks the runtime; later calls are a map lookup).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "kernels.h"

namespace dpia {

namespace {
std::mutex g_mu;
std::map<int, int> g_sms;
std::map<std::tuple<int, const void *, int>, int> g_resident;
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

int resident_blocks(const void *kernel, int threads) {
  const int dev = current_device();
  auto key = std::make_tuple(dev, kernel, threads);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_resident.find(key);
    if (it != g_resident.end()) return it->second;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb <= 0)
    nb = 1;
  std::lock_guard<std::mutex> lk(g_mu);
  g_resident[key] = nb;
  return nb;
}

}  // namespace dpia
