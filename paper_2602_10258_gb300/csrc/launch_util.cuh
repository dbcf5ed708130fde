// Occupancy and device helpers shared by the launch code of several files.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "search_core.cuh"

namespace jag {

// Blocks of kSearchWarps warps that fit on one SM with smem bytes of dynamic
// shared memory (0 if none); also raises the kernel's shared-memory limit.
template <class Kern>
inline int blocks_per_sm(Kern kern, size_t smem, int warps = kSearchWarps) {
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // all of the unified L1 / shared storage may go to shared memory: the
  // occupancy query (and the launch) then count with the largest carve-out
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, warps * 32, smem) != cudaSuccess) b = 0;
  return b > 0 ? b : 0;
}

inline int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace jag
