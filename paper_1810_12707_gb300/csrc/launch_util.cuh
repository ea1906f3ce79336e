// launch_util.cuh -- host helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace mhd {

// Raise the dynamic shared-memory limit of kernel `Fn` to `bytes`, once per device.
template <auto Fn>
cudaError_t ensure_smem(int bytes) {
  static std::atomic<unsigned long long> done{0};
  static std::atomic<int> done_bytes[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if ((done.load() & bit) && done_bytes[dev & 63].load() >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(Fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  done_bytes[dev & 63].store(bytes);
  done.fetch_or(bit);
  return cudaSuccess;
}

}  // namespace mhd
