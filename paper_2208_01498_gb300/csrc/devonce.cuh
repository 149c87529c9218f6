// Per-device one-time kernel set-up shared by the CUDA sources.
//
// cudaFuncSetAttribute(cudaFuncAttributeMaxDynamicSharedMemorySize) belongs
// to the context of the device that is current when it is called, so a
// process that launches on several GPUs must set it once per device.  The
// flags are atomics: the serving thread and caller threads launch
// concurrently (setting the attribute twice is harmless).
#pragma once
#include <cuda_runtime.h>

#include <atomic>

namespace tnc {

constexpr int kMaxDevices = 64;

// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current
// device unless this flag array records that it was done there already.
template <class Kernel>
int smem_attr_once(std::atomic<int>* done, Kernel* kernel, int bytes) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  const bool tracked = dev >= 0 && dev < kMaxDevices;
  if (tracked && done[dev].load(std::memory_order_acquire) >= bytes) return 0;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return (int)e;
  if (tracked) done[dev].store(bytes, std::memory_order_release);
  return 0;
}

}  // namespace tnc
