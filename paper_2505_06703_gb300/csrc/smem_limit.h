// Raising a kernel's dynamic shared-memory limit, once per (kernel, device).
//
// cudaFuncSetAttribute(..., cudaFuncAttributeMaxDynamicSharedMemorySize, ...)
// applies to the device that is current when it is called.  Each launcher
// keeps one SmemLimit per kernel: the largest size set so far on each device
// ordinal, so a second device's first large launch still makes the call, and
// launches that fit make none (which keeps attribute calls out of CUDA graph
// captures after a device's first launch).  Host code only.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace anim {

constexpr int kMaxAttrDevices = 64;

struct SmemLimit {
  std::atomic<size_t> set[kMaxAttrDevices];  // static storage: zero-initialized
};

inline std::mutex &smem_limit_mutex() {
  static std::mutex m;
  return m;
}

// Make sure `fn` may use `smem` bytes of dynamic shared memory on the current
// device.  Sizes up to `floor` need no attribute call.  The fast path is one
// atomic load; updates are serialized so the cached size never exceeds the
// size last set on that device.
inline cudaError_t ensure_smem_limit(const void *fn, SmemLimit &lim, size_t smem, size_t floor = 0) {
  if (smem <= floor) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kMaxAttrDevices;
  if (cached && smem <= lim.set[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(smem_limit_mutex());
  if (cached && smem <= lim.set[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cached) lim.set[dev].store(smem, std::memory_order_release);
  if (e != cudaSuccess) cudaGetLastError();  // returned here: do not leave it for a later launch check
  return e;
}

}  // namespace anim
