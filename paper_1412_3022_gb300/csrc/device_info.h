// Per-device facts the launchers need, cached per device (a process may
// drive several GPUs; each has its own attributes and kernel settings).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace pmrc {

constexpr int kMaxDevices = 64;

// Streaming multiprocessors of the current device.
inline int current_sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  cudaGetDevice(&dev);
  int v = (dev >= 0 && dev < kMaxDevices) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  if (dev >= 0 && dev < kMaxDevices) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// Lets `fn` be launched with up to all the dynamic shared memory the
// current device allows a block (its opt-in limit less the kernel's static
// shared memory).  Made once per (device, slot): the bit in `done` is set
// only after the setting succeeded, so a thread that finds it set can
// launch, and concurrent first callers each make the (idempotent) setting.
// The value is the largest any launch can ask for, so launches of one
// kernel with different sizes never undo each other's setting.
inline cudaError_t allow_max_smem(const void *fn, std::atomic<uint64_t> (&done)[kMaxDevices],
                                  int slot) {
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < kMaxDevices && slot >= 0 && slot < 64;
  const uint64_t bit = cached ? 1ull << slot : 0;
  if (cached && (done[dev].load(std::memory_order_acquire) & bit)) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && cached) done[dev].fetch_or(bit, std::memory_order_release);
  return e;
}

}  // namespace pmrc
