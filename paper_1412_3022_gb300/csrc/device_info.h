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

// One bit per (device, slot) for settings made once per device, e.g. a
// kernel's shared-memory opt-in.  Returns true the first time a pair is
// claimed.
inline bool first_on_device(std::atomic<uint64_t> (&mask)[kMaxDevices], int slot) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices || slot < 0 || slot >= 64) return true;
  const uint64_t bit = 1ull << slot;
  return !(mask[dev].fetch_or(bit, std::memory_order_relaxed) & bit);
}

}  // namespace pmrc
