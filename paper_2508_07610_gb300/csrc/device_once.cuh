// One-time, per-device launch set-up (kernel attributes, SM counts) that is safe when several host
// threads or several devices use the library: the set-up runs once for each device ordinal, under a
// lock, and later calls take a lock-free fast path.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace mpdo {

constexpr int kMaxDevices = 64;

class PerDevice {
 public:
  // Runs f(device) once for the current device; returns f's error (and retries next time) or success.
  template <typename F>
  cudaError_t once(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long bit = 1ull << dev;
    if (done_.load(std::memory_order_acquire) & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lk(mu_);
    if (done_.load(std::memory_order_relaxed) & bit) return cudaSuccess;
    e = f(dev);
    if (e == cudaSuccess) done_.fetch_or(bit, std::memory_order_release);
    return e;
  }

 private:
  std::mutex mu_;
  std::atomic<unsigned long long> done_{0};
};

// Number of SMs of the current device (cached per device).
inline int sm_count() {
  static PerDevice init;
  static int n[kMaxDevices];
  int dev = 0;
  if (init.once([&](int d) {
        int v = 0;
        cudaError_t e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        n[d] = (e == cudaSuccess && v > 0) ? v : 1;
        return cudaSuccess;
      }) != cudaSuccess)
    return 1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  return n[dev];
}

}  // namespace mpdo
