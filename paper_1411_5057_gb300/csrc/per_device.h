// Host-side "once per CUDA device" guard for settings that the runtime keeps
// per device, such as a kernel's dynamic shared-memory limit
// (cudaFuncSetAttribute applies to the current device only).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace firls {

class PerDeviceOnce {
 public:
  // Runs fn() on the current device unless an earlier call on this device
  // succeeded.  fn returns true when every step succeeded; only then is the
  // device marked, so a failed attempt is retried by the next call.  Callers
  // on other host threads wait until the first one has finished, so no
  // launch can run before the settings are in place.  Devices beyond 63 run
  // fn every time.
  template <class Fn>
  void run(Fn&& fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done_.load(std::memory_order_acquire) & bit)) return;
    std::lock_guard<std::mutex> lock(mu_);
    if (bit && (done_.load(std::memory_order_relaxed) & bit)) return;
    if (fn() && bit) done_.fetch_or(bit, std::memory_order_release);
  }

 private:
  std::atomic<unsigned long long> done_{0};
  std::mutex mu_;
};

}  // namespace firls
