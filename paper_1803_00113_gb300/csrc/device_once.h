// One-time set-up per device, safe under concurrent callers.
//
// Kernel attributes (the dynamic shared memory limit) and measured occupancy
// belong to a device, not to the process: a process may drive several
// devices, and the library's callers (the server's worker threads among
// them) call it from several threads.  DeviceOnce runs a set-up function
// once for each device on which it is needed, with that device current, and
// records success per device under a mutex.  Private to the library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace celeste {

constexpr int kMaxDevices = 64;

class DeviceOnce {
 public:
  // Runs f() (returning cudaError_t) unless it already succeeded on the
  // calling thread's current device; a failure is returned and retried by
  // the next call.
  template <class F>
  cudaError_t run(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done_[dev].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu_);
    if (done_[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    e = f();
    if (e == cudaSuccess) done_[dev].store(true, std::memory_order_release);
    return e;
  }

 private:
  std::mutex mu_;
  std::atomic<bool> done_[kMaxDevices] = {};
};

// The calling thread's current device (0 if the query fails).
inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  return dev;
}

}  // namespace celeste
