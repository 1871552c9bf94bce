// Current-device guard for the C-ABI entry points: makes a handle's device
// current for the duration of one call and gives the calling thread its
// previous device back on every return path, so a caller that works with
// another device on the same thread finds it unchanged after the call.
#pragma once
#include <cuda_runtime.h>

namespace lbmib_host {

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      cudaGetLastError();
      prev_ = -1;
    }
    if (prev_ != dev) {
      st_ = cudaSetDevice(dev);
      if (st_ != cudaSuccess) cudaGetLastError();
      changed_ = st_ == cudaSuccess && prev_ >= 0;
    }
  }
  ~DeviceGuard() {
    if (changed_) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  // cudaSuccess when the device is current
  cudaError_t status() const { return st_; }

 private:
  int prev_ = -1;
  bool changed_ = false;
  cudaError_t st_ = cudaSuccess;
};

}  // namespace lbmib_host
