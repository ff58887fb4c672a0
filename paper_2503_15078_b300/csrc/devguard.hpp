// Current-device guard of the C ABI's entry points (internal header).
#pragma once

#include <cuda_runtime.h>

namespace silg {

// Makes `device` current for the scope of an entry point and gives the calling thread its
// own current device back at the end (an entry point leaves no device switch behind).
// device < 0: only save and restore (code in the scope selects the device itself).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device = -1) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (device >= 0 && device != prev) cudaSetDevice(device);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

}  // namespace silg
