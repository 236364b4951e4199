// Error-reporting helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

namespace su2 {

// Record a printf-style message as the thread's last error and return `code`.
int fail(int code, const char* fmt, ...);
void clear_error();
// SU2_OK if every extent is even and >= 2 and the volume fits 31 bits.
int check_dims(const int dims[4]);

// Makes `dev` current for the scope and restores the caller's device after.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace su2

// Return SU2_ECUDA with the failing call's text if a CUDA call fails.
#define SU2_CU(call)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return ::su2::fail(SU2_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// As SU2_CU, running `cleanup` first (used while a handle is half built).
#define SU2_CU_CLEAN(call, cleanup)                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cleanup;                                                                       \
      return ::su2::fail(SU2_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    }                                                                                \
  } while (0)
