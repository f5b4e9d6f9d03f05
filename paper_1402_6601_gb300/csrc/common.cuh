// Shared host/device helpers of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/chol.h"

namespace chol {

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T>
__device__ __forceinline__ T ld_volatile(const T *p) {
  return *(const volatile T *)p;
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
};

// Properties of the current device (queried once per device and cached).
DeviceInfo current_device_info();

}  // namespace chol

#define CHOL_CUDA_TRY(expr)                         \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return CHOL_ERR_CUDA;    \
  } while (0)
