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

// Allow kernel `fn` up to `bytes` of dynamic shared memory on the current device. Function
// attributes belong to a device's context, so this is recorded per (kernel, device): the
// first call for a pair sets the attribute, later calls return at once. Returns the error of
// cudaGetDevice or cudaFuncSetAttribute (nothing is recorded after a failure).
cudaError_t set_smem_attr(const void *fn, int bytes);

}  // namespace chol

#define CHOL_CUDA_TRY(expr)                         \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return CHOL_ERR_CUDA;    \
  } while (0)
