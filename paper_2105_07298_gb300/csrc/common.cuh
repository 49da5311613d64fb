// Shared helpers of the CUDA sources (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/apsp_fw.h"

#define APSP_EXPORT extern "C" __attribute__((visibility("default")))

namespace apsp {

constexpr unsigned kFullMask = 0xffffffffu;

template <typename Real> __device__ __forceinline__ Real inf();
template <> __device__ __forceinline__ float inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double inf<double>() {
  return __longlong_as_double(0x7ff0000000000000ll);
}

// Round-to-nearest addition that the compiler may not contract or reorder.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

inline int status_from(cudaError_t e) { return e == cudaSuccess ? APSP_OK : APSP_ECUDA; }

// Sets the dynamic shared-memory limit of a kernel once per (kernel, device).
template <typename K>
inline int ensure_smem(K kernel, int bytes, int *done_flags /*[64]*/) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (dev < 0 || dev >= 64) return APSP_EUNSUPPORTED;
  if (done_flags[dev] >= bytes) return APSP_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return APSP_ECUDA;
  done_flags[dev] = bytes;
  return APSP_OK;
}

}  // namespace apsp
