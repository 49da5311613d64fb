// Integer (int32) weights, exact (the paper's weights are generic; §2.2).
//
// FP32 sums are exact only while every path sum stays below 2^24.  For int32
// weights the relaxation is carried out exactly by the FP64 path: every int32
// value and every sum of fewer than 2^22 of them is an integer below 2^53, so
// each FP64 addition is exact and the distances equal the integer ones.  The
// FP64 path runs its main loop on FP32 lower bounds (about 1.2e13
// relaxations/s on GB300).  A native integer main loop was measured instead
// (apsp_measure_peak with dtype_bytes = -4): the DPX fused add-then-min
// sustains fewer relaxations per clock than the FP32 instruction pair, so it
// would not be faster.
//
// Conversion kernels: int32 -> double (APSP_I32_INF -> +inf) into a
// stream-ordered n x n scratch, the FP64 solve, then double -> int32 (+inf ->
// APSP_I32_INF; a finite distance outside the int32 range saturates and sets
// the error word to APSP_EUNSUPPORTED, read by apsp_device_status).
#include <stdint.h>

#include "bulk.cuh"
#include "common.cuh"

namespace apsp {

constexpr int32_t kI32Inf = 0x7fffffff;
constexpr double kI32Max = 2147483646.0, kI32Min = -2147483647.0;

__global__ void i32_to_f64(const int32_t *__restrict__ A, int64_t n, int64_t ld, double *__restrict__ B) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const int32_t x = A[i * ld + j];
    B[e] = x == kI32Inf ? inf<double>() : (double)x;
  }
}

__global__ void f64_to_i32(const double *__restrict__ B, int64_t n, int64_t ld, int32_t *__restrict__ A) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const double v = B[e];
    int32_t x;
    if (v == inf<double>()) {
      x = kI32Inf;
    } else if (v > kI32Max || v < kI32Min) {
      x = v > 0 ? (int32_t)kI32Max : (int32_t)kI32Min;
      atomicExch(&g_device_error, APSP_EUNSUPPORTED);
    } else {
      x = (int32_t)v;
    }
    A[i * ld + j] = x;
  }
}

int take_device_error_int32() { return take_tu_device_error(); }

}  // namespace apsp

extern "C" int apsp_fw_f64(double *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream);

APSP_EXPORT int apsp_fw_i32(int32_t *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream) {
  if (n < 0 || n > (1 << 18)) return APSP_EINVAL;
  if (n == 0) return APSP_OK;
  if (!d_dist || ld < n) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  double *tmp = nullptr;
  if (cudaMallocAsync((void **)&tmp, (size_t)n * n * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return APSP_ENOMEM;
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n * n + 255) / 256, cap = (int64_t)sms * 16;
  const int grid = (int)(want < cap ? want : cap);
  apsp::i32_to_f64<<<grid, 256, 0, s>>>(d_dist, n, ld, tmp);
  int st = apsp::status_from(cudaGetLastError());
  if (st == APSP_OK) st = apsp_fw_f64(tmp, n, n, d_path, stream);
  if (st == APSP_OK) {
    apsp::f64_to_i32<<<grid, 256, 0, s>>>(tmp, n, ld, d_dist);
    st = apsp::status_from(cudaGetLastError());
  }
  cudaFreeAsync(tmp, s);
  return st;
}
