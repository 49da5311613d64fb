// Single-graph FP32 solve from and to host memory: the end-to-end call of the
// library (copy the weights in, the blocked FW of §2.2 on the device, copy the
// distances and the path matrix out).  The device work is apsp_fw_f32 itself;
// this file only moves the data and owns the optional work buffers.
#include <stdint.h>

#include "common.cuh"

namespace {

using apsp::status_from;

// Largest n the single-graph kernels take (apsp_fw_f32 checks it again).
constexpr int64_t kHostMaxN = int64_t(1) << 18;

int host_solve(const float *h_w, float *h_d, int32_t *h_p, int64_t n, float *d_d, int32_t *d_p,
               cudaStream_t s) {
  const size_t elems = (size_t)n * (size_t)n;
  float *D = d_d;
  int32_t *P = h_p ? d_p : nullptr;
  bool own_d = false, own_p = false;
  cudaGetLastError();
  if (!D) {
    if (cudaMallocAsync(reinterpret_cast<void **>(&D), elems * sizeof(float), s) != cudaSuccess) {
      cudaGetLastError();
      return APSP_ENOMEM;
    }
    own_d = true;
  }
  if (h_p && !P) {
    if (cudaMallocAsync(reinterpret_cast<void **>(&P), elems * sizeof(int32_t), s) != cudaSuccess) {
      cudaGetLastError();
      if (own_d) cudaFreeAsync(D, s);
      cudaStreamSynchronize(s);
      return APSP_ENOMEM;
    }
    own_p = true;
  }
  int st = status_from(cudaMemcpyAsync(D, h_w, elems * sizeof(float), cudaMemcpyHostToDevice, s));
  if (st == APSP_OK) st = apsp_fw_f32(D, n, n, P, s);
  if (st == APSP_OK) st = status_from(cudaMemcpyAsync(h_d, D, elems * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (st == APSP_OK && h_p)
    st = status_from(cudaMemcpyAsync(h_p, P, elems * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (own_p) cudaFreeAsync(P, s);
  if (own_d) cudaFreeAsync(D, s);
  // Synchronises `s`: the results are in host memory, and a bounded device
  // wait that ran out during the solve comes back as APSP_ETIMEOUT.
  const int dev_st = apsp_device_status(s);
  return st != APSP_OK ? st : dev_st;
}

}  // namespace

APSP_EXPORT int apsp_fw_f32_host(const float *h_weights, float *h_dist, int32_t *h_path, int64_t n,
                                 float *d_work_dist, int32_t *d_work_path, void *stream) {
  if (n < 0 || n > kHostMaxN) return APSP_EINVAL;
  if (n == 0) return APSP_OK;
  if (!h_weights || !h_dist) return APSP_EINVAL;
  return host_solve(h_weights, h_dist, h_path, n, d_work_dist, d_work_path,
                    reinterpret_cast<cudaStream_t>(stream));
}
