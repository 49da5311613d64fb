// Result and fault checks of the C ABI (not part of the paper's method).
//
//  * apsp_check_negative_cycle: after a solve, a vertex on a negative cycle
//    has a negative distance to itself (a closed walk of negative weight), so
//    the scan of the diagonal D[i][i] < 0 tells whether the input had one.
//    Floyd-Warshall (§2.2) assumes there is none.
//  * apsp_wait_timeout_selftest: runs the bounded mbarrier wait the bulk-copy
//    kernels use on a barrier that nothing ever completes, so the timeout path
//    (error word set, kernel returns, context stays usable) can be exercised
//    without a fault.
#include <stdint.h>

#include <mutex>

#include "bulk.cuh"
#include "common.cuh"

namespace apsp {

static __device__ int g_negcycle_flag = 0;
static std::mutex g_negcycle_mu;

template <typename Real>
__global__ void __launch_bounds__(256) diag_negative(const Real *__restrict__ D, int64_t n, int64_t ld) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (D[i * ld + i] < Real(0)) atomicExch(&g_negcycle_flag, 1);
}

// One CTA, one barrier that no thread arrives on and no copy targets: every
// poll finds phase 0 incomplete, the wait gives up after `polls` polls, and the
// CTA records APSP_ETIMEOUT exactly as the product kernels do.
__global__ void wait_timeout_probe(uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, polls);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) report_wait_timeout();
}

int take_device_error_checks() { return take_tu_device_error(); }

}  // namespace apsp

APSP_EXPORT int apsp_check_negative_cycle(const void *d_dist, int elem_bytes, int64_t n, int64_t ld,
                                          void *stream) {
  if ((elem_bytes != 4 && elem_bytes != 8) || n < 0) return APSP_EINVAL;
  if (n == 0) return APSP_OK;
  if (!d_dist || ld < n) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(apsp::g_negcycle_mu);
  cudaGetLastError();
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(apsp::g_negcycle_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return APSP_ECUDA;
  const int64_t want = (n + 255) / 256;
  const int grid = (int)(want < 1024 ? want : 1024);
  if (elem_bytes == 4)
    apsp::diag_negative<float><<<grid, 256, 0, s>>>(static_cast<const float *>(d_dist), n, ld);
  else
    apsp::diag_negative<double><<<grid, 256, 0, s>>>(static_cast<const double *>(d_dist), n, ld);
  int flag = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(&flag, apsp::g_negcycle_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return APSP_ECUDA;
  return flag ? APSP_ENEGCYCLE : APSP_OK;
}

APSP_EXPORT int apsp_wait_timeout_selftest(uint32_t polls, void *stream) {
  if (polls == 0 || polls > apsp::kWaitLimit) return APSP_EINVAL;
  cudaGetLastError();
  apsp::wait_timeout_probe<<<1, 64, 0, reinterpret_cast<cudaStream_t>(stream)>>>(polls);
  return apsp::status_from(cudaGetLastError());
}
