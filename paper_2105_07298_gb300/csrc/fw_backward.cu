// Backward pass of Floyd-Warshall (an extension; the paper has no gradient).
//
// D[i][j] is the sum of the weights along path(i,j), the path encoded by the
// forward pass's P: path(i,j) = (i -> j) when P[i][j] = -1, otherwise
// path(i,k) ++ path(k,j) with k = P[i][j].  Hence for a loss L(D)
//     dL/dW[u][v] = sum of dL/dD[i][j] over the pairs (i,j) whose path uses
//                   the edge (u,v),
// which is piecewise constant in W (exact away from ties).
//
// Kernel: one thread per (graph, i, j); the thread walks its path by
// recomputing it from P (in-order traversal of the split tree, with an
// explicit stack of pending right endpoints) and adds dL/dD[i][j] to every
// edge it meets with an FP32 atomic add.  Nothing but P and D is kept from the
// forward pass.
#include <stdint.h>

#include "common.cuh"

namespace apsp {

constexpr int kWalkDepth = 256;  // pending right endpoints per thread (local memory)

__global__ void zero_matrices(float *__restrict__ G, int64_t n, int64_t ld, int64_t batch,
                              int64_t stride) {
  const int64_t per = n * n, total = per * batch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per, rem = e - b * per, i = rem / n, j = rem - i * n;
    G[b * stride + i * ld + j] = 0.0f;
  }
}

// Adds g to every edge of path(i,j) of one graph (P, gW with leading
// dimension ld, n vertices).  A path of a valid P has at most n - 1 edges, so
// the walk takes at most 2n - 3 steps; the cap also ends the walk on a
// malformed P (an index outside 0..n-1 or a split cycle), which is reported
// as APSP_ETOODEEP like a recursion deeper than the stack.
__device__ __forceinline__ void scatter_path(const int32_t *__restrict__ Pg, float *__restrict__ Gg, int64_t n,
                                             int64_t ld, int64_t i, int64_t j, float g, int32_t (&stack)[kWalkDepth],
                                             int32_t *__restrict__ status) {
  int64_t a = i, c = j;
  int sp = 0;
  for (int64_t steps = 0;; ++steps) {
    const int32_t k = Pg[a * ld + c];
    if (k < 0) {  // leaf: the edge a -> c
      atomicAdd(&Gg[a * ld + c], g);
      if (sp == 0) break;
      a = c;
      c = stack[--sp];
    } else {
      if (sp == kWalkDepth || k >= n || steps > 2 * n) {
        if (status) atomicExch(status, APSP_ETOODEEP);
        break;
      }
      stack[sp++] = (int32_t)c;
      c = k;
    }
  }
}

__global__ void __launch_bounds__(256)
    fw_backward_scatter_f32(const float *__restrict__ gD, const int32_t *__restrict__ P,
                            const float *__restrict__ D, float *__restrict__ gW, int64_t n,
                            int64_t ld, int64_t batch, int64_t stride, int32_t *__restrict__ status) {
  const int64_t per = n * n, total = per * batch;
  int32_t stack[kWalkDepth];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per, rem = e - b * per, i = rem / n, j = rem - i * n;
    if (i == j) continue;
    const int64_t gb = b * stride;
    const float d = D[gb + i * ld + j];
    if (!(d < inf<float>())) continue;  // no path: contributes nothing
    const float g = gD[gb + i * ld + j];
    if (g == 0.0f) continue;
    scatter_path(P + gb, gW + gb, n, ld, i, j, g, stack, status);
  }
}

// Packed batch of uneven graphs (the layout of the batched forward): graph g
// has ns[g] vertices at element offset offs[g] (ld = ns[g]).  One CTA owns a
// graph at a time (grid-stride over graphs): it zeroes the graph's gradient,
// then its threads walk the graph's pairs, so no other CTA touches it.
__global__ void __launch_bounds__(256)
    fw_backward_packed_f32(const float *__restrict__ gD, const int32_t *__restrict__ P,
                           const float *__restrict__ D, float *__restrict__ gW,
                           const int32_t *__restrict__ ns, const int64_t *__restrict__ offs, int num,
                           int32_t *__restrict__ status) {
  int32_t stack[kWalkDepth];
  for (int gi = blockIdx.x; gi < num; gi += gridDim.x) {
    const int64_t n = ns[gi], off = offs[gi];
    if (n <= 0 || off < 0) {  // uniform per CTA
      if (threadIdx.x == 0 && status && n < 0) atomicExch(status, APSP_EINVAL);
      continue;
    }
    const int64_t per = n * n;
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) gW[off + e] = 0.0f;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < per; e += blockDim.x) {
      const int64_t i = e / n, j = e - i * n;
      if (i == j) continue;
      const float d = D[off + e];
      if (!(d < inf<float>())) continue;
      const float g = gD[off + e];
      if (g == 0.0f) continue;
      scatter_path(P + off, gW + off, n, n, i, j, g, stack, status);
    }
    __syncthreads();
  }
}

}  // namespace apsp

APSP_EXPORT int apsp_fw_backward_f32(const float *d_grad_dist, const int32_t *d_path,
                                     const float *d_dist, float *d_grad_w, int64_t n, int64_t ld,
                                     int64_t batch, int64_t stride, int32_t *d_status,
                                     void *stream) {
  if (n < 0 || batch < 0) return APSP_EINVAL;
  if (n == 0 || batch == 0) {
    if (d_status) return cudaMemsetAsync(d_status, 0, 4, reinterpret_cast<cudaStream_t>(stream)) ==
                                 cudaSuccess ? APSP_OK : APSP_ECUDA;
    return APSP_OK;
  }
  if (!d_grad_dist || !d_path || !d_dist || !d_grad_w || ld < n) return APSP_EINVAL;
  if (batch > 1 && stride < n * ld) return APSP_EINVAL;
  if (n > (1 << 18)) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (d_status && cudaMemsetAsync(d_status, 0, 4, s) != cudaSuccess) return APSP_ECUDA;
  const int64_t total = n * n * batch;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (total + 255) / 256, cap = (int64_t)sms * 16;
  const int grid = (int)(want < cap ? want : cap);
  apsp::zero_matrices<<<grid, 256, 0, s>>>(d_grad_w, n, ld, batch, stride);
  apsp::fw_backward_scatter_f32<<<grid, 256, 0, s>>>(d_grad_dist, d_path, d_dist, d_grad_w, n, ld,
                                                      batch, stride, d_status);
  return apsp::status_from(cudaGetLastError());
}

APSP_EXPORT int apsp_fw_backward_packed_f32(const float *d_grad_dist, const int32_t *d_path,
                                            const float *d_dist, float *d_grad_w, const int32_t *d_n,
                                            const int64_t *d_off, int32_t num_graphs, int32_t *d_status,
                                            void *stream) {
  if (num_graphs < 0) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (d_status && cudaMemsetAsync(d_status, 0, 4, s) != cudaSuccess) return APSP_ECUDA;
  if (num_graphs == 0) return APSP_OK;
  if (!d_grad_dist || !d_path || !d_dist || !d_grad_w || !d_n || !d_off) return APSP_EINVAL;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int cap = sms * 8;
  const int grid = num_graphs < cap ? num_graphs : cap;
  apsp::fw_backward_packed_f32<<<grid, 256, 0, s>>>(d_grad_dist, d_path, d_dist, d_grad_w, d_n, d_off,
                                                     num_graphs, d_status);
  return apsp::status_from(cudaGetLastError());
}
