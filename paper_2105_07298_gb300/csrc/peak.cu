// Measured ceiling of the min-plus relaxation on this GPU (a measurement
// hook; the paper quotes datasheet peaks only, Table 1).
//
// The kernel runs the exact instruction pair of the FP32 inner loops - one
// packed add.rn.f32x2 forming two candidates and one three-input min.f32
// folding them into an accumulator - on 16 independent chains per thread,
// with no memory traffic, and times itself with the SM clock.  Every packed
// add takes its previous result as an operand, so the compiler can neither
// hoist nor merge adds (loop-invariant operands would let it, and the rate
// would come out too high).  The FP64 variant runs the pair of the FP64
// path's main loop: the same with add.rm.f32x2 (lower bounds).
#include <stdint.h>

#include "common.cuh"

namespace apsp {

template <int MODE>
__global__ void __launch_bounds__(256) peak_kernel(float *out, unsigned long long *cycles, int iters) {
  constexpr int CH = 16;
  float acc[CH], acc2[CH];
  unsigned long long t[CH], u[CH];
  const unsigned long long c = 0x3380000033800000ull;  // (2^-24, 2^-24): the sums keep changing
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    acc[j] = 1e30f;
    acc2[j] = 1e30f;
    t[j] = ((unsigned long long)__float_as_uint((float)(threadIdx.x + 2 * j + 1)) << 32) |
           __float_as_uint((float)(threadIdx.x + 2 * j));
    u[j] = t[j];
  }
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (MODE == 0) {
        asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(t[j]) : "l"(c));
        asm volatile("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tmin.f32 %0, %0, lo, hi;\n\t}"
                     : "+f"(acc[j])
                     : "l"(t[j]));
      } else {  // lower bounds of two candidates (the FP64 path's main loop)
        asm volatile("add.rm.f32x2 %0, %0, %1;" : "+l"(t[j]) : "l"(c));
        asm volatile("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tmin.f32 %0, %0, lo, hi;\n\t}"
                     : "+f"(acc[j])
                     : "l"(t[j]));
      }
    }
  }
  const unsigned long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < CH; ++j) s += acc[j] + acc2[j] + __uint_as_float((unsigned)t[j]) + __uint_as_float((unsigned)u[j]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The integer candidate of the same relaxation: one DPX fused add-then-min
// (__viaddmin_s32: min(a + b, c)) per relaxation, on 16 independent chains
// per thread.  Every instruction's add operand is its chain's previous
// result, so nothing can be hoisted, and nothing else is in the loop.
__global__ void __launch_bounds__(256) peak_kernel_dpx(int *out, unsigned long long *cycles, int iters) {
  constexpr int CH = 16;
  int acc[CH], lim[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    acc[j] = -(int)threadIdx.x - j;
    lim[j] = (int)threadIdx.x * 7 + j;
  }
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < CH; ++j) acc[j] = __viaddmin_s32(acc[j], 3, lim[j]);  // min(acc + 3, lim)
  }
  const unsigned long long t1 = clock64();
  int s = 0;
#pragma unroll
  for (int j = 0; j < CH; ++j) s += acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace apsp

// Runs the relaxation loop (dtype_bytes 4: FP32 pair; 8: the FP64 path's lower-bound pair;
// -4: the int32 DPX fused add-min)
// on every SM and writes the achieved relaxations per clock per SM.  Uses the
// caller's stream; synchronises it.  Scratch comes from stream-ordered
// allocation and is freed before returning.
APSP_EXPORT int apsp_measure_peak(int dtype_bytes, double *relax_per_clk_per_sm, void *stream) {
  if (!relax_per_clk_per_sm || (dtype_bytes != 4 && dtype_bytes != 8 && dtype_bytes != -4)) return APSP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // One wave of blocks, all resident together, so that the slowest block's
  // clock count covers every block's work (the FP64 variant holds more
  // registers and fits fewer blocks per SM than the FP32 one).
  const int threads = 256, iters = 4096;
  int per_sm = 0;
  const cudaError_t oe =
      dtype_bytes == 4   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apsp::peak_kernel<0>, threads, 0)
      : dtype_bytes == 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apsp::peak_kernel<1>, threads, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apsp::peak_kernel_dpx, threads, 0);
  if (oe != cudaSuccess || per_sm < 1) return APSP_ECUDA;
  const int blocks = sms * (per_sm < 4 ? per_sm : 4);
  float *out = nullptr;
  unsigned long long *cyc = nullptr;
  cudaGetLastError();
  if (cudaMallocAsync((void **)&out, (size_t)blocks * threads * 4, s) != cudaSuccess) return APSP_ENOMEM;
  if (cudaMallocAsync((void **)&cyc, (size_t)blocks * 8, s) != cudaSuccess) {
    cudaFreeAsync(out, s);
    return APSP_ENOMEM;
  }
  for (int rep = 0; rep < 2; ++rep) {  // the first pass warms clocks and caches
    if (dtype_bytes == 4) apsp::peak_kernel<0><<<blocks, threads, 0, s>>>(out, cyc, iters);
    else if (dtype_bytes == 8) apsp::peak_kernel<1><<<blocks, threads, 0, s>>>(out, cyc, iters);
    else apsp::peak_kernel_dpx<<<blocks, threads, 0, s>>>(reinterpret_cast<int *>(out), cyc, iters);
  }
  unsigned long long *h = new unsigned long long[blocks];
  cudaError_t e = cudaMemcpyAsync(h, cyc, (size_t)blocks * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(out, s);
  cudaFreeAsync(cyc, s);
  if (e != cudaSuccess) {
    delete[] h;
    return APSP_ECUDA;
  }
  unsigned long long mx = 1;
  for (int i = 0; i < blocks; ++i) mx = h[i] > mx ? h[i] : mx;
  delete[] h;
  // all blocks are resident at once; two relaxations (FP32, or FP64 lower
  // bounds) per instruction pair, one per DPX add-min.
  const double relax = (dtype_bytes == -4 ? 1.0 : 2.0) * 16.0 * iters * (double)threads * blocks;
  *relax_per_clk_per_sm = relax / sms / (double)mx;
  return APSP_OK;
}
