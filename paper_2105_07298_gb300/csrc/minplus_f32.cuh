// Building blocks shared by the FP32 kernels (internal header): the paired
// min-plus relaxation, the thread-to-output mapping of the register tiles,
// asynchronous 4-byte copies, and the register-resident closure of a
// diagonal block (phase 1 of the blocked FW of §2.2).
//
// Paired relaxation: consecutive k are paired so that one packed
// add.rn.f32x2 produces both candidates of an output and one three-input
// min.f32 folds them into the accumulator.  FADD2 runs on the FMA pipe and
// FMNMX3 on the ALU pipe, so a relaxation costs one issue slot per lane.
#pragma once
#include "common.cuh"

namespace apsp {
namespace mp32 {

constexpr int THREADS = 256;  // 8 warps
constexpr int KS = 32;        // k per shared-memory slab
constexpr int KP = KS / 2;    // k-pairs per slab
constexpr int T = 128;        // block edge of the TM = 8 configuration

// 4-byte asynchronous global -> shared copy (cp.async) and its group fences.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Thread (warp w, lane l): ty = (w/2)*4 + l/8 (0..15), tx = (w%2)*8 + l%8
// (0..15); its TM rows and TM columns come in adjacent pairs:
//   rows i(r) = (r>>1)*32 + ty*2 + (r&1),  cols j(c) = (c>>1)*32 + tx*2 + (c&1).
// Each pair is one 16-byte shared load; one k-pair of a warp touches 64 (A)
// and 128 (B) consecutive bytes, free of bank conflicts.
__device__ __forceinline__ int thread_ty() { return ((threadIdx.x >> 5) >> 1) * 4 + ((threadIdx.x & 31) >> 3); }
__device__ __forceinline__ int thread_tx() { return ((threadIdx.x >> 5) & 1) * 8 + (threadIdx.x & 7); }
__device__ __forceinline__ int row_at(int r, int ty) { return (r >> 1) * 32 + ty * 2 + (r & 1); }
__device__ __forceinline__ int col_at(int c, int tx) { return (c >> 1) * 32 + tx * 2 + (c & 1); }

__device__ __forceinline__ void relax2(float &acc, unsigned long long a, unsigned long long b) {
  asm("{\n\t.reg .b64 t;\n\t.reg .f32 lo, hi;\n\t"
      "add.rn.f32x2 t, %1, %2;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "min.f32 %0, %0, lo, hi;\n\t}"
      : "+f"(acc)
      : "l"(a), "l"(b));
}

// relax2's new accumulator, returned instead of stored (for eager tracking).
__device__ __forceinline__ float min3f_pair(float acc, unsigned long long a, unsigned long long b) {
  float m;
  asm("{\n\t.reg .b64 t;\n\t.reg .f32 lo, hi;\n\t"
      "add.rn.f32x2 t, %1, %2;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "min.f32 %0, %3, lo, hi;\n\t}"
      : "=f"(m)
      : "l"(a), "l"(b), "f"(acc));
  return m;
}

// The two candidate sums of relax2, unfolded (same rounding).
__device__ __forceinline__ float2 sum2(unsigned long long a, unsigned long long b) {
  unsigned long long t;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(a), "l"(b));
  return make_float2(__uint_as_float((unsigned)t), __uint_as_float((unsigned)(t >> 32)));
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// Register-resident classic FW (Algorithm 1, strict "<") on the diagonal
// block (base, base) of edge TB = 16 * TM: every thread keeps its TM x TM
// outputs in registers; at step k the owners of row k and column k publish
// them to shared memory (two alternating buffers, one barrier per step).
// Step k never changes row or column k (D[k][k] = 0), so the published values
// are the ones every thread must use.  k is walked as 32 kb + 2 kk + q with
// kb and q unrolled, so the owners' register index is a constant; candidates
// form in pairs (one add.rn.f32x2 for two adjacent columns), and the block-
// local k of each output's last improvement is kept as a byte in registers.
// Steps past the last valid vertex only meet +inf padding and change nothing.
// Writes D (all valid outputs) and P (where improved).
template <int TB>
struct DiagSmemT {
  float row[2][TB];
  float col[2][TB];
};
using DiagSmem = DiagSmemT<T>;

template <int TM>
__device__ __forceinline__ void diag_closure(float *__restrict__ D, int64_t ld,
                                             int32_t *__restrict__ P, int base, int m,
                                             DiagSmemT<16 * TM> &sm) {
  static_assert(TM % 4 == 0, "columns are kept in pairs and path bytes in fours");
  const int ty = thread_ty(), tx = thread_tx();
  const float INF = inf<float>();
  float d[TM][TM];
  unsigned pk[TM][TM / 4];  // byte cc % 4 of pk[rr][cc / 4]: local k, 0xFF none
#pragma unroll
  for (int rr = 0; rr < TM; ++rr) {
    const int i = row_at(rr, ty);
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int j = col_at(cc, tx);
      d[rr][cc] = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : INF;
    }
#pragma unroll
    for (int c4 = 0; c4 < TM / 4; ++c4) pk[rr][c4] = 0xFFFFFFFFu;
  }
#pragma unroll
  for (int kb = 0; kb < TM / 2; ++kb) {
#pragma unroll 1
    for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = 32 * kb + 2 * kk + q;  // row_at / col_at index 2 kb + q of owner kk
        if (ty == kk) {
#pragma unroll
          for (int cc = 0; cc < TM; cc += 2)
            *reinterpret_cast<float2 *>(&sm.row[q][col_at(cc, tx)]) = make_float2(d[2 * kb + q][cc], d[2 * kb + q][cc + 1]);
        }
        if (tx == kk) {
#pragma unroll
          for (int rr = 0; rr < TM; rr += 2)
            *reinterpret_cast<float2 *>(&sm.col[q][row_at(rr, ty)]) = make_float2(d[rr][2 * kb + q], d[rr + 1][2 * kb + q]);
        }
        __syncthreads();
        float a[TM];
        unsigned long long b[TM / 2];
#pragma unroll
        for (int rr = 0; rr < TM; rr += 2) {
          const float2 t = *reinterpret_cast<const float2 *>(&sm.col[q][row_at(rr, ty)]);
          a[rr] = t.x;
          a[rr + 1] = t.y;
        }
#pragma unroll
        for (int cc = 0; cc < TM; cc += 2) b[cc / 2] = *reinterpret_cast<const unsigned long long *>(&sm.row[q][col_at(cc, tx)]);
#pragma unroll
        for (int rr = 0; rr < TM; ++rr) {
          const unsigned long long aa = pack2(a[rr], a[rr]);
#pragma unroll
          for (int c2 = 0; c2 < TM / 2; ++c2) {
            const float2 cand = sum2(aa, b[c2]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int cc = 2 * c2 + h;
              const float cv = h ? cand.y : cand.x;
              if (cv < d[rr][cc]) {
                d[rr][cc] = cv;
                pk[rr][cc / 4] = __byte_perm(pk[rr][cc / 4], (unsigned)k,
                                             0x3210 ^ ((0x3210 & (0xF << (4 * (cc & 3)))) ^ (4 << (4 * (cc & 3)))));
              }
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < TM; ++rr) {
    const int i = row_at(rr, ty);
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int j = col_at(cc, tx);
      if (i < m && j < m) {
        D[(int64_t)(base + i) * ld + base + j] = d[rr][cc];
        const unsigned kl = (pk[rr][cc / 4] >> (8 * (cc & 3))) & 0xFFu;
        if (P && kl != 0xFFu) P[(int64_t)(base + i) * ld + base + j] = base + (int)kl;
      }
    }
  }
}

}  // namespace mp32
}  // namespace apsp
