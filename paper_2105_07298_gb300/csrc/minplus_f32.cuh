// FP32 min-plus block product and register-resident diagonal closure, the two
// building blocks of the FP32 kernels (single-graph phase 4 and the batched
// kernel).  Internal header.
//
// Block product (one CTA of 256 threads, TB = 128):
//     C[i][j] <- min(C[i][j], min_k A[i][k] + B[k][j]),  P[i][j] <- argmin k
// for a TB x TB block C of the matrix D, A = block (I,K), B = block (K,J).
// This is phase 4 of the blocked FW of §2.2 and, with A or B the closed
// diagonal block, phases 2 and 3 as well.
//
// Inner loop: every thread owns an 8 x 8 register tile; consecutive k are
// paired so that one packed add.rn.f32x2 produces both candidates of an
// output and one three-input min.f32 folds them into the accumulator.  FADD2
// runs on the FMA pipe and FMNMX3 on the ALU pipe, so a relaxation costs one
// issue slot per lane.
//
// P without path state in the inner loop: after the loop, every output whose
// minimum improved (strictly below the old value) looks for the FIRST k whose
// rounded sum equals that minimum; the 32 lanes of a warp test 32 values of k
// at a time.  Ascending k with a strict "<" keeps exactly that k, so P equals
// the one the sequential loop of Algorithm 1 writes.
#pragma once
#include "common.cuh"

namespace apsp {
namespace mp32 {

constexpr int T = 128;        // block edge
constexpr int THREADS = 256;  // 8 warps, 8 x 8 outputs per thread
constexpr int KS = 32;        // k per shared-memory slab
constexpr int KP = KS / 2;    // k-pairs per slab

// Shared layout of one slab: As[kp][i] = (A[i][2kp], A[i][2kp+1]),
// Bs[kp][j] = (B[2kp][j], B[2kp+1][j]), 8 bytes per pair.
struct Smem {
  unsigned long long As[KP][T];
  unsigned long long Bs[KP][T];
};

// Thread (warp w, lane l), wy = w/2, wx = w%2, ly = l/8, lx = l%8:
//   rows i(r) = (r>>2)*64 + wy*16 + ((r>>1)&1)*8 + ly*2 + (r&1)
//   cols j(c) = (c>>2)*64 + wx*32 + ((c>>1)&1)*16 + lx*2 + (c&1)
// Consecutive r (c) pairs are adjacent rows (columns), so each pair is one
// 16-byte shared load; one k-pair of a warp touches 64 (A) and 128 (B)
// consecutive bytes, free of bank conflicts.
__device__ __forceinline__ int row_of(int r, int wy, int ly) {
  return (r >> 2) * 64 + wy * 16 + ((r >> 1) & 1) * 8 + ly * 2 + (r & 1);
}
__device__ __forceinline__ int col_of(int c, int wx, int lx) {
  return (c >> 2) * 64 + wx * 32 + ((c >> 1) & 1) * 16 + lx * 2 + (c & 1);
}

__device__ __forceinline__ void relax2(float &acc, unsigned long long a, unsigned long long b) {
  asm("{\n\t.reg .b64 t;\n\t.reg .f32 lo, hi;\n\t"
      "add.rn.f32x2 t, %1, %2;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "min.f32 %0, %0, lo, hi;\n\t}"
      : "+f"(acc)
      : "l"(a), "l"(b));
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// Warp-cooperative first-argmin (all 32 lanes, warp-uniform arguments).
// arow[k] = A[i][k], bcol[k * ld] = B[k][j] for k < mK.
__device__ __forceinline__ int first_argmin(const float *arow, const float *bcol, int64_t ld,
                                            float target, int mK, int lane) {
  for (int k0 = 0; k0 < mK; k0 += 32) {
    const int k = k0 + lane;
    bool hit = false;
    if (k < mK) hit = (__fadd_rn(arow[k], bcol[(int64_t)k * ld]) == target);
    const unsigned bal = __ballot_sync(kFullMask, hit);
    if (bal) return k0 + (__ffs(bal) - 1);
  }
  return -1;  // unreachable when target is one of the candidates
}

// C(baseI, baseJ) <- min(C, A(baseI, baseK) (x) B(baseK, baseJ)).  mI, mJ, mK:
// valid extents (<= T) of the row, column and k ranges.  vec_ok: ld % 4 == 0
// and D 16-byte aligned (enables 16/8-byte global accesses).  The epilogue
// first recovers P (reading A and B from global memory), then waits at a
// barrier, then writes C, so C may be the same block as A or B (phases 2/3).
// Must be called by all 256 threads of the CTA.
__device__ __forceinline__ void block_product(float *__restrict__ D, int64_t ld,
                                              int32_t *__restrict__ P, int baseI, int baseJ,
                                              int baseK, int mI, int mJ, int mK, int vec_ok,
                                              Smem &sm) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wy = w >> 1, wx = w & 1, ly = lane >> 3, lx = lane & 7;
  const float INF = inf<float>();

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = INF;

  for (int k0 = 0; k0 < mK; k0 += KS) {
    __syncthreads();  // previous slab (or previous use of sm) fully consumed
    // A slab: 128 rows x 32 k; a float4 along k gives two pairs
#pragma unroll
    for (int q = 0; q < (T * KS / 4) / THREADS; ++q) {
      const int idx = tid + q * THREADS;
      const int i = idx >> 3, k4 = (idx & 7) * 4;
      const int kk = k0 + k4;
      float v[4];
      const float *src = D + (int64_t)(baseI + i) * ld + baseK + kk;
      if (vec_ok && i < mI && kk + 3 < mK) {
        const float4 t = *reinterpret_cast<const float4 *>(src);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (i < mI && kk + u < mK) ? src[u] : INF;
      }
      sm.As[k4 / 2][i] = pack2(v[0], v[1]);
      sm.As[k4 / 2 + 1][i] = pack2(v[2], v[3]);
    }
    // B slab: rows k and k+1 over 128 columns -> pairs
#pragma unroll
    for (int q = 0; q < (KP * T / 4) / THREADS; ++q) {
      const int idx = tid + q * THREADS;
      const int kp = idx >> 5, j4 = (idx & 31) * 4;
      const int kk = k0 + 2 * kp;
      float v0[4], v1[4];
      const float *s0 = D + (int64_t)(baseK + kk) * ld + baseJ + j4;
      const float *s1 = s0 + ld;
      if (vec_ok && j4 + 3 < mJ && kk + 1 < mK) {
        const float4 t0 = *reinterpret_cast<const float4 *>(s0);
        const float4 t1 = *reinterpret_cast<const float4 *>(s1);
        v0[0] = t0.x; v0[1] = t0.y; v0[2] = t0.z; v0[3] = t0.w;
        v1[0] = t1.x; v1[1] = t1.y; v1[2] = t1.z; v1[3] = t1.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v0[u] = (j4 + u < mJ && kk < mK) ? s0[u] : INF;
          v1[u] = (j4 + u < mJ && kk + 1 < mK) ? s1[u] : INF;
        }
      }
      ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(&sm.Bs[kp][j4]);
      dst[0] = make_ulonglong2(pack2(v0[0], v1[0]), pack2(v0[1], v1[1]));
      dst[1] = make_ulonglong2(pack2(v0[2], v1[2]), pack2(v0[3], v1[3]));
    }
    __syncthreads();
#pragma unroll 4
    for (int kp = 0; kp < KP; ++kp) {
      unsigned long long a[8], b[8];
#pragma unroll
      for (int rr = 0; rr < 8; rr += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.As[kp][row_of(rr, wy, ly)]);
        a[rr] = t.x;
        a[rr + 1] = t.y;
      }
#pragma unroll
      for (int cc = 0; cc < 8; cc += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.Bs[kp][col_of(cc, wx, lx)]);
        b[cc] = t.x;
        b[cc + 1] = t.y;
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) relax2(acc[rr][cc], a[rr], b[cc]);
    }
  }

  // Epilogue 1: improvement flags against the old block (one bit per output).
  unsigned long long imp = 0ull;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int i = row_of(rr, wy, ly);
    const float *src = D + (int64_t)(baseI + i) * ld + baseJ;
#pragma unroll
    for (int cc = 0; cc < 8; cc += 2) {
      const int j = col_of(cc, wx, lx);
      if (i < mI) {
        float o0 = INF, o1 = INF;
        if (vec_ok && j + 1 < mJ) {
          const float2 o = *reinterpret_cast<const float2 *>(src + j);
          o0 = o.x;
          o1 = o.y;
        } else {
          if (j < mJ) o0 = src[j];
          if (j + 1 < mJ) o1 = src[j + 1];
        }
        if (j < mJ && acc[rr][cc] < o0) imp |= 1ull << (rr * 8 + cc);
        if (j + 1 < mJ && acc[rr][cc + 1] < o1) imp |= 1ull << (rr * 8 + cc + 1);
      }
    }
  }
  // Epilogue 2: P recovery for improved outputs, one output per warp pass.
  if (P) {
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        unsigned bal = __ballot_sync(kFullMask, (imp >> (rr * 8 + cc)) & 1ull);
        while (bal) {
          const int src = __ffs(bal) - 1;
          bal &= bal - 1;
          const float tgt = __shfl_sync(kFullMask, acc[rr][cc], src);
          const int si = row_of(rr, __shfl_sync(kFullMask, wy, src), __shfl_sync(kFullMask, ly, src));
          const int sj = col_of(cc, __shfl_sync(kFullMask, wx, src), __shfl_sync(kFullMask, lx, src));
          const int64_t gi = baseI + si, gj = baseJ + sj;
          const int k = first_argmin(D + gi * ld + baseK, D + (int64_t)baseK * ld + gj, ld, tgt,
                                     mK, lane);
          if (lane == 0 && k >= 0) P[gi * ld + gj] = baseK + k;
        }
      }
    }
  }
  __syncthreads();  // every read of A and B (staging and recovery) precedes the writes
  // Epilogue 3: write the improved outputs.
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int i = row_of(rr, wy, ly);
    float *dst = D + (int64_t)(baseI + i) * ld + baseJ;
#pragma unroll
    for (int cc = 0; cc < 8; cc += 2) {
      const int j = col_of(cc, wx, lx);
      const bool i0 = (imp >> (rr * 8 + cc)) & 1ull, i1 = (imp >> (rr * 8 + cc + 1)) & 1ull;
      if (i0 && i1 && vec_ok) {
        *reinterpret_cast<float2 *>(dst + j) = make_float2(acc[rr][cc], acc[rr][cc + 1]);
      } else {
        if (i0) dst[j] = acc[rr][cc];
        if (i1) dst[j + 1] = acc[rr][cc + 1];
      }
    }
  }
}

// Register-resident classic FW (Algorithm 1, strict "<") on the diagonal
// block (base, base): every thread keeps its 8 x 8 outputs in registers; at
// step k the owners of row k and column k publish them to shared memory (two
// alternating buffers, one barrier per step).  Step k never changes row or
// column k (D[k][k] = 0), so the published values are the ones every thread
// must use.  Writes D (all valid outputs) and P (where improved).
struct DiagSmem {
  float row[2][T];
  float col[2][T];
};

__device__ __forceinline__ void diag_closure(float *__restrict__ D, int64_t ld,
                                             int32_t *__restrict__ P, int base, int m,
                                             DiagSmem &sm) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int wy = w >> 1, wx = w & 1, ly = lane >> 3, lx = lane & 7;
  const float INF = inf<float>();
  float d[8][8];
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int i = row_of(rr, wy, ly);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int j = col_of(cc, wx, lx);
      d[rr][cc] = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : INF;
    }
  }
  for (int k = 0; k < m; ++k) {
    const int buf = k & 1;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
      if (row_of(rr, wy, ly) == k) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) sm.row[buf][col_of(cc, wx, lx)] = d[rr][cc];
      }
#pragma unroll
    for (int cc = 0; cc < 8; ++cc)
      if (col_of(cc, wx, lx) == k) {
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) sm.col[buf][row_of(rr, wy, ly)] = d[rr][cc];
      }
    __syncthreads();
    float a[8], b[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) a[rr] = sm.col[buf][row_of(rr, wy, ly)];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) b[cc] = sm.row[buf][col_of(cc, wx, lx)];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      const int i = row_of(rr, wy, ly);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const float cand = __fadd_rn(a[rr], b[cc]);
        if (cand < d[rr][cc]) {
          d[rr][cc] = cand;
          if (P) P[(int64_t)(base + i) * ld + base + col_of(cc, wx, lx)] = base + k;
        }
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int i = row_of(rr, wy, ly);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int j = col_of(cc, wx, lx);
      if (i < m && j < m) D[(int64_t)(base + i) * ld + base + j] = d[rr][cc];
    }
  }
}

}  // namespace mp32
}  // namespace apsp
