// FP32 min-plus block product and register-resident diagonal closure, the two
// building blocks of the FP32 kernels (single-graph phase 4 and the batched
// kernel).  Internal header.
//
// Block product (one CTA of 256 threads, TB = 16 * TM, TM x TM outputs per
// thread; TM = 8 gives TB = 128, TM = 4 gives TB = 64):
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

constexpr int THREADS = 256;  // 8 warps
constexpr int KS = 32;        // k per shared-memory slab
constexpr int KP = KS / 2;    // k-pairs per slab
constexpr int T = 128;        // block edge of the TM = 8 configuration

// Shared layout of one slab: As[kp][i] = (A[i][2kp], A[i][2kp+1]),
// Bs[kp][j] = (B[2kp][j], B[2kp+1][j]), 8 bytes per pair.
template <int TB>
union SmemT {
  struct {
    unsigned long long As[2][KP][TB];  // two slab buffers (cp.async double buffering)
    unsigned long long Bs[2][KP][TB];
  };
  float Cs[TB][TB];  // epilogue: the block of new candidates
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
using Smem = SmemT<T>;

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

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// Warp-cooperative first-argmin (all 32 lanes, warp-uniform arguments).
// arow[k] = A[i][k], bcol[k * ld] = B[k][j] for k < mK <= T.  All T/32 loads
// of a lane are issued before the first compare, so an output costs one
// memory round trip.
template <int TB>
__device__ __forceinline__ int first_argmin(const float *arow, const float *bcol, int64_t ld,
                                            float target, int mK, int lane) {
  constexpr int Q = TB / 32;
  float s[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int k = q * 32 + lane;
    s[q] = (k < mK) ? __fadd_rn(arow[k], bcol[(int64_t)k * ld]) : inf<float>();
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int k = q * 32 + lane;
    const unsigned bal = __ballot_sync(kFullMask, k < mK && s[q] == target);
    if (bal) return q * 32 + (__ffs(bal) - 1);
  }
  return -1;  // unreachable when target is one of the candidates
}

// C(baseI, baseJ) <- min(C, A(baseI, baseK) (x) B(baseK, baseJ)).  mI, mJ, mK:
// valid extents (<= TB) of the row, column and k ranges.  vec_ok: ld % 4 == 0
// and D 16-byte aligned (enables 16/8-byte global accesses).  The epilogue
// first recovers P (reading A and B from global memory), then waits at a
// barrier, then writes C, so C may be the same block as A or B (phases 2/3).
// Must be called by all 256 threads of the CTA.
template <int TM>
__device__ __forceinline__ void block_product(float *__restrict__ D, int64_t ld,
                                              int32_t *__restrict__ P, int baseI, int baseJ,
                                              int baseK, int mI, int mJ, int mK, int vec_ok,
                                              SmemT<16 * TM> &sm) {
  constexpr int TB = 16 * TM;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ty = thread_ty(), tx = thread_tx();
  const float INF = inf<float>();

  float acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TM; ++c) acc[a][c] = INF;

  // Slab staging: every element is one 4-byte asynchronous copy straight into
  // its place in the k-pair layout (As[kp][i] = (A[i][2kp], A[i][2kp+1]),
  // Bs[kp][j] = (B[2kp][j], B[2kp+1][j])); entries outside the matrix get +inf
  // by a plain store.  Two buffers: slab s+1 is in flight while s is used.
  auto stage = [&](int k0, int buf) {
    float *as = reinterpret_cast<float *>(&sm.As[buf][0][0]);
    float *bs = reinterpret_cast<float *>(&sm.Bs[buf][0][0]);
#pragma unroll
    for (int q = 0; q < TB * KS / THREADS; ++q) {  // A: lanes walk k along a row
      const int idx = tid + q * THREADS, i = idx / KS, k = idx % KS;
      float *dst = as + ((k >> 1) * TB + i) * 2 + (k & 1);
      if (i < mI && k0 + k < mK) cp_async4(dst, D + (int64_t)(baseI + i) * ld + baseK + k0 + k);
      else *dst = INF;
    }
#pragma unroll
    for (int q = 0; q < KS * TB / THREADS; ++q) {  // B: lanes walk j along a row
      const int idx = tid + q * THREADS, k = idx / TB, j = idx % TB;
      float *dst = bs + ((k >> 1) * TB + j) * 2 + (k & 1);
      if (j < mJ && k0 + k < mK) cp_async4(dst, D + (int64_t)(baseK + k0 + k) * ld + baseJ + j);
      else *dst = INF;
    }
    cp_async_commit();
  };
  const int nslab = (mK + KS - 1) / KS;
  __syncthreads();  // the previous user of sm is done with it
  stage(0, 0);
  for (int s = 0; s < nslab; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslab) {
      stage((s + 1) * KS, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // slab s visible to every thread
#pragma unroll 1
    for (int kp = 0; kp < KP; ++kp) {
      unsigned long long a[TM], b[TM];
#pragma unroll
      for (int rr = 0; rr < TM; rr += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.As[buf][kp][row_at(rr, ty)]);
        a[rr] = t.x;
        a[rr + 1] = t.y;
      }
#pragma unroll
      for (int cc = 0; cc < TM; cc += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.Bs[buf][kp][col_at(cc, tx)]);
        b[cc] = t.x;
        b[cc + 1] = t.y;
      }
#pragma unroll
      for (int rr = 0; rr < TM; ++rr)
#pragma unroll
        for (int cc = 0; cc < TM; ++cc) relax2(acc[rr][cc], a[rr], b[cc]);
    }
    __syncthreads();  // slab s consumed before its buffer is refilled
  }

  // Epilogue.  The new candidates go to shared memory; then each warp owns
  // TB/8 whole rows (lane l: columns CPL*l .. CPL*l+CPL-1), in compact rolled
  // loops.  Pass 1 computes the improvement flags and recovers P, reading A
  // and B from global memory; pass 2 (after a barrier) writes the improved
  // outputs, so C may be the same block as A or B (phases 2/3).
  constexpr int CPL = TB / 32, RPW = TB / 8;
  __syncthreads();
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; cc += 2)
      *reinterpret_cast<float2 *>(&sm.Cs[row_at(rr, ty)][col_at(cc, tx)]) =
          make_float2(acc[rr][cc], acc[rr][cc + 1]);
  __syncthreads();
  const int w = tid >> 5, j0 = CPL * lane, i0 = w * RPW;
  // Pass 1 (unrolled): every old value of the warp's rows is loaded before
  // any is used (one memory round trip), then the improvements are flagged.
  float o[RPW][CPL];
#pragma unroll
  for (int t = 0; t < RPW; ++t)
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      o[t][q] = (i0 + t < mI && j0 + q < mJ) ? D[(int64_t)(baseI + i0 + t) * ld + baseJ + j0 + q] : INF;
  unsigned long long flags = 0ull;  // bit (t * CPL + q): row i0 + t, column j0 + q
#pragma unroll
  for (int t = 0; t < RPW; ++t)
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if (sm.Cs[i0 + t][j0 + q] < o[t][q]) flags |= 1ull << (t * CPL + q);
  // Pass 2 (rolled): P for each improved output, one per warp pass; lane l
  // tests k = CPL*l .. CPL*l + CPL-1, reading A and B from global memory.
  if (P) {
    unsigned long long wflags = __reduce_or_sync(kFullMask, (unsigned)(flags >> 32));
    wflags = (wflags << 32) | __reduce_or_sync(kFullMask, (unsigned)flags);
    constexpr unsigned long long kRowMask = (1ull << CPL) - 1;
#pragma unroll 1
    while (wflags) {
      const int t = (__ffsll((long long)wflags) - 1) / CPL;
      wflags &= ~(kRowMask << (t * CPL));
      const int i = i0 + t;
      unsigned imp = (unsigned)(flags >> (t * CPL)) & (unsigned)kRowMask;
      unsigned bal = __ballot_sync(kFullMask, imp != 0);
      const float *arow = D + (int64_t)(baseI + i) * ld + baseK;
      float av[CPL];
#pragma unroll
      for (int q = 0; q < CPL; ++q) av[q] = (j0 + q < mK) ? arow[j0 + q] : INF;
      while (bal) {
        const int src = __ffs(bal) - 1;
        const unsigned sim = __shfl_sync(kFullMask, imp, src);
        const int q0 = __ffs(sim) - 1;
        if (lane == src) imp &= imp - 1;
        if (!(sim & (sim - 1))) bal &= bal - 1;
        const int sj = CPL * src + q0;
        const float tgt = sm.Cs[i][sj];
        const float *bcol = D + (int64_t)baseK * ld + baseJ + sj;
        unsigned h = 0u;
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          if (j0 + q < mK && __fadd_rn(av[q], bcol[(int64_t)(j0 + q) * ld]) == tgt) h |= 1u << q;
        const unsigned hb = __ballot_sync(kFullMask, h != 0);
        const int L = __ffs(hb) - 1;
        const unsigned hL = __shfl_sync(kFullMask, h, L & 31);
        if (lane == 0 && hb) P[(int64_t)(baseI + i) * ld + baseJ + sj] = baseK + CPL * L + (__ffs(hL) - 1);
      }
    }
  }
  __syncthreads();  // every read of A and B (staging and recovery) precedes the writes
  // Pass 3: write the improved outputs.
#pragma unroll
  for (int t = 0; t < RPW; ++t)
#pragma unroll
    for (int q = 0; q < CPL; ++q)
      if ((flags >> (t * CPL + q)) & 1ull) D[(int64_t)(baseI + i0 + t) * ld + baseJ + j0 + q] = sm.Cs[i0 + t][j0 + q];
}

// Register-resident classic FW (Algorithm 1, strict "<") on the diagonal
// block (base, base) of edge TB = 16 * TM: every thread keeps its TM x TM
// outputs in registers; at step k the owners of row k and column k publish
// them to shared memory (two alternating buffers, one barrier per step).
// Step k never changes row or column k (D[k][k] = 0), so the published values
// are the ones every thread must use.  Writes D (all valid outputs) and P
// (where improved).
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
  const int ty = thread_ty(), tx = thread_tx();
  const float INF = inf<float>();
  float d[TM][TM];
#pragma unroll
  for (int rr = 0; rr < TM; ++rr) {
    const int i = row_at(rr, ty);
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int j = col_at(cc, tx);
      d[rr][cc] = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : INF;
    }
  }
  for (int k = 0; k < m; ++k) {
    const int buf = k & 1;
#pragma unroll
    for (int rr = 0; rr < TM; ++rr)
      if (row_at(rr, ty) == k) {
#pragma unroll
        for (int cc = 0; cc < TM; ++cc) sm.row[buf][col_at(cc, tx)] = d[rr][cc];
      }
#pragma unroll
    for (int cc = 0; cc < TM; ++cc)
      if (col_at(cc, tx) == k) {
#pragma unroll
        for (int rr = 0; rr < TM; ++rr) sm.col[buf][row_at(rr, ty)] = d[rr][cc];
      }
    __syncthreads();
    float a[TM], b[TM];
#pragma unroll
    for (int rr = 0; rr < TM; ++rr) a[rr] = sm.col[buf][row_at(rr, ty)];
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) b[cc] = sm.row[buf][col_at(cc, tx)];
#pragma unroll
    for (int rr = 0; rr < TM; ++rr) {
      const int i = row_at(rr, ty);
#pragma unroll
      for (int cc = 0; cc < TM; ++cc) {
        const float cand = __fadd_rn(a[rr], b[cc]);
        if (cand < d[rr][cc]) {
          d[rr][cc] = cand;
          if (P) P[(int64_t)(base + i) * ld + base + col_at(cc, tx)] = base + k;
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
      if (i < m && j < m) D[(int64_t)(base + i) * ld + base + j] = d[rr][cc];
    }
  }
}

}  // namespace mp32
}  // namespace apsp
