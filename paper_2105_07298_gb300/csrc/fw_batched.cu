// Batched Floyd-Warshall: thousands of independent graphs of uneven size in
// one persistent launch (an extension; the paper solves one matrix at a time).
//
// Work distribution: the plan orders the graphs largest first (longest
// processing time first) and the CTAs of a grid sized to fill every SM pop
// graph indices from one atomic counter.  A CTA solves its graph alone, so no
// CTA ever waits on another.
//
// Per graph (n_g <= 1024, row-major, ld = n_g) the CTA runs the blocked FW of
// §2.2 on the matrix in global memory, with one of three kernel variants
// chosen per size class by the autotuner:
//   variants 0 and 1, 64 x 64 blocks, 4 x 4 register tile per thread:
//     phase 1     register-resident closure of the diagonal block;
//     phases 2+3  row block (r,J) <- min(C, D*(r,r) (x) C) and column block
//                 (I,r) <- min(C, C (x) D*(r,r)): once the diagonal block is
//                 closed, the sequential k loop over a panel block equals one
//                 min-plus product with the closed block (same value in exact
//                 arithmetic), so these phases use the phase-4 block product;
//     phase 4     (I,J) <- min(C, D(I,r) (x) D(r,J)), both operand blocks whole
//                 in shared memory (k-pair layout);
//     path matrix: variant 0 recovers each improved output's first argmin k
//     from the operands after the product (lazy), variant 1 keeps the index
//     of the last improving k-pair in the inner loop (eager);
//     variant 1, and every variant run without a path matrix, pipelines the
//     products of a phase group: the operands of the next product are copied
//     into a second shared-memory stage while the current one computes.
//   variant 2, 128 x 128 blocks, 8 x 4 register tile per thread: the
//     single-graph kernels' code run by one CTA: the register-resident closure
//     for phase 1, the k-sequential line kernel for phases 2+3 (the paper's
//     order), which also writes the round's operand panels into this CTA's
//     scratch, and the bulk-copy ring product for phase 4 (two 128 x 64
//     halves per block), tracking the path eagerly in the product's inner
//     loop (a graph of n <= 1024 has at most 8 rounds, all dense in
//     improvements).
// On integer-valued weights all sums are exact and D equals every other
// correct FW whatever the variant; on real weights variant 2 gives the
// sequential blocked FW's values at TB = 128 (those of apsp_fw_f32), variants
// 0 and 1 round phases 2/3 through the closed block instead.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "bulk.cuh"
#include "common.cuh"
#include "minplus_f32.cuh"
#include "phases_f32.cuh"

namespace apsp {

constexpr int kBatchedMaxN = 1024;

constexpr int kNumClasses = 4;
static const int32_t kClassLo[kNumClasses] = {1, 65, 129, 257};
static const int32_t kClassHi[kNumClasses] = {64, 128, 256, kBatchedMaxN};
__host__ __device__ constexpr int class_of_n(int32_t n) {
  return n <= 64 ? 0 : n <= 128 ? 1 : n <= 256 ? 2 : 3;
}
constexpr int kNumVariants = 3;
static int g_variant[kNumClasses] = {1, 1, 1, 1};
// Block edge, register tile and path tracking of each variant (for the
// autotuner's table).
static const int kVariantBlock[kNumVariants] = {64, 64, 128};
static const int kVariantTileRows[kNumVariants] = {4, 4, 8};
static const int kVariantTileCols[kNumVariants] = {4, 4, 4};
static const int kVariantEager[kNumVariants] = {0, 1, 1};
constexpr int kT128 = mp32::T;
// Per-CTA operand panels of the 128-block variants: Apan, Bpan, Acp and Bt of
// every block of one round (R <= 8 blocks for n <= 1024), 4-byte words.
__host__ __device__ constexpr size_t panel_words_per_array(int rmax) { return (size_t)rmax * kT128 * kT128; }
__host__ __device__ constexpr size_t panel_bytes_per_cta(int rmax) { return 4 * panel_words_per_array(rmax) * 4; }

static int class_of(int32_t n) { return class_of_n(n); }

namespace b64 {
constexpr int T = 64;           // block edge
constexpr int TM = 4;           // 4 x 4 outputs per thread, 256 threads
constexpr int KP = T / 2;       // k-pairs per block
constexpr int ST = T + 2;       // row stride of the pair arrays (16-byte rows, fewer conflicts)
constexpr int CS = T + 8;       // row stride of Cs: a warp's 8-byte stores (four rows two
                                // apart) take the minimum two shared-memory wavefronts

struct ProdSmem {
  unsigned long long As[KP][ST];  // As[kp][i] = (A[i][2kp], A[i][2kp+1])
  unsigned long long Bs[KP][ST];  // Bs[kp][j] = (B[2kp][j], B[2kp+1][j])
  float Cs[T][CS];                // new candidates
};
// Operand stage of the pipelined products: the same k-pair layout.
struct Stage {
  unsigned long long As[KP][ST];
  unsigned long long Bs[KP][ST];
};
// Output tile of thread (warp w, lane l) in the pipelined products:
// ty = 2 w + l / 16, tx = l % 16 (rows and columns from mp32::row_at/col_at).
// A quarter-warp shares its A pairs with the next one and its B pairs with
// the one two further (measured 2 % faster than the phase-4 mapping here).
__device__ __forceinline__ int prod_ty() { return (threadIdx.x >> 5) * 2 + ((threadIdx.x & 31) >> 4); }
__device__ __forceinline__ int prod_tx() { return threadIdx.x & 15; }
}  // namespace b64

union BatchedSmem {
  b64::ProdSmem prod;
  b64::Stage stage[2];
  mp32::DiagSmemT<64> diag;
  mp32::DiagSmemT<128> diag128;
  float lines_M[k2::T * k2::MS];
  k3::Smem prod128;
};

// Eager path tracking per k-pair: the three-input min writes the new
// accumulator, and the pair index is kept when it lowered the accumulator
// strictly.  Which k of the last such pair reached the final value is settled
// once per output after the loop (the lower k if its candidate equals the
// final value: the strict "<" of the sequential loop keeps the first k
// reaching a minimum).
__device__ __forceinline__ void relax2_argpair(float &acc, int &kp_last, unsigned long long a,
                                               unsigned long long b, int kp) {
  float m;
  asm("{\n\t.reg .b64 t;\n\t.reg .f32 lo, hi;\n\t"
      "add.rn.f32x2 t, %1, %2;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "min.f32 %0, %3, lo, hi;\n\t}"
      : "=f"(m)
      : "l"(a), "l"(b), "f"(acc));
  kp_last = m < acc ? kp : kp_last;
  acc = m;
}

// C(baseI, baseJ) <- min(C, A(baseI, baseK) (x) B(baseK, baseJ)), TB = 64,
// all 256 threads, the lazy path matrix of variant 0 (each improved output's
// first argmin k recovered from the operands after the product).  C may be
// the same block as A or B: the operands are copied to shared memory first
// and C is written only after every read.
__device__ __forceinline__ void product64_lazy(float *__restrict__ D, int ld, int32_t *__restrict__ P,
                                               int baseI, int baseJ, int baseK, int mI, int mJ, int mK,
                                               b64::ProdSmem &sm) {
  using namespace b64;
  using mp32::col_at;
  using mp32::row_at;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ty = mp32::thread_ty(), tx = mp32::thread_tx();
  const float INF = inf<float>();
  __syncthreads();  // the previous user of sm is done with it
  {  // both operand blocks, every element one 4-byte asynchronous copy
    float *as = reinterpret_cast<float *>(&sm.As[0][0]);
    float *bs = reinterpret_cast<float *>(&sm.Bs[0][0]);
#pragma unroll
    for (int q = 0; q < T * T / 256; ++q) {
      const int idx = tid + q * 256, i = idx / T, k = idx % T;
      float *dst = as + ((k >> 1) * ST + i) * 2 + (k & 1);
      if (i < mI && k < mK) mp32::cp_async4(dst, D + (int64_t)(baseI + i) * ld + baseK + k);
      else *dst = INF;
    }
#pragma unroll
    for (int q = 0; q < T * T / 256; ++q) {
      const int idx = tid + q * 256, k = idx / T, j = idx % T;
      float *dst = bs + ((k >> 1) * ST + j) * 2 + (k & 1);
      if (j < mJ && k < mK) mp32::cp_async4(dst, D + (int64_t)(baseK + k) * ld + baseJ + j);
      else *dst = INF;
    }
    mp32::cp_async_commit();
    mp32::cp_async_wait<0>();
  }
  __syncthreads();
  float acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TM; ++c) acc[a][c] = INF;
  const int kpn = (mK + 1) / 2;
  auto load_pair = [&](int kp, unsigned long long (&a)[TM], unsigned long long (&b)[TM]) {
#pragma unroll
    for (int rr = 0; rr < TM; rr += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.As[kp][row_at(rr, ty)]);
      a[rr] = t.x;
      a[rr + 1] = t.y;
    }
#pragma unroll
    for (int cc = 0; cc < TM; cc += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&sm.Bs[kp][col_at(cc, tx)]);
      b[cc] = t.x;
      b[cc + 1] = t.y;
    }
  };
#pragma unroll 1
  for (int kp = 0; kp < kpn; ++kp) {
    unsigned long long a[TM], b[TM];
    load_pair(kp, a, b);
#pragma unroll
    for (int rr = 0; rr < TM; ++rr)
#pragma unroll
      for (int cc = 0; cc < TM; ++cc) mp32::relax2(acc[rr][cc], a[rr], b[cc]);
  }
  // Epilogue: candidates to shared memory; each warp then owns 8 whole rows,
  // lane l the columns 2l and 2l+1.
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; cc += 2) {
      *reinterpret_cast<float2 *>(&sm.Cs[row_at(rr, ty)][col_at(cc, tx)]) =
          make_float2(acc[rr][cc], acc[rr][cc + 1]);
    }
  __syncthreads();
  const int i0 = w * 8, j0 = 2 * lane;
  float o[8][2];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 2; ++q)
      o[t][q] = (i0 + t < mI && j0 + q < mJ) ? D[(int64_t)(baseI + i0 + t) * ld + baseJ + j0 + q] : INF;
  unsigned flags = 0u;  // bit 2t + q: row i0 + t, column j0 + q improved
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (sm.Cs[i0 + t][j0 + q] < o[t][q]) flags |= 1u << (2 * t + q);
  if (P) {
    // lazy P: one improved output per warp pass; lane l tests k = 2l, 2l+1
    // with one paired add of As[l][i] and Bs[l][j] (shared memory).
    unsigned wflags = __reduce_or_sync(kFullMask, flags);
#pragma unroll 1
    while (wflags) {
      const int t = (__ffs(wflags) - 1) >> 1;
      wflags &= ~(3u << (2 * t));
      const int i = i0 + t;
      unsigned imp = (flags >> (2 * t)) & 3u;
      unsigned bal = __ballot_sync(kFullMask, imp != 0);
      const unsigned long long av = sm.As[lane][i];
      while (bal) {
        const int src = __ffs(bal) - 1;
        const unsigned sim = __shfl_sync(kFullMask, imp, src);
        const int q0 = __ffs(sim) - 1;
        if (lane == src) imp &= imp - 1;
        if (!(sim & (sim - 1))) bal &= bal - 1;
        const int sj = 2 * src + q0;
        const float tgt = sm.Cs[i][sj];
        const unsigned long long bv = sm.Bs[lane][sj];
        float c0, c1;
        asm("{\n\t.reg .b64 t;\n\tadd.rn.f32x2 t, %2, %3;\n\tmov.b64 {%0, %1}, t;\n\t}"
            : "=f"(c0), "=f"(c1)
            : "l"(av), "l"(bv));
        const unsigned h = (c0 == tgt ? 1u : 0u) | (c1 == tgt ? 2u : 0u);
        const unsigned hb = __ballot_sync(kFullMask, h != 0);
        const int L = __ffs(hb) - 1;
        const unsigned hL = __shfl_sync(kFullMask, h, L & 31);
        if (lane == 0 && hb) P[(int64_t)(baseI + i) * ld + baseJ + sj] = baseK + 2 * L + (__ffs(hL) - 1);
      }
    }
  }
  __syncthreads();  // every read of the operands precedes the writes
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if ((flags >> (2 * t + q)) & 1u) {
        const int64_t g = (int64_t)(baseI + i0 + t) * ld + baseJ + j0 + q;
        D[g] = sm.Cs[i0 + t][j0 + q];
      }
}

// Variant 0 with a path matrix: unpipelined products, lazy path recovery.
__device__ __forceinline__ void solve_graph_lazy_f32(float *__restrict__ D, int32_t *__restrict__ P,
                                                int n, BatchedSmem &sm) {
  constexpr int T = b64::T;
  const int ld = n;
  const int R = (n + T - 1) / T;
  for (int r = 0; r < R; ++r) {
    const int base = r * T, m = min(T, n - base);
    __syncthreads();
    mp32::diag_closure<4>(D, ld, P, base, m, sm.diag);
    __syncthreads();
    for (int J = 0; J < R; ++J) {
      if (J == r) continue;
      product64_lazy(D, ld, P, base, J * T, base, m, min(T, n - J * T), m, sm.prod);
    }
    for (int I = 0; I < R; ++I) {
      if (I == r) continue;
      product64_lazy(D, ld, P, I * T, base, base, min(T, n - I * T), m, m, sm.prod);
    }
    __syncthreads();
    for (int I = 0; I < R; ++I) {
      if (I == r) continue;
      for (int J = 0; J < R; ++J) {
        if (J == r) continue;
        product64_lazy(D, ld, P, I * T, J * T, base, min(T, n - I * T), min(T, n - J * T), m, sm.prod);
      }
    }
  }
  __syncthreads();
}

// --------------------------------------------------------------------------
// Pipelined 64-block products (variant 1, and every variant without a path
// matrix).  The products of one group (phases 2+3 of a round, or its phase 4)
// neither read nor write a block another product of the group writes, so the
// operands of product p+1 are copied into the second stage while product p
// computes.  The accumulator starts at C itself, so an output's pair index is
// set only when a candidate beats C strictly, which is the sequential loop's
// rule, and only such outputs are resolved and written (from registers).
// --------------------------------------------------------------------------

// Both operand blocks of one product into a stage (4-byte asynchronous
// copies into the k-pair layout, +inf outside the valid extents), committed
// as one group.
__device__ __forceinline__ void stage_operands(b64::Stage &s, const float *__restrict__ D, int ld, int baseI,
                                               int baseJ, int baseK, int mI, int mJ, int mK) {
  using namespace b64;
  const int tid = threadIdx.x;
  const float INF = inf<float>();
  float *as = reinterpret_cast<float *>(&s.As[0][0]);
  float *bs = reinterpret_cast<float *>(&s.Bs[0][0]);
#pragma unroll
  for (int q = 0; q < T * T / 256; ++q) {
    const int idx = tid + q * 256, i = idx / T, k = idx % T;
    float *dst = as + ((k >> 1) * ST + i) * 2 + (k & 1);
    if (i < mI && k < mK) mp32::cp_async4(dst, D + (int64_t)(baseI + i) * ld + baseK + k);
    else *dst = INF;
  }
#pragma unroll
  for (int q = 0; q < T * T / 256; ++q) {
    const int idx = tid + q * 256, k = idx / T, j = idx % T;
    float *dst = bs + ((k >> 1) * ST + j) * 2 + (k & 1);
    if (j < mJ && k < mK) mp32::cp_async4(dst, D + (int64_t)(baseK + k) * ld + baseJ + j);
    else *dst = INF;
  }
  mp32::cp_async_commit();
}

// C(baseI, baseJ) <- min(C, A (x) B) from a filled stage, TB = 64, all 256
// threads; TRACK writes P (the first k whose candidate beats C strictly).
template <bool TRACK>
__device__ __forceinline__ void product64_staged(float *__restrict__ D, int ld, int32_t *__restrict__ P, int baseI,
                                                 int baseJ, int baseK, int mI, int mJ, int mK,
                                                 const b64::Stage &s) {
  using namespace b64;
  using mp32::col_at;
  using mp32::row_at;
  const int ty = prod_ty(), tx = prod_tx();
  const float INF = inf<float>();
  float acc[TM][TM];
  // TRACK: the first pair of the last chunk that lowered the accumulator
  // (-1: none); otherwise C itself, to find the improved outputs.
  int aux[TM][TM];
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int i = row_at(rr, ty), j = col_at(cc, tx);
      acc[rr][cc] = (i < mI && j < mJ) ? D[(int64_t)(baseI + i) * ld + baseJ + j] : INF;
      aux[rr][cc] = TRACK ? -1 : __float_as_int(acc[rr][cc]);
    }
  const int kpn = (mK + 1) / 2;
  auto load_pair = [&](int kp, unsigned long long (&a)[TM], unsigned long long (&b)[TM]) {
#pragma unroll
    for (int rr = 0; rr < TM; rr += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&s.As[kp][row_at(rr, ty)]);
      a[rr] = t.x;
      a[rr + 1] = t.y;
    }
#pragma unroll
    for (int cc = 0; cc < TM; cc += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&s.Bs[kp][col_at(cc, tx)]);
      b[cc] = t.x;
      b[cc + 1] = t.y;
    }
  };
  int kp0 = 0;
  if constexpr (TRACK) {
    // Two k-pairs (four k) per step, one compare and one select per output.
#pragma unroll 1
    for (; kp0 + 1 < kpn; kp0 += 2) {
      unsigned long long a0[TM], b0[TM], a1[TM], b1[TM];
      load_pair(kp0, a0, b0);
      load_pair(kp0 + 1, a1, b1);
#pragma unroll
      for (int rr = 0; rr < TM; ++rr)
#pragma unroll
        for (int cc = 0; cc < TM; ++cc) {
          const float m1 = mp32::min3f_pair(acc[rr][cc], a0[rr], b0[cc]);
          const float m2 = mp32::min3f_pair(m1, a1[rr], b1[cc]);
          aux[rr][cc] = m2 < acc[rr][cc] ? kp0 : aux[rr][cc];
          acc[rr][cc] = m2;
        }
    }
  }
#pragma unroll 1
  for (int kp = kp0; kp < kpn; ++kp) {  // TRACK: an odd last pair only
    unsigned long long a[TM], b[TM];
    load_pair(kp, a, b);
#pragma unroll
    for (int rr = 0; rr < TM; ++rr)
#pragma unroll
      for (int cc = 0; cc < TM; ++cc) {
        if (TRACK) relax2_argpair(acc[rr][cc], aux[rr][cc], a[rr], b[cc], kp);
        else mp32::relax2(acc[rr][cc], a[rr], b[cc]);
      }
  }
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int i = row_at(rr, ty), j = col_at(cc, tx);
      const float g = acc[rr][cc];
      const int64_t e = (int64_t)(baseI + i) * ld + baseJ + j;
      if constexpr (TRACK) {
        const int kp = aux[rr][cc];
        if (kp >= 0) {  // improved: the first k of the chunk whose candidate is the final value
          // both pairs of the chunk, without branches (a lone last pair
          // has its value in c0; c1 is then unused)
          const int kq = min(kp + 1, KP - 1);
          const float2 c0 = mp32::sum2(s.As[kp][i], s.Bs[kp][j]);
          const float2 c1 = mp32::sum2(s.As[kq][i], s.Bs[kq][j]);
          const int k = c0.x == g ? 2 * kp : c0.y == g ? 2 * kp + 1 : c1.x == g ? 2 * kp + 2 : 2 * kp + 3;
          D[e] = g;
          P[e] = baseK + k;
        }
      } else {
        if (g < __int_as_float(aux[rr][cc])) D[e] = g;
      }
    }
}

// The products of round r (base = 64 r, m valid vertices) in group 0 (phases
// 2+3: the row blocks (r, J), then the column blocks (I, r), each a product
// with the closed diagonal block) or group 1 (phase 4), two stages deep.
template <bool TRACK>
__device__ __forceinline__ void run_group64(float *__restrict__ D, int ld, int32_t *__restrict__ P, int n, int r,
                                            int group, b64::Stage (&st)[2]) {
  constexpr int T = b64::T;
  const int R = (n + T - 1) / T, base = r * T, m = min(T, n - base);
  const int np = group == 0 ? 2 * (R - 1) : (R - 1) * (R - 1);
  auto coords = [&](int p, int &bI, int &bJ, int &mI, int &mJ) {
    int I, J;
    if (group == 0) {
      const int o = p % (R - 1), O = o < r ? o : o + 1;
      I = p < R - 1 ? r : O;
      J = p < R - 1 ? O : r;
    } else {
      const int a = p / (R - 1), b = p % (R - 1);
      I = a < r ? a : a + 1;
      J = b < r ? b : b + 1;
    }
    bI = I * T;
    bJ = J * T;
    mI = min(T, n - bI);
    mJ = min(T, n - bJ);
  };
  int bI, bJ, mI, mJ;
  coords(0, bI, bJ, mI, mJ);
  stage_operands(st[0], D, ld, bI, bJ, base, mI, mJ, m);
#pragma unroll 1
  for (int p = 0; p < np; ++p) {
    int cI, cJ, cmI, cmJ;
    coords(p, cI, cJ, cmI, cmJ);
    if (p + 1 < np) {
      __syncthreads();  // product p-1 is done with the stage refilled here
      coords(p + 1, bI, bJ, mI, mJ);
      stage_operands(st[(p + 1) & 1], D, ld, bI, bJ, base, mI, mJ, m);
      mp32::cp_async_wait<1>();
    } else {
      mp32::cp_async_wait<0>();
    }
    __syncthreads();  // every thread's copies into stage p & 1 are visible
    product64_staged<TRACK>(D, ld, P, cI, cJ, base, cmI, cmJ, m, st[p & 1]);
  }
}

template <bool TRACK>
__device__ __forceinline__ void solve_graph_pipe_f32(float *__restrict__ D, int32_t *__restrict__ P, int n,
                                                     BatchedSmem &sm) {
  constexpr int T = b64::T;
  const int ld = n;
  const int R = (n + T - 1) / T;
  for (int r = 0; r < R; ++r) {
    const int base = r * T, m = min(T, n - base);
    __syncthreads();  // the previous round's products are done with the stages
    mp32::diag_closure<4>(D, ld, P, base, m, sm.diag);
    __syncthreads();
    if (R == 1) break;
    run_group64<TRACK>(D, ld, P, n, r, 0, sm.stage);
    __syncthreads();  // the panels are final (and visible) before phase 4 copies them
    run_group64<TRACK>(D, ld, P, n, r, 1, sm.stage);
  }
  __syncthreads();
}

// The 128-block variant: the single-graph phases run by this CTA alone.
// The panels (this CTA's scratch) are rewritten every round, so the product's
// path recovery reads them through the coherent path (NC = false), and every
// thread fences its generic writes before the bulk copies read them.
// Returns false if a bounded copy wait ran out (error word set).
__device__ __forceinline__ bool solve_graph128_f32(float *__restrict__ D, int32_t *__restrict__ P, int n,
                                                   const Panels &pan, bool aligned, unsigned char *smem_raw) {
  constexpr int T = kT128;
  BatchedSmem &sm = *reinterpret_cast<BatchedSmem *>(smem_raw);
  const int64_t ld = n;
  const int R = (n + T - 1) / T;
  const int vec_ok = aligned && (n % 4 == 0);
  for (int r = 0; r < R; ++r) {
    const int base = r * T, m = min(T, n - base);
    __syncthreads();
    mp32::diag_closure<8>(D, ld, P, base, m, sm.diag128);
    __syncthreads();
    if (R == 1) break;
    for (int side = 0; side < 2; ++side) {  // row blocks (r, J), then column blocks (I, r)
      const bool is_row = side == 0;
      lines_load_diag(D, ld, n, r, is_row);
      __syncthreads();
      for (int o = 0; o < R; ++o) {
        if (o == r) continue;
        for (int part = 0; part < k2::PARTS; ++part) lines_part_f32(D, ld, P, n, r, o, is_row, part, pan);
      }
      __syncthreads();
    }
    fence_proxy_async_global();
    __syncthreads();
    for (int I = 0; I < R; ++I) {
      if (I == r) continue;
      for (int J = 0; J < R; ++J) {
        if (J == r) continue;
        for (int hJ = 0; hJ < 2; ++hJ) {
          __syncthreads();  // the previous product's epilogue is done with the shared memory
          if (!minplus_half_f32<true, false>(D, ld, P, n, I, J, hJ, r, vec_ok, pan)) return false;
        }
      }
    }
  }
  __syncthreads();
  return true;
}

// Work item t: graph order[t] & 0x3fffffff, variant order[t] >> 30.
// scratch: per-CTA panel space of the 128-block variant (panel_bytes_per_cta(rmax)
// bytes per CTA).  Two instances: the 64-block variants alone (three CTAs per
// SM), and all variants (two CTAs per SM: the 128-block code needs more
// registers); a plan launches the second only if some graph uses variant 2.
template <bool WITH128>
__device__ __forceinline__ void persistent_body(float *__restrict__ Dp, int32_t *__restrict__ Pp,
                                                const int32_t *__restrict__ order, const int32_t *__restrict__ ns,
                                                const int64_t *__restrict__ offs, int num, int *__restrict__ counter,
                                                unsigned char *__restrict__ scratch, int rmax) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchedSmem &sm = *reinterpret_cast<BatchedSmem *>(smem_raw);
  __shared__ int s_next;
  Panels pan{};
  if (WITH128 && scratch) {
    unsigned char *base = scratch + (size_t)blockIdx.x * panel_bytes_per_cta(rmax);
    const size_t words = panel_words_per_array(rmax);
    pan.Apan = reinterpret_cast<unsigned long long *>(base);
    pan.Bpan = reinterpret_cast<unsigned long long *>(base + words * 4);
    pan.Acp = reinterpret_cast<float *>(base + 2 * words * 4);
    pan.Bt = reinterpret_cast<float *>(base + 3 * words * 4);
  }
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_next;
    __syncthreads();  // all threads have read s_next before it is overwritten
    if (t >= num) break;
    const int item = order[t];
    const int g = item & 0x3fffffff, variant = (int)((unsigned)item >> 30);
    const int64_t off = offs[g];
    const int n = ns[g];
    float *D = Dp + off;
    int32_t *P = Pp ? Pp + off : nullptr;
    if (P) {
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) P[e] = -1;
    }
    bool ok = true;
    if constexpr (WITH128) {
      if (variant == 2 && scratch) {
        const bool aligned = (reinterpret_cast<uintptr_t>(D) & 15) == 0;
        ok = solve_graph128_f32(D, P, n, pan, aligned, smem_raw);
        if (!ok) return;  // a copy wait ran out: the error word is set, this CTA stops
        continue;
      }
    }
    if (!P)
      solve_graph_pipe_f32<false>(D, P, n, sm);
    else if (variant == 1 || variant == 2)
      solve_graph_pipe_f32<true>(D, P, n, sm);
    else
      solve_graph_lazy_f32(D, P, n, sm);
  }
}

__global__ void __launch_bounds__(mp32::THREADS, 3)
    fw_batched_persistent_f32(float *__restrict__ Dp, int32_t *__restrict__ Pp,
                              const int32_t *__restrict__ order, const int32_t *__restrict__ ns,
                              const int64_t *__restrict__ offs, int num, int *__restrict__ counter,
                              unsigned char *__restrict__ scratch, int rmax) {
  persistent_body<false>(Dp, Pp, order, ns, offs, num, counter, scratch, rmax);
}

__global__ void __launch_bounds__(mp32::THREADS, 2)
    fw_batched_persistent128_f32(float *__restrict__ Dp, int32_t *__restrict__ Pp,
                                 const int32_t *__restrict__ order, const int32_t *__restrict__ ns,
                                 const int64_t *__restrict__ offs, int num, int *__restrict__ counter,
                                 unsigned char *__restrict__ scratch, int rmax) {
  persistent_body<true>(Dp, Pp, order, ns, offs, num, counter, scratch, rmax);
}

}  // namespace apsp

struct apsp_batched_plan {
  int32_t num;
  int32_t *d_order;
  int32_t *d_n;
  int64_t *d_off;
  int *d_counter;
  int grid;
  unsigned char *d_scratch;  // panels of the 128-block variants (grid CTAs), or NULL
  int rmax;                  // blocks per side of the largest graph that uses them
};

namespace {

int validate(const int32_t *h_n, const int64_t *h_off, int32_t num) {
  if (num < 0 || (num > 0 && (!h_n || !h_off))) return APSP_EINVAL;
  if (num > (1 << 30)) return APSP_EUNSUPPORTED;
  for (int32_t g = 0; g < num; ++g) {
    if (h_n[g] < 1 || h_n[g] > apsp::kBatchedMaxN) return h_n[g] < 1 ? APSP_EINVAL : APSP_EUNSUPPORTED;
    if (h_off[g] < 0 || (h_off[g] & 3)) return APSP_EINVAL;
  }
  return APSP_OK;
}

// Largest graphs first (longest processing time first); each entry carries
// the variant of its size class in bits 30-31.  *rmax: blocks per side (of
// 128) of the largest graph given a 128-block variant, 0 if none is.
std::vector<int32_t> lpt_order(const int32_t *h_n, int32_t num, int *rmax) {
  std::vector<int32_t> order(num);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return h_n[a] > h_n[b]; });
  *rmax = 0;
  for (auto &g : order) {
    const int v = apsp::g_variant[apsp::class_of(h_n[g])];
    if (v >= 2) *rmax = std::max(*rmax, (h_n[g] + apsp::kT128 - 1) / apsp::kT128);
    g |= v << 30;
  }
  return order;
}

int g_smem_batched[64], g_smem_batched128[64];

using PersistentKernel = void (*)(float *, int32_t *, const int32_t *, const int32_t *, const int64_t *, int, int *,
                                  unsigned char *, int);

PersistentKernel kernel_for(bool with128) {
  return with128 ? apsp::fw_batched_persistent128_f32 : apsp::fw_batched_persistent_f32;
}

// Grid of the persistent launch: every SM filled with resident CTAs.
int grid_for(int32_t num, bool with128) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  const PersistentKernel k = kernel_for(with128);
  if (apsp::ensure_smem(k, (int)sizeof(apsp::BatchedSmem), with128 ? g_smem_batched128 : g_smem_batched))
    return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem)) !=
      cudaSuccess)
    return -1;
  const int g = sms * std::max(occ, 1);
  return std::max(1, std::min<int>(g, num));
}

}  // namespace

APSP_EXPORT int apsp_batched_plan_create(const int32_t *h_n, const int64_t *h_off, int32_t num,
                                         apsp_batched_plan **out_plan) {
  if (!out_plan) return APSP_EINVAL;
  *out_plan = nullptr;
  int st = validate(h_n, h_off, num);
  if (st) return st;
  apsp_batched_plan *p = (apsp_batched_plan *)calloc(1, sizeof(apsp_batched_plan));
  if (!p) return APSP_ENOMEM;
  p->num = num;
  const size_t cnt = (size_t)std::max(num, 1);
  if (cudaMalloc(&p->d_order, cnt * 4) != cudaSuccess || cudaMalloc(&p->d_n, cnt * 4) != cudaSuccess ||
      cudaMalloc(&p->d_off, cnt * 8) != cudaSuccess || cudaMalloc(&p->d_counter, 4) != cudaSuccess) {
    apsp_batched_plan_destroy(p);
    return APSP_ENOMEM;
  }
  if (num > 0) {
    std::vector<int32_t> order = lpt_order(h_n, num, &p->rmax);
    if (cudaMemcpy(p->d_order, order.data(), (size_t)num * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      apsp_batched_plan_destroy(p);
      return APSP_ECUDA;
    }
  }
  p->grid = grid_for(num, p->rmax > 0);
  if (p->grid < 0) {
    apsp_batched_plan_destroy(p);
    return APSP_ECUDA;
  }
  if (p->rmax > 0 &&
      cudaMalloc(&p->d_scratch, (size_t)p->grid * apsp::panel_bytes_per_cta(p->rmax)) != cudaSuccess) {
    cudaGetLastError();
    apsp_batched_plan_destroy(p);
    return APSP_ENOMEM;
  }
  *out_plan = p;
  return APSP_OK;
}

APSP_EXPORT int apsp_batched_plan_destroy(apsp_batched_plan *p) {
  if (!p) return APSP_OK;
  cudaFree(p->d_order);
  cudaFree(p->d_n);
  cudaFree(p->d_off);
  cudaFree(p->d_counter);
  cudaFree(p->d_scratch);
  free(p);
  return APSP_OK;
}

APSP_EXPORT int apsp_fw_batched_run_f32(const apsp_batched_plan *p, float *d_dist, int32_t *d_path,
                                        void *stream) {
  if (!p) return APSP_EINVAL;
  if (p->num == 0) return APSP_OK;
  if (!d_dist) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (cudaMemsetAsync(p->d_counter, 0, sizeof(int), s) != cudaSuccess) return APSP_ECUDA;
  kernel_for(p->rmax > 0)<<<p->grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
      d_dist, d_path, p->d_order, p->d_n, p->d_off, p->num, p->d_counter, p->d_scratch, p->rmax);
  return apsp::status_from(cudaGetLastError());
}

APSP_EXPORT int apsp_fw_batched_f32(float *d_dist, int32_t *d_path, const int32_t *h_n,
                                    const int64_t *h_off, int32_t num, void *stream) {
  int st = validate(h_n, h_off, num);
  if (st) return st;
  if (num == 0) return APSP_OK;
  if (!d_dist) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rmax = 0;
  std::vector<int32_t> order = lpt_order(h_n, num, &rmax);
  int grid = grid_for(num, rmax > 0);
  if (grid <= 0) return APSP_ECUDA;
  // one scratch block: counter | order | n | offsets | panels of the
  // 128-block variants (stream-ordered allocation)
  const size_t list_bytes = (16 + (size_t)num * 8 + (size_t)num * 8 + (size_t)num * 8 + 255) & ~(size_t)255;
  const size_t bytes = list_bytes + (rmax > 0 ? (size_t)grid * apsp::panel_bytes_per_cta(rmax) : 0);
  char *scratch = nullptr;
  cudaGetLastError();
  if (cudaMallocAsync((void **)&scratch, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return APSP_ENOMEM;
  }
  unsigned char *panels = rmax > 0 ? reinterpret_cast<unsigned char *>(scratch + list_bytes) : nullptr;
  int *d_counter = reinterpret_cast<int *>(scratch);
  int32_t *d_order = reinterpret_cast<int32_t *>(scratch + 16);
  int32_t *d_n = d_order + num;
  int64_t *d_off = reinterpret_cast<int64_t *>(scratch + 16 + (((size_t)num * 8 + 15) & ~(size_t)15));
  // offsets region starts 16-byte aligned after order and n (2 * 4 * num bytes)
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    kernel_for(rmax > 0)<<<grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
        d_dist, d_path, d_order, d_n, d_off, num, d_counter, panels, rmax);
    e = cudaGetLastError();
  }
  // Copies from pageable host memory have consumed their sources when they
  // return, so `order` may go out of scope; the scratch is freed in stream order.
  cudaFreeAsync(scratch, s);
  return apsp::status_from(e);
}

APSP_EXPORT int apsp_batched_num_classes(void) { return apsp::kNumClasses; }

APSP_EXPORT int apsp_batched_class_bounds(int cls, int32_t *lo, int32_t *hi) {
  if (cls < 0 || cls >= apsp::kNumClasses || !lo || !hi) return APSP_EINVAL;
  *lo = apsp::kClassLo[cls];
  *hi = apsp::kClassHi[cls];
  return APSP_OK;
}

APSP_EXPORT int apsp_batched_num_variants(int cls) {
  return (cls < 0 || cls >= apsp::kNumClasses) ? 0 : apsp::kNumVariants;
}

APSP_EXPORT int apsp_batched_set_variant(int cls, int variant) {
  if (cls < 0 || cls >= apsp::kNumClasses || variant < 0 || variant >= apsp::kNumVariants)
    return APSP_EINVAL;
  apsp::g_variant[cls] = variant;
  return APSP_OK;
}

APSP_EXPORT int apsp_batched_get_variant(int cls) {
  return (cls < 0 || cls >= apsp::kNumClasses) ? -1 : apsp::g_variant[cls];
}

APSP_EXPORT int apsp_batched_variant_info(int variant, int32_t *block, int32_t *tile_rows, int32_t *tile_cols,
                                          int32_t *eager) {
  if (variant < 0 || variant >= apsp::kNumVariants || !block || !tile_rows || !tile_cols || !eager)
    return APSP_EINVAL;
  *block = apsp::kVariantBlock[variant];
  *tile_rows = apsp::kVariantTileRows[variant];
  *tile_cols = apsp::kVariantTileCols[variant];
  *eager = apsp::kVariantEager[variant];
  return APSP_OK;
}

// ---------------------------------------------------------------------------
// No-allocation batched entry point (no counterpart in the paper).
//
// Some callers cannot allocate device memory at call time: a serving loop
// that forbids cudaMalloc on its hot path, code whose device memory comes
// from an allocator CUDA does not own, or a library embedded where any hidden
// allocation is an error.  This entry point takes the work list (counter,
// largest-first order, sizes, offsets) from one file-scope device array of
// fixed size instead of allocating it, and builds the order on the GPU, so it
// allocates nothing, on the device or on the host.
//
// The array (1 MiB + 16 bytes, up to kNoAllocMaxGraphs graphs) is held by
// every GPU that loads the library until the process exits.  Host code cannot
// pass the array's name to a kernel (in host code it is only a stand-in, not
// a device address): every call looks its address up with
// cudaGetSymbolAddress while the caller's device is current.  The first call
// on a device also loads the library's module there, so it should come
// before any stream capture on that device.  All calls
// share the array and it keeps the previous call's contents; each call
// resets the counter it needs.  Calls that overlap on the GPU (other streams,
// other host threads) race on the array and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace apsp {

constexpr int kNoAllocMaxGraphs = 65536;
constexpr size_t kNoAllocBytes = 16 + (size_t)kNoAllocMaxGraphs * (4 + 4 + 8);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// One CTA: counting sort of the graphs by decreasing size (ties in any
// order), each entry tagged with its class's variant; also resets the work
// counter.
__global__ void __launch_bounds__(1024)
    fw_batched_order(const int32_t *__restrict__ ns, int num, int32_t *__restrict__ order,
                     int *__restrict__ counter, int v0, int v1, int v2, int v3) {
  __shared__ int start[kBatchedMaxN + 2];
  for (int v = threadIdx.x; v < kBatchedMaxN + 2; v += blockDim.x) start[v] = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < num; g += blockDim.x) atomicAdd(&start[ns[g]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan from the largest size down
    int run = 0;
    for (int v = kBatchedMaxN; v >= 1; --v) {
      const int c = start[v];
      start[v] = run;
      run += c;
    }
    *counter = 0;
  }
  __syncthreads();
  const int var[kNumClasses] = {v0, v1, v2, v3};
  for (int g = threadIdx.x; g < num; g += blockDim.x) {
    const int n = ns[g];
    order[atomicAdd(&start[n], 1)] = g | (var[class_of_n(n)] << 30);
  }
}

}  // namespace apsp

APSP_EXPORT int apsp_fw_batched_f32_noalloc(float *d_dist, int32_t *d_path, const int32_t *h_n,
                                            const int64_t *h_off, int32_t num, void *stream) {
  int st = validate(h_n, h_off, num);
  if (st) return st;
  if (num > apsp::kNoAllocMaxGraphs) return APSP_EUNSUPPORTED;
  if (num == 0) return APSP_OK;
  if (!d_dist) return APSP_EINVAL;
  // The array's device address on the current device, looked up on every call
  // (cheap, allocates nothing) so that it stays right after a device reset
  // reloads the module.  The first call on a device loads the module there.
  void *ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, apsp::g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return APSP_ECUDA;
  }
  unsigned char *base = static_cast<unsigned char *>(ptr);
  int *d_counter = reinterpret_cast<int *>(base);
  int32_t *d_order = reinterpret_cast<int32_t *>(base + 16);
  int32_t *d_n = d_order + apsp::kNoAllocMaxGraphs;
  int64_t *d_off = reinterpret_cast<int64_t *>(d_n + apsp::kNoAllocMaxGraphs);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = grid_for(num, false);
  if (grid <= 0) return APSP_ECUDA;
  cudaGetLastError();
  cudaError_t e = cudaMemcpyAsync(d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return APSP_ECUDA;
  // The 128-block variant needs per-CTA panel space this entry point does not
  // have: its classes run the 64-block variant with the same path tracking.
  int v[apsp::kNumClasses];
  for (int c = 0; c < apsp::kNumClasses; ++c) v[c] = apsp::g_variant[c] == 2 ? 1 : apsp::g_variant[c];
  apsp::fw_batched_order<<<1, 1024, 0, s>>>(d_n, num, d_order, d_counter, v[0], v[1], v[2], v[3]);
  apsp::fw_batched_persistent_f32<<<grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
      d_dist, d_path, d_order, d_n, d_off, num, d_counter, nullptr, 0);
  return apsp::status_from(cudaGetLastError());
}
