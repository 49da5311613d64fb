// Single-graph blocked Floyd-Warshall for sm_103a.
//
// Schedule (§2.2 "Blocked FW Algorithm", kernels as in §3.2): the n x n
// matrix is cut into TB x TB blocks; each of the R = ceil(n / TB) rounds runs
//   K1  fw_phase1_diag      phase 1: the diagonal block (r,r), k sequential;
//   K2  fw_phase2_lines     phases 2+3: the row blocks (r,J) and the column
//                           blocks (I,r), k sequential inside each block;
//   K3  fw_phase3_minplus   phase 4: every other block (I,J) gets
//                           C = min(C, A (x) B) with A = block (I,r) and
//                           B = block (r,J), a min-plus product over the
//                           round's TB values of k.
// Relaxation rule: Algorithm 1 with a strict "<" (see apsp_fw.h).
//
// Rounds overlap: phase 4 of round r first updates row and column r+1, then
// the rest of the matrix while K1/K2 of round r+1 run on a second stream.
//
// Differences from the Pascal design of §3.2 (one output per thread, TB <= 32):
//  * K3 runs two CTAs per 128 x 128 block, three per SM, an 8 x 4 register
//    tile per thread (FP32, TB = 128), and pairs consecutive k: one packed
//    add.rn.f32x2 forms the two candidates of an output and one three-input
//    min.f32 folds both into the accumulator (FADD2 and FMNMX3 run on
//    different pipes).  Operands arrive by bulk copy into a two-stage ring.
//  * Path state: in rounds 0-15 (nearly every output improves) an eager
//    instance of K3 keeps, per output, the k-pair of the last strict decrease
//    as a byte; later rounds keep none in the inner loop, and after the loop
//    the improved outputs recover the first k that attains the new minimum
//    (lane-parallel for dense 8-row groups, warp-cooperative otherwise).
//    Either way P is exactly that of the sequential loop (ascending k, strict
//    "<" keeps the first k reaching the final minimum).
//  * K1 keeps only minima in its step loop and recovers P afterwards from a
//    per-step history; K2 keeps each row/column line in registers.
//  * Nothing reads P: K1/K2/K3 write P only where D strictly improved.
#include <stdint.h>

#include "common.cuh"
#include "bulk.cuh"
#include "minplus_f32.cuh"
#include "phases_f32.cuh"
#include "profile.h"

namespace apsp {

// --------------------------------------------------------------------------
// K0: P := -1 over an n x n region with leading dimension ld.
// --------------------------------------------------------------------------
__global__ void fw_path_init(int32_t *__restrict__ P, int64_t n, int64_t ld) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    P[i * ld + j] = -1;
  }
}

__global__ void __launch_bounds__(k2::THREADS, 2) fw_phase2_lines_f32(float *__restrict__ D, int64_t ld,
                                                                  int32_t *__restrict__ P, int n, int r,
                                                                  int R, Panels pan) {
  using namespace k2;
  const int b = blockIdx.x / PARTS, part = blockIdx.x % PARTS;
  const bool is_row = b < R - 1;
  int other = is_row ? b : b - (R - 1);
  other += (other >= r);
  lines_load_diag(D, ld, n, r, is_row);
  __syncthreads();
  lines_part_f32(D, ld, P, n, r, other, is_row, part, pan);
}

// --------------------------------------------------------------------------
// K1 (FP32): phase 1 with the register-resident closure of minplus_f32.cuh.
// K3 (FP32): phase 4, one 128 x 128 block product per CTA (minplus_f32.cuh).
// Grid: (R-1)^2 CTAs in row-major (I', J') order over the blocks I, J != r,
// so consecutive CTAs share the column-panel block A and sweep the row panel.
// --------------------------------------------------------------------------
// K1 (FP32): Algorithm 1 on the diagonal block, minima only in the step
// loop, path entries recovered afterwards.  Each thread keeps its 8 x 8
// elements in registers; at step k the owners of row k and column k publish
// them into a per-step history in shared memory (k-paired layout:
// hr[k/2][j] = (row 2kp at its step, row 2kp+1 at its step), hc likewise for
// columns), one barrier per step.  Step k never changes row or column k
// (D[k][k] = 0), so the published values are the ones every thread uses.
// Within the round an element's last strict improvement is the first step
// whose candidate hc[k][i] + hr[k][j] equals the element's final value, so
// after the loop each improved element finds that k by scanning its
// candidate sums from the history (folded 8 k at a time, lowest matching
// chunk kept, then the first k inside it) - the P of the sequential loop.
namespace k1 {
constexpr int T = mp32::T, TM = 8;
struct Hist {
  unsigned long long hc[T / 2][T];  // (D[i][2kp], D[i][2kp+1]) as published at steps 2kp, 2kp+1
  unsigned long long hr[T / 2][T];  // (D[2kp][j], D[2kp+1][j]) likewise
};
}  // namespace k1

__global__ void __launch_bounds__(mp32::THREADS)
    fw_phase1_diag_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r) {
  using namespace k1;
  using mp32::col_at;
  using mp32::row_at;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Hist &h = *reinterpret_cast<Hist *>(smem_raw);
  float *hc = reinterpret_cast<float *>(&h.hc[0][0]), *hr = reinterpret_cast<float *>(&h.hr[0][0]);
  const int base = r * T, m = min(T, n - base);
  const int ty = mp32::thread_ty(), tx = mp32::thread_tx();
  const float INF = inf<float>();
  float d[TM][TM];
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int i = row_at(rr, ty), j = col_at(cc, tx);
      d[rr][cc] = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : INF;
    }
  // k = 32 kb + 2 kk + q: row_at / col_at index 2 kb + q of owner kk; k-pair 16 kb + kk.
#pragma unroll
  for (int kb = 0; kb < TM / 2; ++kb) {
#pragma unroll 1
    for (int kk = 0; kk < 16; ++kk) {
      const int kp = 16 * kb + kk;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (ty == kk) {
#pragma unroll
          for (int cc = 0; cc < TM; ++cc) hr[(kp * T + col_at(cc, tx)) * 2 + q] = d[2 * kb + q][cc];
        }
        if (tx == kk) {
#pragma unroll
          for (int rr = 0; rr < TM; ++rr) hc[(kp * T + row_at(rr, ty)) * 2 + q] = d[rr][2 * kb + q];
        }
        __syncthreads();
        float a[TM], b[TM];
#pragma unroll
        for (int rr = 0; rr < TM; ++rr) a[rr] = hc[(kp * T + row_at(rr, ty)) * 2 + q];
#pragma unroll
        for (int cc = 0; cc < TM; ++cc) b[cc] = hr[(kp * T + col_at(cc, tx)) * 2 + q];
#pragma unroll
        for (int rr = 0; rr < TM; ++rr) {
          const unsigned long long aa = mp32::pack2(a[rr], a[rr]);
#pragma unroll
          for (int c2 = 0; c2 < TM / 2; ++c2) {
            const float2 cand = mp32::sum2(aa, mp32::pack2(b[2 * c2], b[2 * c2 + 1]));
            d[rr][2 * c2] = fminf(d[rr][2 * c2], cand.x);
            d[rr][2 * c2 + 1] = fminf(d[rr][2 * c2 + 1], cand.y);
          }
        }
      }
    }
  }
  // D where improved (the old value is still in global memory).
  unsigned long long imp = 0ull;  // bit 8 rr + cc
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      const int i = row_at(rr, ty), j = col_at(cc, tx);
      if (i < m && j < m) {
        const int64_t g = (int64_t)(base + i) * ld + base + j;
        if (d[rr][cc] < D[g]) {
          D[g] = d[rr][cc];
          imp |= 1ull << (TM * rr + cc);
        }
      }
    }
  if (!P || __syncthreads_count(imp != 0ull) == 0) return;  // the history is complete past this barrier
  if (imp == 0ull) return;
  // P: lowest 8-k chunk (4 k-pairs) whose minimum candidate equals the final
  // value, then the first k inside it.  Chunks are walked from high to low
  // and the byte of an element is overwritten on every match.
  unsigned ch[TM][TM / 4];
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int c4 = 0; c4 < TM / 4; ++c4) ch[rr][c4] = 0u;
#pragma unroll 1
  for (int c = T / 8 - 1; c >= 0; --c) {
    unsigned long long bq[4][TM];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int cc = 0; cc < TM; ++cc) bq[q][cc] = h.hr[4 * c + q][col_at(cc, tx)];
#pragma unroll
    for (int rr = 0; rr < TM; ++rr) {
      unsigned long long aq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) aq[q] = h.hc[4 * c + q][row_at(rr, ty)];
#pragma unroll
      for (int cc = 0; cc < TM; ++cc) {
        const float2 s0 = mp32::sum2(aq[0], bq[0][cc]), s1 = mp32::sum2(aq[1], bq[1][cc]);
        const float2 s2 = mp32::sum2(aq[2], bq[2][cc]), s3 = mp32::sum2(aq[3], bq[3][cc]);
        float mm = mp32::min3f(s0.x, s0.y, s1.x);
        mm = mp32::min3f(mm, s1.y, s2.x);
        mm = mp32::min3f(mm, s2.y, s3.x);
        mm = fminf(mm, s3.y);
        if (mm == d[rr][cc])
          ch[rr][cc / 4] = __byte_perm(ch[rr][cc / 4], (unsigned)c,
                                       0x3210 ^ ((0x3210 & (0xF << (4 * (cc & 3)))) ^ (4 << (4 * (cc & 3)))));
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < TM; ++rr)
#pragma unroll
    for (int cc = 0; cc < TM; ++cc) {
      if (!((imp >> (TM * rr + cc)) & 1ull)) continue;
      const int c = (ch[rr][cc / 4] >> (8 * (cc & 3))) & 0xFF;  // an improved element's chunk
      const int i = row_at(rr, ty), j = col_at(cc, tx);
      int kf = 8 * c + 7;
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        const float2 sv = mp32::sum2(h.hc[4 * c + q][i], h.hr[4 * c + q][j]);
        kf = sv.y == d[rr][cc] ? 8 * c + 2 * q + 1 : kf;
        kf = sv.x == d[rr][cc] ? 8 * c + 2 * q : kf;
      }
      P[(int64_t)(base + i) * ld + base + j] = base + kf;
    }
}

template <bool EAGER>
__global__ void __launch_bounds__(mp32::THREADS, EAGER ? APSP_K3_EAGER_MIN_BLOCKS : APSP_K3_MIN_BLOCKS)
    fw_phase3_minplus_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r,
                          int R, int vec_ok, Panels pan, int set) {
  using namespace k3;
  using mp32::col_at;
  using mp32::row_at;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  const int Rm = R - 1, tile = blockIdx.x >> 1, hJ = blockIdx.x & 1;
  int I, J;
  if (set == kSetAll) {  // every block off row and column r
    I = tile / Rm;
    J = tile % Rm;
    I += (I >= r);
    J += (J >= r);
  } else if (set == kSetNext) {  // row r+1, then column r+1: the next round's K1/K2 input
    if (tile < Rm) {
      I = r + 1;
      J = tile + (tile >= r);
    } else {
      I = tile - Rm;
      I += (I >= r);
      I += (I >= r + 1);
      J = r + 1;
    }
  } else {  // the rest: rows and columns other than r and r+1
    I = tile / (R - 2);
    J = tile % (R - 2);
    I += (I >= r);
    I += (I >= r + 1);
    J += (J >= r);
    J += (J >= r + 1);
  }
  const int baseI = I * T, baseJ = J * T + hJ * H, baseK = r * T;
  const int mI = min(T, n - baseI), mJ = min(H, n - baseJ), mK = min(T, n - baseK);
  if (mJ <= 0) return;  // empty half of the last (narrow) block; uniform exit
  const int nslab = (mK + KS - 1) / KS;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ty = mp32::thread_ty(), tx = mp32::thread_tx();
  const float INF = inf<float>();
  const unsigned long long *srcA = pan.Apan + (int64_t)I * (T / 2) * T;
  const unsigned long long *srcB = pan.Bpan + ((int64_t)J * 2 + hJ) * (T / 2) * H;

  if (tid == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(&sm.bar[st], 1);
    fence_mbar_init();
    for (int s = 0; s < STAGES && s < nslab; ++s) {
      mbar_expect_tx(&sm.bar[s], A_SLAB + B_SLAB);
      bulk_g2s(&sm.As[s][0][0], srcA + (int64_t)s * KP * T, A_SLAB, &sm.bar[s]);
      bulk_g2s(&sm.Bs[s][0][0], srcB + (int64_t)s * KP * H, B_SLAB, &sm.bar[s]);
    }
  }
  __syncthreads();

  float acc[8][4];
  unsigned kid[8];  // EAGER: byte c of kid[a] = the round's k-pair of the last strict decrease, 0xFF none
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    kid[a] = 0xFFFFFFFFu;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = INF;
  }

  for (int s = 0; s < nslab; ++s) {
    const int st = s % STAGES;
    const bool ok = mbar_wait(&sm.bar[st], (s / STAGES) & 1);
    if (__syncthreads_or(!ok)) {
      // A copy never completed: record it, wait (bounded) for the other
      // copies this CTA issued, and leave without touching D or P.
      if (tid == 0) {
        report_wait_timeout();
        for (int s2 = s + 1; s2 < nslab && s2 < s + STAGES; ++s2)
          mbar_wait(&sm.bar[s2 % STAGES], (s2 / STAGES) & 1);
      }
      return;
    }
    // Operand loads are software-pipelined by hand: the B pairs of k-pair
    // kp+1 load while kp computes (two named buffers, k-pairs two at a time),
    // and each A row-pair loads one row-pair ahead of its use.
    const unsigned long long *Asl = &sm.As[st][0][0];
    const unsigned long long *Bsl = &sm.Bs[st][0][0];
    auto load_b = [&](int kp, unsigned long long (&b)[4]) {
#pragma unroll
      for (int cc = 0; cc < 4; cc += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&Bsl[kp * H + col_at(cc, tx)]);
        b[cc] = t.x;
        b[cc + 1] = t.y;
      }
    };
    const unsigned kbase = (unsigned)(s * KP);
    auto compute = [&](int kp, const unsigned long long (&b)[4]) {
      ulonglong2 an = *reinterpret_cast<const ulonglong2 *>(&Asl[kp * T + row_at(0, ty)]);
#pragma unroll
      for (int rp = 0; rp < 4; ++rp) {
        const ulonglong2 ac = an;
        if (rp < 3) an = *reinterpret_cast<const ulonglong2 *>(&Asl[kp * T + row_at(2 * rp + 2, ty)]);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          if constexpr (EAGER) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float m = mp32::min3f_pair(acc[2 * rp + h][cc], h ? ac.y : ac.x, b[cc]);
              if (m < acc[2 * rp + h][cc])
                kid[2 * rp + h] = __byte_perm(kid[2 * rp + h], kbase + kp,
                                              0x3210 ^ ((0x3210 & (0xF << (4 * cc))) ^ (4 << (4 * cc))));
              acc[2 * rp + h][cc] = m;
            }
          } else {
            mp32::relax2(acc[2 * rp][cc], ac.x, b[cc]);
            mp32::relax2(acc[2 * rp + 1][cc], ac.y, b[cc]);
          }
        }
      }
    };
    unsigned long long b0[4], b1[4];
    load_b(0, b0);
    if constexpr (EAGER) {
      // Both k-pairs of a step per output, one compare and one byte permute
      // per four candidates: the byte keeps the step's first k-pair.
      auto compute2 = [&](int kp, const unsigned long long (&p0)[4], const unsigned long long (&p1)[4]) {
        ulonglong2 n0 = *reinterpret_cast<const ulonglong2 *>(&Asl[kp * T + row_at(0, ty)]);
        ulonglong2 n1 = *reinterpret_cast<const ulonglong2 *>(&Asl[(kp + 1) * T + row_at(0, ty)]);
#pragma unroll
        for (int rp = 0; rp < 4; ++rp) {
          const ulonglong2 c0 = n0, c1 = n1;
          if (rp < 3) {
            n0 = *reinterpret_cast<const ulonglong2 *>(&Asl[kp * T + row_at(2 * rp + 2, ty)]);
            n1 = *reinterpret_cast<const ulonglong2 *>(&Asl[(kp + 1) * T + row_at(2 * rp + 2, ty)]);
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float &acc_o = acc[2 * rp + h][cc];
              const float m1 = mp32::min3f_pair(acc_o, h ? c0.y : c0.x, p0[cc]);
              const float m2 = mp32::min3f_pair(m1, h ? c1.y : c1.x, p1[cc]);
              if (m2 < acc_o)
                kid[2 * rp + h] = __byte_perm(kid[2 * rp + h], kbase + kp,
                                              0x3210 ^ ((0x3210 & (0xF << (4 * cc))) ^ (4 << (4 * cc))));
              acc_o = m2;
            }
        }
      };
#pragma unroll 4
      for (int kp = 0; kp < KP; kp += 2) {
        load_b(kp + 1, b1);
        compute2(kp, b0, b1);
        if (kp + 2 < KP) load_b(kp + 2, b0);
      }
    } else {
// Unrolled by four (measured best of 1, 2, 4 and 8).
#pragma unroll 4
    for (int kp = 0; kp < KP; kp += 2) {
      load_b(kp + 1, b1);
      compute(kp, b0);
      if (kp + 2 < KP) load_b(kp + 2, b0);
      compute(kp + 1, b1);
    }
    }
    __syncthreads();  // stage st fully read
    if (tid == 0 && s + STAGES < nslab) {
      fence_proxy_async_smem();
      const int s2 = s + STAGES;
      mbar_expect_tx(&sm.bar[st], A_SLAB + B_SLAB);
      bulk_g2s(&sm.As[st][0][0], srcA + (int64_t)s2 * KP * T, A_SLAB, &sm.bar[st]);
      bulk_g2s(&sm.Bs[st][0][0], srcB + (int64_t)s2 * KP * H, B_SLAB, &sm.bar[st]);
    }
  }

  // Epilogue.  The ring is free now: the half block of new candidates goes to
  // shared memory so that the rest runs as compact loops with each warp
  // owning 16 whole rows (lane l: columns 2l, 2l+1), which keeps the code small
  // (instruction-cache friendly) and every global access coalesced.
  float *Cs = reinterpret_cast<float *>(smem_raw);  // [T][H]
  unsigned char *Ks = smem_raw + sizeof(Smem::As);  // EAGER: [T][H] k-pair bytes, in the B ring
  __syncthreads();
#pragma unroll
  for (int rr = 0; rr < 8; ++rr)
#pragma unroll
    for (int cc = 0; cc < 4; cc += 2) {
      *reinterpret_cast<float2 *>(&Cs[row_at(rr, ty) * H + col_at(cc, tx)]) =
          make_float2(acc[rr][cc], acc[rr][cc + 1]);
      if constexpr (EAGER)
        *reinterpret_cast<unsigned short *>(&Ks[row_at(rr, ty) * H + col_at(cc, tx)]) =
            (unsigned short)(kid[rr] >> (8 * cc));
    }
  __syncthreads();
  const float *acp = pan.Acp + (int64_t)I * T * T;
  const float *bt = pan.Bt + ((int64_t)J * T + hJ * H) * T;
  const int w = tid >> 5, j0 = 2 * lane, i0 = w * 16;
  const bool vec = vec_ok && j0 + 1 < mJ;
  // Pass 1 (unrolled): all 16 old rows of the warp are loaded before any is
  // used (one memory round trip), improvements are flagged and written.
  float2 o[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const float *row = D + (int64_t)(baseI + i0 + t) * ld + baseJ;
    o[t] = make_float2(INF, INF);
    if (i0 + t < mI) {
      if (vec) {
        o[t] = *reinterpret_cast<const float2 *>(row + j0);
      } else {
        if (j0 < mJ) o[t].x = row[j0];
        if (j0 + 1 < mJ) o[t].y = row[j0 + 1];
      }
    }
  }
  unsigned flags = 0u;  // bit 2t + q: row i0 + t, column j0 + q improved
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    if (i0 + t >= mI) continue;
    const float2 c = *reinterpret_cast<const float2 *>(&Cs[(i0 + t) * H + j0]);
    unsigned imp = 0u;
    if (j0 < mJ && c.x < o[t].x) imp |= 1u;
    if (j0 + 1 < mJ && c.y < o[t].y) imp |= 2u;
    if (!imp) continue;
    flags |= imp << (2 * t);
    float *row = D + (int64_t)(baseI + i0 + t) * ld + baseJ;
    if (vec) {
      *reinterpret_cast<float2 *>(row + j0) = make_float2(imp & 1 ? c.x : o[t].x, imp & 2 ? c.y : o[t].y);
    } else {
      if (imp & 1) row[j0] = c.x;
      if (imp & 2) row[j0 + 1] = c.y;
    }
  }
  if (!P) return;
  if constexpr (EAGER) {
    // The k inside each improved output's last decreasing step (two k-pairs):
    // the first whose candidate equals the new value (the sequential loop
    // keeps the first k reaching a minimum).
#pragma unroll 1
    for (int t = 0; t < 16; ++t)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!((flags >> (2 * t + q)) & 1u)) continue;
        const int i = i0 + t, j = j0 + q;
        const int kp = Ks[i * H + j];  // an improved output has one
        const float g = Cs[i * H + j];
        const float2 c = mp32::sum2(srcA[(int64_t)kp * T + i], srcB[(int64_t)kp * H + j]);
        int k;
        if (c.x == g) {
          k = 2 * kp;
        } else if (c.y == g) {
          k = 2 * kp + 1;
        } else {  // the second k-pair of the step
          const float2 c2 = mp32::sum2(srcA[(int64_t)(kp + 1) * T + i], srcB[(int64_t)(kp + 1) * H + j]);
          k = c2.x == g ? 2 * kp + 2 : 2 * kp + 3;
        }
        P[(int64_t)(baseI + i) * ld + baseJ + j] = baseK + k;
      }
    return;
  }
  // Pass 2a: each 8-row group of the warp with many improved outputs (the
  // early rounds, where most outputs improve) is resolved lane-parallel: lane
  // l scans the 128 candidates of its own two columns in the paired panel
  // layout the main loop read (B pairs coalesced, A pairs broadcast), folds
  // every 8 k into one minimum with three-input mins, keeps the lowest 8-k
  // chunk whose minimum equals the output's new value, and finds the first
  // such k inside that chunk.  The operands stream from L2 once per group
  // instead of once per improved output.
  {
    const unsigned long long *pa = srcA + i0, *pb = srcB + j0;
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {
      const unsigned gm = 0xFFFFu << (16 * G);
      if ((int)__reduce_add_sync(kFullMask, (unsigned)__popc(flags & gm)) < kDenseMin) continue;
      const int tg0 = 8 * G;
      float g[8][2];
      unsigned hit[8];  // bit c (+16 for column j0 + 1): chunk c's minimum equals g
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 c = *reinterpret_cast<const float2 *>(&Cs[(i0 + tg0 + t) * H + j0]);
        g[t][0] = c.x;
        g[t][1] = c.y;
        hit[t] = 0u;
      }
#pragma unroll 1
      for (int c = T / 8 - 1; c >= 0; --c) {
        ulonglong2 b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = __ldg(reinterpret_cast<const ulonglong2 *>(pb + (4 * c + q) * H));
        const unsigned bit = 1u << c;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          unsigned long long a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = __ldg(pa + (4 * c + q) * T + tg0 + t);
#pragma unroll
          for (int q2 = 0; q2 < 2; ++q2) {
            float2 s0 = mp32::sum2(a[0], q2 ? b[0].y : b[0].x), s1 = mp32::sum2(a[1], q2 ? b[1].y : b[1].x);
            float2 s2 = mp32::sum2(a[2], q2 ? b[2].y : b[2].x), s3 = mp32::sum2(a[3], q2 ? b[3].y : b[3].x);
            float m = mp32::min3f(s0.x, s0.y, s1.x);
            m = mp32::min3f(m, s1.y, s2.x);
            m = mp32::min3f(m, s2.y, s3.x);
            m = fminf(m, s3.y);
            if (m == g[t][q2]) hit[t] |= bit << (16 * q2);
          }
        }
      }
      // Resolution: both outputs of a row load their chunk's eight operand
      // pairs at once (one memory round trip per row); a descending select
      // chain keeps the first k whose sum equals g.
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const unsigned fl = (flags >> (2 * (tg0 + t))) & 3u;
        if (!fl) continue;
        int c[2];
        unsigned long long av[2][4], bv[2][4];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          // an improved output's chunk mask is not empty: g is one of the sums
          c[q2] = ((fl >> q2) & 1u) ? __ffs((hit[t] >> (16 * q2)) & 0xFFFFu) - 1 : 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            av[q2][q] = __ldg(pa + (4 * c[q2] + q) * T + tg0 + t);
            bv[q2][q] = __ldg(pb + (4 * c[q2] + q) * H + q2);
          }
        }
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          if (!((fl >> q2) & 1u)) continue;
          int k = 8 * c[q2] + 7;
#pragma unroll
          for (int q = 3; q >= 0; --q) {
            const float2 sv = mp32::sum2(av[q2][q], bv[q2][q]);
            k = sv.y == g[t][q2] ? 8 * c[q2] + 2 * q + 1 : k;
            k = sv.x == g[t][q2] ? 8 * c[q2] + 2 * q : k;
          }
          P[(int64_t)(baseI + i0 + tg0 + t) * ld + baseJ + j0 + q2] = baseK + k;
        }
      }
      flags &= ~gm;
    }
  }
  // Pass 2b: P for every remaining improved output.  The warp walks them
  // (all rows, all lanes) as one stream, four at a time: the A-row and B-row
  // loads of the four are issued together (one memory round trip per group),
  // then for each output lane l tests k = 4l..4l+3 and the lowest hit wins.
  unsigned wf = __reduce_or_sync(kFullMask, flags);
  unsigned bal = 0u;
  int pos = 0;
  auto next = [&](int &t, int &sj) -> bool {  // warp-uniform
    while (!bal) {
      if (!wf) return false;
      pos = __ffs(wf) - 1;
      wf &= wf - 1;
      bal = __ballot_sync(kFullMask, (flags >> pos) & 1u);
    }
    const int src = __ffs(bal) - 1;
    bal &= bal - 1;
    t = pos >> 1;
    sj = 2 * src + (pos & 1);
    return true;
  };
#pragma unroll 1
  for (;;) {
    int t[4], sj[4];
    bool v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = next(t[u], sj[u]);
    if (!v[0]) break;
    float4 av[4], bv[4];
    float tg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!v[u]) continue;
      av[u] = reinterpret_cast<const float4 *>(acp + (i0 + t[u]) * T)[lane];
      bv[u] = reinterpret_cast<const float4 *>(bt + sj[u] * T)[lane];
      tg[u] = Cs[(i0 + t[u]) * H + sj[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!v[u]) continue;
      const float g = tg[u];
      const unsigned h = (__fadd_rn(av[u].x, bv[u].x) == g ? 1u : 0u) |
                         (__fadd_rn(av[u].y, bv[u].y) == g ? 2u : 0u) |
                         (__fadd_rn(av[u].z, bv[u].z) == g ? 4u : 0u) |
                         (__fadd_rn(av[u].w, bv[u].w) == g ? 8u : 0u);
      const unsigned hb = __ballot_sync(kFullMask, h != 0);
      const int L = __ffs(hb) - 1;  // hb != 0: g is one of the candidates
      const unsigned hL = __shfl_sync(kFullMask, h, L & 31);
      if (lane == 0 && hb)
        P[(int64_t)(baseI + i0 + t[u]) * ld + baseJ + sj[u]] = baseK + 4 * L + (__ffs(hL) - 1);
    }
  }
}

// Phase timing state (see profile.h).
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<PhaseRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;

// --------------------------------------------------------------------------
// Host side: argument checks and the round loop (all launches on `stream`).
// --------------------------------------------------------------------------
// Largest n: vertex indices and block coordinates stay in 32-bit integers,
// element offsets are 64-bit.  In practice device memory bounds n first
// (FP32 D + P take 8 n^2 bytes: 128 GiB at n = 131072).
constexpr int kMaxN = 1 << 18;

constexpr int kT32 = mp32::T, kT64 = 128;
static int g_smem_k1f[64], g_smem_p2f[64], g_smem_k3[64], g_smem_k3e[64];

int run_fw_f64_interval(double *D, int n, int64_t ld, int32_t *P, cudaStream_t s);
int take_device_error_f64();
int take_device_error_checks();
int take_device_error_int32();

static void path_init(int32_t *P, int64_t n, int64_t ld, cudaStream_t s) {
  const int64_t total = n * n;
  const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
  PhaseScope ps(0, s);
  fw_path_init<<<blocks, 256, 0, s>>>(P, n, ld);
}

static int check_args(const void *D, int64_t n, int64_t ld) {
  if (n < 0 || n > kMaxN) return APSP_EINVAL;
  if (n == 0) return APSP_OK;
  if (!D || ld < n) return APSP_EINVAL;
  return APSP_OK;
}

static int run_fw_f32(float *D, int64_t n64, int64_t ld, int32_t *P, void *stream) {
  int st = check_args(D, n64, ld);
  if (st || n64 == 0) return st;
  const int n = (int)n64;
  constexpr int T = kT32;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if ((st = ensure_smem(fw_phase1_diag_f32, (int)sizeof(k1::Hist), g_smem_k1f))) return st;
  if ((st = ensure_smem(fw_phase2_lines_f32, k2::SMEM, g_smem_p2f))) return st;
  if ((st = ensure_smem(fw_phase3_minplus_f32<false>, (int)sizeof(k3::Smem), g_smem_k3))) return st;
  if ((st = ensure_smem(fw_phase3_minplus_f32<true>, (int)sizeof(k3::Smem), g_smem_k3e))) return st;
  cudaGetLastError();  // clear any stale error so the checks below are ours
  const int R = (n + T - 1) / T;
  // Phase-4 operand panels, written by K2 each round: two sets (round parity)
  // of 4 arrays of R*T*T 4-byte words, so that K2 of round r+1 can run while
  // phase 4 of round r still reads round r's panels.  Stream-ordered scratch,
  // freed after the last round.
  Panels pan[2]{};
  char *scratch = nullptr;
  if (R > 1) {
    const size_t words = (size_t)R * T * T;
    if (cudaMallocAsync((void **)&scratch, 8 * words * 4, s) != cudaSuccess) {
      cudaGetLastError();
      return APSP_ENOMEM;
    }
    for (int q = 0; q < 2; ++q) {
      char *base = scratch + (size_t)q * 4 * words * 4;
      pan[q].Apan = reinterpret_cast<unsigned long long *>(base);
      pan[q].Bpan = reinterpret_cast<unsigned long long *>(base + words * 4);
      pan[q].Acp = reinterpret_cast<float *>(base + 2 * words * 4);
      pan[q].Bt = reinterpret_cast<float *>(base + 3 * words * 4);
    }
  }
  if (P) path_init(P, n64, ld, s);
  const int vec_ok = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
  auto diag_and_panels = [&](int r, cudaStream_t st) {
    {
      PhaseScope ps(1, st);
      fw_phase1_diag_f32<<<1, mp32::THREADS, sizeof(k1::Hist), st>>>(D, ld, P, n, r);
    }
    if (R > 1) {
      PhaseScope ps(2, st);
      fw_phase2_lines_f32<<<2 * (R - 1) * k2::PARTS, k2::THREADS, k2::SMEM, st>>>(D, ld, P, n, r, R, pan[r & 1]);
    }
  };
  auto phase4 = [&](int r, int set, int blocks) {
    if (blocks <= 0) return;
    PhaseScope ps(3, s);
    if (P && r < kEagerRounds)
      fw_phase3_minplus_f32<true><<<2 * blocks, mp32::THREADS, sizeof(k3::Smem), s>>>(D, ld, P, n, r, R, vec_ok,
                                                                                   pan[r & 1], set);
    else
      fw_phase3_minplus_f32<false><<<2 * blocks, mp32::THREADS, sizeof(k3::Smem), s>>>(D, ld, P, n, r, R, vec_ok,
                                                                                    pan[r & 1], set);
  };
  // Look-ahead: phase 4 of round r first updates row and column r+1 (the
  // blocks K1/K2 of round r+1 read), then the rest of the matrix while K1/K2
  // of round r+1 run on a second, higher-priority stream; the two touch
  // disjoint blocks and write/read different panel sets.
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_next = nullptr, ev_panels = nullptr;
  // While the caller's stream is being captured into a CUDA graph every
  // phase stays on that stream (no stream is created or destroyed mid-capture).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    if (scratch) cudaFreeAsync(scratch, s);
    cudaGetLastError();
    return APSP_ECUDA;
  }
  if (R > 2 && cap == cudaStreamCaptureStatusNone) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_next, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_panels, cudaEventDisableTiming) != cudaSuccess) {
      if (s2) cudaStreamDestroy(s2);
      if (ev_next) cudaEventDestroy(ev_next);
      if (scratch) cudaFreeAsync(scratch, s);
      cudaGetLastError();
      return APSP_ECUDA;
    }
  }
  diag_and_panels(0, s);
  for (int r = 0; r < R; ++r) {
    if (R == 1) break;
    if (r + 1 < R && s2) {
      phase4(r, k3::kSetNext, 2 * R - 3);
      cudaEventRecord(ev_next, s);
      cudaStreamWaitEvent(s2, ev_next, 0);
      diag_and_panels(r + 1, s2);
      cudaEventRecord(ev_panels, s2);
      phase4(r, k3::kSetRest, (R - 2) * (R - 2));
      cudaStreamWaitEvent(s, ev_panels, 0);
    } else {
      phase4(r, k3::kSetAll, (R - 1) * (R - 1));
      if (r + 1 < R) diag_and_panels(r + 1, s);
    }
  }
  if (s2) {
    cudaStreamDestroy(s2);
    cudaEventDestroy(ev_next);
    cudaEventDestroy(ev_panels);
  }
  cudaError_t e = cudaGetLastError();
  if (scratch) {
    cudaError_t f = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = f;
  }
  return status_from(e);
}

static int run_fw_f64(double *D, int64_t n64, int64_t ld, int32_t *P, void *stream) {
  int st = check_args(D, n64, ld);
  if (st || n64 == 0) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (P) path_init(P, n64, ld, s);
  return run_fw_f64_interval(D, (int)n64, ld, P, s);
}

}  // namespace apsp

APSP_EXPORT int apsp_fw_f32(float *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream) {
  return apsp::run_fw_f32(d_dist, n, ld, d_path, stream);
}

APSP_EXPORT int apsp_fw_f64(double *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream) {
  return apsp::run_fw_f64(d_dist, n, ld, d_path, stream);
}

APSP_EXPORT int apsp_fw_block_size(int elem_bytes) {
  return elem_bytes == 4 ? apsp::kT32 : elem_bytes == 8 ? apsp::kT64 : 0;
}

APSP_EXPORT const char *apsp_status_string(int status) {
  switch (status) {
    case APSP_OK: return "APSP_OK";
    case APSP_EINVAL: return "APSP_EINVAL: invalid argument";
    case APSP_ECUDA: return "APSP_ECUDA: CUDA call or launch failed";
    case APSP_ENOMEM: return "APSP_ENOMEM: device allocation failed";
    case APSP_EUNSUPPORTED: return "APSP_EUNSUPPORTED: outside supported sizes";
    case APSP_ETOODEEP: return "APSP_ETOODEEP: path recursion deeper than the walk stack";
    case APSP_ENEGCYCLE: return "APSP_ENEGCYCLE: negative cycle (a diagonal distance is below 0)";
    case APSP_ETIMEOUT: return "APSP_ETIMEOUT: a kernel's bounded wait for an asynchronous copy ran out";
    default: return "APSP: unknown status";
  }
}

APSP_EXPORT int apsp_version(void) { return 100; }

APSP_EXPORT int apsp_profile_enable(int on) {
  std::lock_guard<std::mutex> g(apsp::g_prof_mu);
  if (on) {  // a new recording starts: recycle the old records' events
    for (auto &r : apsp::g_prof_recs) {
      apsp::g_prof_pool.push_back(r.a);
      apsp::g_prof_pool.push_back(r.b);
    }
    apsp::g_prof_recs.clear();
  }
  apsp::g_prof_on = on != 0;
  return APSP_OK;
}

APSP_EXPORT int apsp_profile_collect(double *ms, int64_t *launches) {
  if (!ms || !launches) return APSP_EINVAL;
  for (int p = 0; p < 4; ++p) {
    ms[p] = 0.0;
    launches[p] = 0;
  }
  std::lock_guard<std::mutex> g(apsp::g_prof_mu);
  for (auto &r : apsp::g_prof_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return APSP_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return APSP_ECUDA;
    ms[r.phase] += t;
    launches[r.phase] += 1;
  }
  return APSP_OK;
}

APSP_EXPORT int apsp_profile_records(int32_t *phase, float *ms, int64_t cap, int64_t *count) {
  if (!count || cap < 0 || (cap > 0 && (!phase || !ms))) return APSP_EINVAL;
  std::lock_guard<std::mutex> g(apsp::g_prof_mu);
  int64_t i = 0;
  for (auto &r : apsp::g_prof_recs) {
    if (i < cap) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) return APSP_ECUDA;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return APSP_ECUDA;
      phase[i] = r.phase;
      ms[i] = t;
    }
    ++i;
  }
  *count = i;
  return APSP_OK;
}

APSP_EXPORT int apsp_device_status(void *stream) {
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return APSP_ECUDA;
  const int v = apsp::take_tu_device_error();
  const int v64 = apsp::take_device_error_f64();
  const int vc = apsp::take_device_error_checks();
  const int vi = apsp::take_device_error_int32();
  return v != 0 ? v : v64 != 0 ? v64 : vc != 0 ? vc : vi;
}
