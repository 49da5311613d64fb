// FP64 blocked Floyd-Warshall for sm_103a, exact, on the FP32 pipes.
//
// GB300 executes FP64 adds and mins at about 2 per clock per SM, 1/64 of its
// FP32 rate, so a native FP64 min-plus product runs ~60x slower than FP32.
// This path keeps every result bit-exact with IEEE FP64 (round to nearest)
// while doing almost all of the work in FP32:
//
//  * each FP64 operand x is held as the float interval [rd(x), ru(x)]
//    (largest float <= x, smallest float >= x);
//  * a candidate a + b then lies in [lo, up] with lo = rd(rd(a) + rd(b)) and
//    up = ru(ru(a) + ru(b)) (add.rm / add.rp), and so does its FP64 rounding
//    fl(a + b), since rounding is monotone;
//  * the min-plus product runs on the lower bounds alone (one packed
//    add.rm.f32x2 and one three-input min per two candidates, as the FP32
//    kernel) and keeps X = min lo per output.  If X >= ru(old) nothing can
//    beat the old value.  Otherwise the exact FP64 minimum is X when some
//    candidate with lo = X has an exact sum X (its upper bound is X, or one
//    FP64 add says so; integer-valued weights always land here), and the
//    first such k is the path entry; if none has, the candidates with
//    lo <= min(ru(old), their up) are evaluated with a real FP64 add.
//
// Schedule per round r (TB = 128), the blocked FW of §2.2, every phase in the
// paper's k order:
//  K1  fw64_diag         phase 1: Algorithm 1 on block (r,r), k sequential,
//                        with the interval filter per relaxation.
//  K2  fw64_lines        phases 2 and 3: the row blocks (r,J) and column
//                        blocks (I,r), k sequential per line with the same
//                        filter; packs the finished blocks as phase-4 operands.
//  K3  fw64_product      phase 4: (I,J) <- min(C, D(I,r) (x) D(r,J)); rounds
//                        0-15 run an eager instance that also keeps, per
//                        output, the k-pair where min lo last decreased.
// As in the FP32 path, phase 4 of round r updates row and column r+1 first,
// then the rest while K1/K2 of round r+1 run on a second stream.
// Every candidate sum is one IEEE FP64 addition rounded to nearest, taken in
// the order of the sequential blocked FW, so D and P are bit-exact with it on
// any weights (and with every correct FW on integer-valued weights).
#include <float.h>
#include <stdint.h>

#include "bulk.cuh"
#include "common.cuh"
#include "profile.h"

namespace apsp {
namespace f64 {

constexpr int T = 128;
constexpr int THREADS = 256;  // product: 8 warps, 4 x 8 outputs per thread, 128 x 64 per CTA
constexpr int H = T / 2;      // output columns per CTA (one half of a block)
constexpr int KS = 32, KP = 16, STAGES = 2;
constexpr uint32_t SLAB_BYTES = KP * H * 8;  // one half of one paired array, one slab
#ifndef APSP_F64_DENSE_MIN
#define APSP_F64_DENSE_MIN 40
#endif
// Quick improvements (of 512) above which an 8-row group takes recovery pass 2a.
constexpr int kDenseMin64 = APSP_F64_DENSE_MIN;

// One operand block packed for the product kernel.  For an A operand
// (A[i][k]): lo[i/64][kp][i%64] = (rd A[i][2kp], rd A[i][2kp+1]), hi likewise
// with ru, rlo[i][k] = rd A[i][k], rhi[i][k] = ru A[i][k], r64[i][k] = A[i][k].
// For a B operand (B[k][j]): lo[j/64][kp][j%64] = (rd B[2kp][j],
// rd B[2kp+1][j]), ..., rlo[j][k] = rd B[k][j], rhi[j][k], r64[j][k] = B[k][j]
// (transposed).  The paired arrays are split in two 64-wide halves so that a
// 16-k-pair slab of one half is one contiguous 8 KiB piece.  Entries outside
// the matrix hold +inf.
// 128-byte aligned so that every pack of an array starts on a 16-byte
// boundary (bulk copies and 16-byte loads read from it).
struct __align__(128) Pack {
  unsigned long long lo[2][T / 2][T / 2];
  unsigned long long hi[2][T / 2][T / 2];
  float rlo[T][T];
  float rhi[T][T];
  double r64[T][T];
  int exact;  // 1: every value is a float (rlo == rhi), so upper bounds follow from rlo
};

// ---------------------------------------------------------------- bounds
// Largest float <= x and smallest float >= x for any non-NaN double, from the
// bit pattern (integer pipes only).  Tight in the normal float range; below
// it the bound is loosened to 0 / +-FLT_MIN, which keeps it valid.
__device__ __forceinline__ float f64_up(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if ((b << 1) == 0) return 0.0f;
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ff);
  if (e == 0x7ff) return sign ? -__int_as_float(0x7f800000) : __int_as_float(0x7f800000);
  const int fe = e - 1023 + 127;
  if (fe >= 255) return sign ? -FLT_MAX : __int_as_float(0x7f800000);
  if (fe <= 0) return sign ? -0.0f : FLT_MIN;
  const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned f = sign | ((unsigned)fe << 23) | m23;  // toward zero
  if ((lo & 0x1fffffffu) && !sign) f += 1u;
  return __uint_as_float(f);
}

__device__ __forceinline__ float f64_down(double x) { return -f64_up(-x); }

// Exact x < d for a float x and a double d (no NaN).  Equal to x < ru(d),
// since a float below d is below the smallest float >= d.  Both non-negative
// with x normal: the doubles' bit patterns order as unsigned integers, so x's
// double pattern is built (exponent rebiased, mantissa shifted) and compared.
__device__ __forceinline__ bool f32_lt_f64(float x, double d) {
  const unsigned ux = __float_as_uint(x);
  const unsigned long long ud = (unsigned long long)__double_as_longlong(d);
  const unsigned e = ux >> 23;  // sign bit clear: the biased exponent
  if (!(ud >> 63) && e - 1u < 254u) {
    const unsigned long long bx = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(ux & 0x7fffffu) << 29);
    return bx < ud;
  }
  return x < f64_up(d);
}

// Exact float -> double bits (integer pipes; subnormal floats via cvt).
__device__ __forceinline__ unsigned long long f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xff;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) {
    if ((u & 0x7fffffu) == 0) return sign;
    return (unsigned long long)__double_as_longlong((double)f);
  }
  if (e == 0xff) return sign | 0x7ff0000000000000ull | ((unsigned long long)(u & 0x7fffffu) << 29);
  return sign | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
}

// Signed integer key with the order of the doubles (-0 sorts just below +0;
// neither arises from sums of the non-negative-cycle inputs except -0 + -0).
__device__ __forceinline__ long long dkey(unsigned long long b) {
  return (long long)(b ^ ((unsigned long long)((long long)b >> 63) >> 1));
}
__device__ __forceinline__ unsigned long long dkey_bits(long long k) {
  return (unsigned long long)k ^ ((unsigned long long)(k >> 63) >> 1);
}

__device__ __forceinline__ unsigned long long packf2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// Lower- and upper-bound sums of two candidates (add.rm / add.rp, as the main loop).
__device__ __forceinline__ float2 sum2_rm(unsigned long long a, unsigned long long b) {
  unsigned long long t;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(t) : "l"(a), "l"(b));
  return make_float2(__uint_as_float((unsigned)t), __uint_as_float((unsigned)(t >> 32)));
}
__device__ __forceinline__ float2 sum2_rp(unsigned long long a, unsigned long long b) {
  unsigned long long t;
  asm("add.rp.f32x2 %0, %1, %2;" : "=l"(t) : "l"(a), "l"(b));
  return make_float2(__uint_as_float((unsigned)t), __uint_as_float((unsigned)(t >> 32)));
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

__device__ __forceinline__ void relax2_rm(float &acc, unsigned long long a, unsigned long long b) {
  asm("{\n\t.reg .b64 t;\n\t.reg .f32 x, y;\n\t"
      "add.rm.f32x2 t, %1, %2;\n\t"
      "mov.b64 {x, y}, t;\n\t"
      "min.f32 %0, %0, x, y;\n\t}"
      : "+f"(acc)
      : "l"(a), "l"(b));
}

// ---------------------------------------------------------------- K1
// Phase 1 on block (r,r): Algorithm 1 (strict "<", k ascending), k
// sequential as the paper's phase 1.  The block's values live in shared
// memory as doubles (d) with their lower float bounds (dlo = rd d); each
// thread keeps the upper bounds (dhi = ru d) of its 4 x 8 elements in
// registers.  At step k a candidate d[i][k] + d[k][j] is skipped without an
// FP64 add when its lower bound rd(dlo[i][k] + dlo[k][j]) is not below dhi[i][j]
// (then fl(d[i][k] + d[k][j]) >= d[i][j]); otherwise one FP64 add decides.
// Step k never changes row or column k (D[k][k] = 0), so every thread reads
// them straight from shared memory while the step writes other elements; one
// barrier per step.  Element (i, j) of thread (ty, tx) = (tid / 16, tid % 16):
// i = ty + 32 rr (rr 0..3), j = 2 tx + q + 32 cb (cb 0..3, q 0..1).
// Also marks every operand pack of the round's set exact (the phase-2/3
// kernel clears the flag of a pack holding a value that is not a float).
constexpr int K1_THREADS = 512;
struct K1Smem {
  double d[T * T];
  float dlo[T * T];
  unsigned char pk[T * T];  // block-local k of the last improvement, 0xFF none
};

__global__ void __launch_bounds__(K1_THREADS, 1)
    fw64_diag(double *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r, int R, Pack *packA,
              Pack *packB) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  K1Smem &sm = *reinterpret_cast<K1Smem *>(smem_raw);
  const int base = r * T, m = min(T, n - base), tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const double INF = inf<double>();
  for (int e = tid; e < T * T; e += K1_THREADS) {
    const int i = e / T, j = e % T;
    const double v = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : INF;
    sm.d[e] = v;
    sm.dlo[e] = f64_down(v);
    sm.pk[e] = 0xFF;
  }
  if (packA)
    for (int b = tid; b < R; b += K1_THREADS) {
      packA[b].exact = 1;
      packB[b].exact = 1;
    }
  __syncthreads();
  // element t = 8 rr + c of this thread: i = ty + 32 rr, j = 2 tx + (c & 1) + 32 (c >> 1)
  float dhi[32];
#pragma unroll
  for (int t = 0; t < 32; ++t)
    dhi[t] = f64_up(sm.d[(ty + 32 * (t >> 3)) * T + 2 * tx + (t & 1) + 32 * ((t & 7) >> 1)]);
#pragma unroll 1
  for (int k = 0; k < m; ++k) {
    float alo[4];
    unsigned long long blo[4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) alo[rr] = sm.dlo[(ty + 32 * rr) * T + k];
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) blo[cb] = *reinterpret_cast<const unsigned long long *>(&sm.dlo[k * T + 2 * tx + 32 * cb]);
    unsigned cand_mask = 0u;  // bit t: the candidate's lower bound is below element t's upper bound
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const unsigned long long aa = packf2(alo[rr], alo[rr]);
#pragma unroll
      for (int cb = 0; cb < 4; ++cb) {
        const float2 lo = sum2_rm(aa, blo[cb]);
        cand_mask |= (lo.x < dhi[8 * rr + 2 * cb] ? 1u : 0u) << (8 * rr + 2 * cb);
        cand_mask |= (lo.y < dhi[8 * rr + 2 * cb + 1] ? 1u : 0u) << (8 * rr + 2 * cb + 1);
      }
    }
    // The exact test, once per flagged element (rolled: the code stays small).
#pragma unroll 1
    while (cand_mask) {
      const int t = __ffs(cand_mask) - 1;
      cand_mask &= cand_mask - 1;
      const int i = ty + 32 * (t >> 3), j = 2 * tx + (t & 1) + 32 * ((t & 7) >> 1);
      const double cand = __dadd_rn(sm.d[i * T + k], sm.d[k * T + j]);
      if (cand < sm.d[i * T + j]) {
        sm.d[i * T + j] = cand;
        sm.dlo[i * T + j] = f64_down(cand);
        sm.pk[i * T + j] = (unsigned char)k;
        const float up = f64_up(cand);
#pragma unroll
        for (int u = 0; u < 32; ++u) dhi[u] = u == t ? up : dhi[u];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < T * T; e += K1_THREADS) {
    const int i = e / T, j = e % T;
    const unsigned kl = sm.pk[e];
    if (kl != 0xFFu && i < m && j < m) {
      const int64_t g = (int64_t)(base + i) * ld + base + j;
      D[g] = sm.d[e];
      if (P) P[g] = base + (int)kl;
    }
  }
}

// ---------------------------------------------------------------- K2
// Phases 2 and 3, k sequential in the paper's order (as the FP32 path):
// within a row block (r,J) every column j evolves on its own,
//   own[i][j] <- min(own[i][j], diag[i][k] + own[k][j])   (k ascending),
// within a column block (I,r) every row i does,
//   own[i][j] <- min(own[i][j], own[i][k] + diag[k][j]),
// with the diagonal block final after K1.  A warp keeps four such lines in
// registers as doubles with their float bounds (lane l: positions 2l, 2l+1,
// 2l+64, 2l+65).  At step k the lower bound of the pivot own[k] is broadcast
// by a shuffle and paired with the diagonal's lower bounds from shared memory
// (one add.rm.f32x2 per two candidates); only when some lane's candidate
// lower bound is below its upper bound does the warp fetch the pivot's double
// and run the exact FP64 adds.  Then the finished lines are written (D and P
// where improved) and packed as phase-4 operands: a row block as the B
// operand packB[J] (B[k][j] = own[k][j]), a column block as the A operand
// packA[I] (A[i][k] = own[i][k]); in (line, position) terms both are
// lo[line / 64][pos / 2][line % 64] = (rd at pos, rd at pos + 1), hi likewise
// with ru, and rlo/rhi/r64[line][pos].  Entries outside the matrix are +inf.
namespace k2 {
constexpr int K2_THREADS = 256, LINES = 2, PARTS = T / (K2_THREADS / 32 * LINES), MS = T + 2;
constexpr int SMEM = T * MS * 4;
}  // namespace k2

__global__ void __launch_bounds__(k2::K2_THREADS, 2)
    fw64_lines(double *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r, int R, Pack *packA,
               Pack *packB) {
  using namespace k2;
  extern __shared__ __align__(16) float Mlo[];  // [T][MS]: Mlo[k][pos] = rd of the diagonal entry
  const int b = blockIdx.x / PARTS, part = blockIdx.x % PARTS;
  const bool is_row = b < R - 1;
  int other = is_row ? b : b - (R - 1);
  other += (other >= r);
  const int base_r = r * T, m_r = min(T, n - base_r);
  const int base_o = other * T, m_o = min(T, n - base_o);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const double INF = inf<double>();
  const double *diag = D + (int64_t)base_r * ld + base_r;
  for (int e = tid; e < T * T; e += K2_THREADS) {
    const int i = e / T, k = e % T;
    const double x = (i < m_r && k < m_r) ? diag[(int64_t)i * ld + k] : INF;
    Mlo[is_row ? k * MS + i : i * MS + k] = f64_down(x);  // Mlo[k][pos]
  }
  const int line0 = part * (T / PARTS) + w * LINES;
  // Element (line, pos) of the own block sits at D[g0 + line * sl + pos * sp].
  const int64_t g0 = is_row ? (int64_t)base_r * ld + base_o : (int64_t)base_o * ld + base_r;
  const int64_t sl = is_row ? 1 : ld, sp = is_row ? ld : 1;
  // the diagonal entry paired with position pos at step k: row block diag[pos][k], column block diag[k][pos]
  const int64_t dpos = is_row ? ld : 1, dk = is_row ? 1 : ld;
  double v[LINES][4];
  float vlo[LINES][4], vhi[LINES][4];
  unsigned pk[LINES];  // byte q: round-local k of the last improvement of slot q, 0xFF: none
#pragma unroll
  for (int c = 0; c < LINES; ++c) {
    pk[c] = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int line = line0 + c, pos = 2 * lane + (q & 1) + 64 * (q >> 1);
      v[c][q] = (line < m_o && pos < m_r) ? D[g0 + line * sl + pos * sp] : INF;
      vlo[c][q] = f64_down(v[c][q]);
      vhi[c][q] = f64_up(v[c][q]);
    }
  }
  __syncthreads();
  // Step k: owner lane (k mod 64) / 2, slot 2 (k / 64) + (k mod 2).  The
  // filter runs unrolled over the warp's lines; the exact FP64 tests run in a
  // rolled loop over the flagged elements, so the loop body stays small.
#pragma unroll 1
  for (int k = 0; k < T; ++k) {
    const int owner = (k & 63) >> 1, slot = 2 * (k >> 6) + (k & 1);
    const unsigned long long m01 = *reinterpret_cast<const unsigned long long *>(&Mlo[k * MS + 2 * lane]);
    const unsigned long long m23 = *reinterpret_cast<const unsigned long long *>(&Mlo[k * MS + 64 + 2 * lane]);
    unsigned pass = 0u;  // bit 4 c + q
#pragma unroll
    for (int c = 0; c < LINES; ++c) {
      const float own_lo = slot == 0 ? vlo[c][0] : slot == 1 ? vlo[c][1] : slot == 2 ? vlo[c][2] : vlo[c][3];
      const float vk_lo = __shfl_sync(kFullMask, own_lo, owner);
      const unsigned long long vv = packf2(vk_lo, vk_lo);
      const float2 l01 = sum2_rm(m01, vv), l23 = sum2_rm(m23, vv);
      pass |= ((l01.x < vhi[c][0] ? 1u : 0u) | (l01.y < vhi[c][1] ? 2u : 0u) | (l23.x < vhi[c][2] ? 4u : 0u) |
               (l23.y < vhi[c][3] ? 8u : 0u)) << (4 * c);
    }
    const unsigned any = __ballot_sync(kFullMask, pass != 0u);
    if (!any) continue;  // warp-uniform
    double vk[LINES];
#pragma unroll
    for (int c = 0; c < LINES; ++c) {
      const double own = slot == 0 ? v[c][0] : slot == 1 ? v[c][1] : slot == 2 ? v[c][2] : v[c][3];
      vk[c] = __shfl_sync(kFullMask, own, owner);
    }
#pragma unroll 1
    while (pass) {
      const int b = __ffs(pass) - 1, c = b >> 2, q = b & 3;
      pass &= pass - 1;
      const int pos = 2 * lane + (q & 1) + 64 * (q >> 1);
      double vkc = vk[0];
#pragma unroll
      for (int u = 1; u < LINES; ++u) vkc = u == c ? vk[u] : vkc;
      const double cand = __dadd_rn(__ldg(diag + pos * dpos + k * dk), vkc);
      double cur = 0.0;
#pragma unroll
      for (int u = 0; u < 4 * LINES; ++u) cur = u == b ? v[u >> 2][u & 3] : cur;
      if (cand < cur) {
        const float lo = f64_down(cand), up = f64_up(cand);
#pragma unroll
        for (int u = 0; u < 4 * LINES; ++u)
          if (u == b) {
            v[u >> 2][u & 3] = cand;
            vlo[u >> 2][u & 3] = lo;
            vhi[u >> 2][u & 3] = up;
            pk[u >> 2] = __byte_perm(pk[u >> 2], (unsigned)k,
                                     0x3210 ^ ((0x3210 & (0xF << (4 * (u & 3)))) ^ (4 << (4 * (u & 3)))));
          }
      }
    }
  }
  // D and P where the line improved; the phase-4 operand pack everywhere.
  Pack *dst = is_row ? &packB[other] : &packA[other];
  bool ex = true;
#pragma unroll
  for (int c = 0; c < LINES; ++c) {
    const int line = line0 + c;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned kq = (pk[c] >> (8 * q)) & 0xFFu;
      if (kq != 0xFFu) {  // improved: inside the matrix
        const int pos = 2 * lane + (q & 1) + 64 * (q >> 1);
        const int64_t g = g0 + line * sl + pos * sp;
        D[g] = v[c][q];
        if (P) P[g] = base_r + (int)kq;
      }
      ex = ex && vlo[c][q] == vhi[c][q];
    }
#pragma unroll
    for (int hq = 0; hq < 2; ++hq) {  // positions 2 lane + 64 hq + {0, 1}: k-pair lane + 32 hq
      const int kp = lane + 32 * hq, pos = 2 * kp;
      dst->lo[line >> 6][kp][line & 63] = packf2(vlo[c][2 * hq], vlo[c][2 * hq + 1]);
      dst->hi[line >> 6][kp][line & 63] = packf2(vhi[c][2 * hq], vhi[c][2 * hq + 1]);
      *reinterpret_cast<float2 *>(&dst->rlo[line][pos]) = make_float2(vlo[c][2 * hq], vlo[c][2 * hq + 1]);
      *reinterpret_cast<float2 *>(&dst->rhi[line][pos]) = make_float2(vhi[c][2 * hq], vhi[c][2 * hq + 1]);
      *reinterpret_cast<double2 *>(&dst->r64[line][pos]) = make_double2(v[c][2 * hq], v[c][2 * hq + 1]);
    }
  }
  if (__syncthreads_or(!ex) && tid == 0) dst->exact = 0;
}

// ---------------------------------------------------------------- products
// Phase 4: a CTA computes one 128 x 64 half of an output block C = (I,J)
// (two CTAs per block, three CTAs per SM) from A = packA[I] and B = packB[J],
// both final for the round.
//
// Only the lower bounds enter the main loop.  X = min_k lo_k is a lower bound
// of the exact FP64 minimum s* (lo_k <= s_k for every k), so X >= ru(old)
// means no improvement.  Otherwise s* = X exactly when some k with lo_k = X
// has an exact sum of X (its upper bound is X too, or one FP64 add says so),
// and the first such k is the path entry; if none has, s* > X and the exact
// minimum is taken over the candidates with lo_k <= min(ru(old),
// min{up_k : lo_k = X}) (an upper bound of s*).  With integer weights every
// sum is exact and the first case always holds.
struct ProdSmem {
  unsigned long long Alo[STAGES][2][KP][H];  // both row halves of the A slab
  unsigned long long Blo[STAGES][KP][H];     // this CTA's column half of the B slab
  uint64_t bar[STAGES];
};

// Thread (warp w, lane l): ty = 4w + l/8 (0..31), tx = l%8 (0..7);
//   rows i(r) = (r>>1)*64 + ty*2 + (r&1)        (r = 0..3, row half r>>1)
//   cols j(c) = (c>>1)*16 + tx*2 + (c&1)        (c = 0..7, within the CTA's half)
// Row and column pairs are adjacent, so each pair is one 16-byte shared load;
// a warp's loads of one k-pair touch 64 (A) and 128 (B) consecutive bytes.
__device__ __forceinline__ int row4(int r, int ty) { return (r >> 1) * 64 + ty * 2 + (r & 1); }
__device__ __forceinline__ int col8(int c, int tx) { return (c >> 1) * 16 + tx * 2 + (c & 1); }

__device__ __forceinline__ void issue_slab(ProdSmem &sm, int st, const Pack *A, const Pack *B, int hJ,
                                           int s) {
  mbar_expect_tx(&sm.bar[st], 3 * SLAB_BYTES);
  for (int h = 0; h < 2; ++h) bulk_g2s(&sm.Alo[st][h][0][0], &A->lo[h][s * KP][0], SLAB_BYTES, &sm.bar[st]);
  bulk_g2s(&sm.Blo[st][0][0], &B->lo[hJ][s * KP][0], SLAB_BYTES, &sm.bar[st]);
}

// Block sets of one phase-4 launch (grid: 2 CTAs per block).
constexpr int kSetAll = 0;   // all (R-1)^2 blocks off row/column r
constexpr int kSetNext = 1;  // the 2R-3 blocks in row r+1 or column r+1
constexpr int kSetRest = 2;  // the (R-2)^2 blocks off rows/columns r and r+1

__device__ __forceinline__ double f32_as_f64(float x) { return __longlong_as_double((long long)f32_to_f64_bits(x)); }

#ifndef APSP_F64_EAGER_ROUNDS
#define APSP_F64_EAGER_ROUNDS 16
#endif
// Phase-4 rounds whose main loop also keeps, per output, the k-pair where
// min lo last decreased strictly (EAGER): in the first rounds nearly every
// output may improve, and one compare and one byte permute per k-pair cost
// less than scanning every candidate again to find the k that reaches X.
constexpr int kEagerRounds64 = APSP_F64_EAGER_ROUNDS;

template <bool EAGER>
__global__ void __launch_bounds__(THREADS, EAGER ? 2 : 3)
    fw64_product(double *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r, int R,
                 const Pack *packA, const Pack *packB, int set) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  ProdSmem &sm = *reinterpret_cast<ProdSmem *>(smem_raw);
  const int tile = blockIdx.x >> 1, hJ = blockIdx.x & 1;
  int I, J;
  if (set == kSetAll) {
    I = tile / (R - 1);
    J = tile % (R - 1);
    I += (I >= r);
    J += (J >= r);
  } else if (set == kSetNext) {  // row r+1, then column r+1: the next round's K1/K2 input
    if (tile < R - 1) {
      I = r + 1;
      J = tile + (tile >= r);
    } else {
      I = tile - (R - 1);
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
  const Pack *A = &packA[I];
  const Pack *B = &packB[J];
  const int baseI = I * T, baseJ = J * T + hJ * H, baseK = r * T;
  const int mI = min(T, n - baseI), mJ = min(H, n - baseJ), mK = min(T, n - baseK);
  if (mJ <= 0) return;  // an empty half of the last (narrow) block (uniform exit, no barrier used)
  const int nslab = (mK + KS - 1) / KS;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int ty = 4 * w + (lane >> 3), tx = lane & 7;
  const float FINF = __int_as_float(0x7f800000);
  // Both operands hold floats only: a candidate's upper bound is ru of the
  // same operands as its lower bound.
  const bool exact = A->exact && B->exact;

  if (tid == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(&sm.bar[st], 1);
    fence_mbar_init();
    for (int s = 0; s < STAGES && s < nslab; ++s) issue_slab(sm, s, A, B, hJ, s);
  }
  __syncthreads();

  float lo[4][8];
  unsigned kid[4][2];  // EAGER: byte c%4 of kid[a][c/4] = k-pair of the last strict decrease, 0xFF none
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    kid[a][0] = kid[a][1] = 0xFFFFFFFFu;
#pragma unroll
    for (int c = 0; c < 8; ++c) lo[a][c] = FINF;
  }

  for (int s = 0; s < nslab; ++s) {
    const int st = s % STAGES;
    const bool ok = mbar_wait(&sm.bar[st], (s / STAGES) & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        report_wait_timeout();
        for (int s2 = s + 1; s2 < nslab && s2 < s + STAGES; ++s2)
          mbar_wait(&sm.bar[s2 % STAGES], (s2 / STAGES) & 1);
      }
      return;
    }
    const unsigned long long(*As)[KP][H] = sm.Alo[st];
    const unsigned long long(*Bs)[H] = sm.Blo[st];
// Unrolled by four: the shared loads of later k-pairs are scheduled ahead of
    // the current one's arithmetic (measured best of 1, 2, 4, 8 and 16).
#pragma unroll 4
    for (int kp = 0; kp < KP; ++kp) {
      unsigned long long a[4], b[8];
#pragma unroll
      for (int rr = 0; rr < 4; rr += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&As[rr >> 1][kp][ty * 2]);
        a[rr] = t.x;
        a[rr + 1] = t.y;
      }
#pragma unroll
      for (int cc = 0; cc < 8; cc += 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&Bs[kp][col8(cc, tx)]);
        b[cc] = t.x;
        b[cc + 1] = t.y;
      }
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          if constexpr (EAGER) {
            const float2 t2 = sum2_rm(a[rr], b[cc]);
            const float m = min3f(lo[rr][cc], t2.x, t2.y);
            if (m < lo[rr][cc])
              kid[rr][cc >> 2] = __byte_perm(kid[rr][cc >> 2], (unsigned)(s * KP + kp),
                                             0x3210 ^ ((0x3210 & (0xF << (4 * (cc & 3)))) ^ (4 << (4 * (cc & 3)))));
            lo[rr][cc] = m;
          } else {
            relax2_rm(lo[rr][cc], a[rr], b[cc]);
          }
        }
    }
    __syncthreads();
    if (tid == 0 && s + STAGES < nslab) {
      fence_proxy_async_smem();
      issue_slab(sm, st, A, B, hJ, s + STAGES);
    }
  }

  // Epilogue.  The ring is free: X = min lo goes to shared memory, then each
  // warp owns 16 whole rows (lane l: columns 2l, 2l+1 of the half).
  float *Lo = reinterpret_cast<float *>(smem_raw);            // [T][H]
  unsigned char *Ks = smem_raw + sizeof(ProdSmem::Alo);        // EAGER: [T][H] k-pair bytes
  __syncthreads();
#pragma unroll
  for (int rr = 0; rr < 4; ++rr)
#pragma unroll
    for (int cc = 0; cc < 8; cc += 2) {
      *reinterpret_cast<float2 *>(&Lo[row4(rr, ty) * H + col8(cc, tx)]) = make_float2(lo[rr][cc], lo[rr][cc + 1]);
      if constexpr (EAGER)
        *reinterpret_cast<unsigned short *>(&Ks[row4(rr, ty) * H + col8(cc, tx)]) =
            (unsigned short)(kid[rr][cc >> 2] >> (8 * (cc & 3)));
    }
  __syncthreads();
  const int j0 = 2 * lane, i0 = w * 16, jb0 = hJ * H;
  // Pass 1: outputs that may improve (X < ru(old)).  Bit 2t + q of `pot`:
  // row i0 + t, column j0 + q.  Old values load eight rows at a time.
  unsigned pot = 0u;
#pragma unroll
  for (int t8 = 0; t8 < 16; t8 += 8) {
    double o[8][2];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
      for (int q = 0; q < 2; ++q)
        o[t][q] = (i0 + t8 + t < mI && j0 + q < mJ) ? D[(int64_t)(baseI + i0 + t8 + t) * ld + baseJ + j0 + q]
                                                     : inf<double>();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float2 x = *reinterpret_cast<const float2 *>(&Lo[(i0 + t8 + t) * H + j0]);
      if (i0 + t8 + t < mI) {
        if (j0 < mJ && f32_lt_f64(x.x, o[t][0])) pot |= 1u << (2 * (t8 + t));
        if (j0 + 1 < mJ && f32_lt_f64(x.y, o[t][1])) pot |= 2u << (2 * (t8 + t));
      }
    }
  }
  if constexpr (EAGER) {
    // The k-pair where min lo last decreased holds the first k with lo_k = X
    // (the lower one if its lower bound is X).  If that candidate's exact sum
    // is X, s* = X and k is the path entry; otherwise pass 2b decides.
#pragma unroll 1
    for (int t = 0; t < 16; ++t)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned bitq = 1u << (2 * t + q);
        if (!(pot & bitq)) continue;
        const int i = i0 + t, jl = j0 + q, jb = jb0 + jl;
        const int kp = Ks[i * H + jl];  // a candidate output has one (X is finite)
        const float X = Lo[i * H + jl];
        const unsigned long long al = A->lo[i >> 6][kp][i & 63], bl = B->lo[hJ][kp][jl];
        const float2 l = sum2_rm(al, bl);
        const int k = l.x == X ? 2 * kp : 2 * kp + 1;
        const float up_ = exact ? (l.x == X ? sum2_rp(al, bl).x : sum2_rp(al, bl).y)
                                : __fadd_ru(A->rhi[i][k], B->rhi[jb][k]);
        if (up_ == X || __dadd_rn(A->r64[i][k], B->r64[jb][k]) == f32_as_f64(X)) {
          const int64_t gi = (int64_t)(baseI + i) * ld + baseJ + jl;
          D[gi] = f32_as_f64(X);  // X < old (pass 1)
          if (P) P[gi] = baseK + k;
          pot &= ~bitq;
        }
      }
  }
  // Pass 2a: each 8-row group of the warp with many candidates (the early
  // rounds) is scanned lane-parallel: lane l walks the lower-bound pairs of
  // its two columns over all k (B pairs coalesced, A pairs broadcast,
  // add.rm.f32x2 as in the main loop), folds every 8 k into one minimum, and
  // keeps the lowest 8-k chunk whose minimum is X.  Inside that chunk the
  // first k with lo_k = X and an exact sum X settles the output (D where X <
  // old, and P); an output without one there is left to pass 2b.
  {
    const unsigned long long *pbl = &B->lo[hJ][0][j0];
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {
      const unsigned gm = 0xFFFFu << (16 * G);
      if (EAGER || (int)__reduce_add_sync(kFullMask, (unsigned)__popc(pot & gm)) < kDenseMin64) continue;
      const int tg0 = 8 * G;
      float g[8][2];
      unsigned hit[8];  // bit c (+16 for column j0 + 1): chunk c's minimum lo equals X
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const float2 x = *reinterpret_cast<const float2 *>(&Lo[(i0 + tg0 + t) * H + j0]);
        g[t][0] = x.x;
        g[t][1] = x.y;
        hit[t] = 0u;
      }
#pragma unroll 1
      for (int c = T / 8 - 1; c >= 0; --c) {
        ulonglong2 b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) b[q] = __ldg(reinterpret_cast<const ulonglong2 *>(pbl + (4 * c + q) * H));
        const unsigned bit = 1u << c;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int i = i0 + tg0 + t;
          const unsigned long long *pal = &A->lo[i >> 6][0][i & 63];
          unsigned long long a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = __ldg(pal + (4 * c + q) * H);
#pragma unroll
          for (int q2 = 0; q2 < 2; ++q2) {
            const float2 s0 = sum2_rm(a[0], q2 ? b[0].y : b[0].x), s1 = sum2_rm(a[1], q2 ? b[1].y : b[1].x);
            const float2 s2 = sum2_rm(a[2], q2 ? b[2].y : b[2].x), s3 = sum2_rm(a[3], q2 ? b[3].y : b[3].x);
            float m = min3f(s0.x, s0.y, s1.x);
            m = min3f(m, s1.y, s2.x);
            m = min3f(m, s2.y, s3.x);
            m = fminf(m, s3.y);
            if (m == g[t][q2]) hit[t] |= bit << (16 * q2);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = i0 + tg0 + t;
        const unsigned long long *pal = &A->lo[i >> 6][0][i & 63];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
          const unsigned bitq = 1u << (2 * (tg0 + t) + q2);
          if (!(pot & bitq)) continue;
          const unsigned cm = (hit[t] >> (16 * q2)) & 0xFFFFu;  // not empty: X is some lo
          const int c = __ffs(cm) - 1;
          const float X = g[t][q2];
          const int jb = jb0 + j0 + q2;
          // the chunk's eight lower-bound sums; upper bounds (and FP64 sums)
          // only for a k whose lower bound is X, in ascending k
          unsigned eq = 0u, equp = 0u;  // lo_k = X; and up_k = X (exact operands only)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const unsigned long long av = __ldg(pal + (4 * c + q) * H), bv = __ldg(pbl + (4 * c + q) * H + q2);
            const float2 l = sum2_rm(av, bv);
            eq |= (l.x == X ? 1u : 0u) << (2 * q);
            eq |= (l.y == X ? 1u : 0u) << (2 * q + 1);
            if (exact) {
              const float2 u = sum2_rp(av, bv);
              equp |= (u.x == X ? 1u : 0u) << (2 * q);
              equp |= (u.y == X ? 1u : 0u) << (2 * q + 1);
            }
          }
          int kf = -1;
#pragma unroll 1
          while (eq) {
            const int b = __ffs(eq) - 1, k = 8 * c + b;
            eq &= eq - 1;
            if ((exact ? ((equp >> b) & 1u) != 0u : __fadd_ru(A->rhi[i][k], B->rhi[jb][k]) == X) ||
                __dadd_rn(A->r64[i][k], B->r64[jb][k]) == f32_as_f64(X)) {
              kf = k;
              break;
            }
          }
          if (kf >= 0) {  // s* = X exactly
            const int64_t gi = (int64_t)(baseI + i) * ld + baseJ + j0 + q2;
            const double xd = f32_as_f64(X);
            if (xd < D[gi]) {
              D[gi] = xd;
              if (P) P[gi] = baseK + kf;
            }
            pot &= ~bitq;
          }
        }
      }
    }
  }
  // Pass 2b: every remaining candidate output, walked as one stream two at a
  // time; lane l tests k = 4l..4l+3.  The lower-bound rows load first; a k
  // with lo_k = X fetches its upper bounds (and, if they differ, its FP64
  // operands).  The first exact X settles the output; without one, the exact
  // FP64 minimum over the candidates with lo_k <= min(ru(old), min up over
  // lo_k = X) does (first k on ties).
  unsigned wf = __reduce_or_sync(kFullMask, pot), bal = 0u;
  int pos = 0;
  auto next = [&](int &t, int &sj) -> bool {  // warp-uniform
    while (!bal) {
      if (!wf) return false;
      pos = __ffs(wf) - 1;
      wf &= wf - 1;
      bal = __ballot_sync(kFullMask, (pot >> pos) & 1u);
    }
    const int src = __ffs(bal) - 1;
    bal &= bal - 1;
    t = pos >> 1;
    sj = 2 * src + (pos & 1);
    return true;
  };
#pragma unroll 1
  for (;;) {
    int t[2], sj[2];
    bool v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) v[u] = next(t[u], sj[u]);
    if (!v[0]) break;
    float4 al[2], bl[2];
    double old[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!v[u]) continue;
      const int i = i0 + t[u];
      al[u] = reinterpret_cast<const float4 *>(&A->rlo[i][0])[lane];
      bl[u] = reinterpret_cast<const float4 *>(&B->rlo[jb0 + sj[u]][0])[lane];
      old[u] = D[(int64_t)(baseI + i) * ld + baseJ + sj[u]];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!v[u]) continue;
      const int i = i0 + t[u], jb = jb0 + sj[u];
      const int64_t gi = (int64_t)(baseI + i) * ld + baseJ + sj[u];
      const float X = Lo[i * H + sj[u]];
      const float la[4] = {al[u].x, al[u].y, al[u].z, al[u].w};
      const float lb[4] = {bl[u].x, bl[u].y, bl[u].z, bl[u].w};
      float l4[4];
      unsigned h = 0u;
      float upx = FINF;  // min up over this lane's k with lo_k = X
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * lane + q;
        l4[q] = __fadd_rd(la[q], lb[q]);
        if (l4[q] == X) {
          const float up_ = exact ? __fadd_ru(la[q], lb[q]) : __fadd_ru(A->rhi[i][k], B->rhi[jb][k]);
          upx = fminf(upx, up_);
          if (up_ == X || __dadd_rn(A->r64[i][k], B->r64[jb][k]) == f32_as_f64(X)) h |= 1u << q;
        }
      }
      const unsigned hb = __ballot_sync(kFullMask, h != 0u);
      if (hb) {  // s* = X exactly; the lowest hit is the first k
        const int L = __ffs(hb) - 1;
        const unsigned hL = __shfl_sync(kFullMask, h, L);
        const double xd = f32_as_f64(X);
        if (lane == 0 && xd < old[u]) {
          D[gi] = xd;
          if (P) P[gi] = baseK + 4 * L + (__ffs(hL) - 1);
        }
        continue;
      }
      // s* > X: exact FP64 minimum over the candidates that can reach it.
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) upx = fminf(upx, __shfl_xor_sync(kFullMask, upx, off));
      const float th = fminf(upx, f64_up(old[u]));
      long long best = 0x7fffffffffffffffll;
      int bestk = 0x7fffffff;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 4 * lane + q;
        if (l4[q] <= th) {
          const float up_ = exact ? __fadd_ru(la[q], lb[q]) : __fadd_ru(A->rhi[i][k], B->rhi[jb][k]);
          const unsigned long long vb =
              l4[q] == up_ ? f32_to_f64_bits(l4[q])
                           : (unsigned long long)__double_as_longlong(__dadd_rn(A->r64[i][k], B->r64[jb][k]));
          const long long key = dkey(vb);
          if (key < best) {
            best = key;
            bestk = k;
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {  // warp argmin over (key, k)
        const long long ob = __shfl_xor_sync(kFullMask, best, off);
        const int okk = __shfl_xor_sync(kFullMask, bestk, off);
        if (ob < best || (ob == best && okk < bestk)) {
          best = ob;
          bestk = okk;
        }
      }
      if (lane == 0 && bestk != 0x7fffffff &&
          best < dkey((unsigned long long)__double_as_longlong(old[u]))) {
        D[gi] = __longlong_as_double((long long)dkey_bits(best));
        if (P) P[gi] = baseK + bestk;
      }
    }
  }
}

static int g_smem_k1[64], g_smem_k2[64], g_smem_p0[64], g_smem_p0e[64];

}  // namespace f64

// Host round loop for FP64 (called by apsp_fw_f64).
int run_fw_f64_interval(double *D, int n, int64_t ld, int32_t *P, cudaStream_t s) {
  using namespace f64;
  const int R = (n + T - 1) / T;
  int st;
  const int smem1 = (int)sizeof(K1Smem), smemp = (int)sizeof(ProdSmem);
  if ((st = ensure_smem(fw64_diag, smem1, g_smem_k1))) return st;
  if ((st = ensure_smem(fw64_lines, k2::SMEM, g_smem_k2))) return st;
  if ((st = ensure_smem(fw64_product<false>, smemp, g_smem_p0))) return st;
  if ((st = ensure_smem(fw64_product<true>, smemp, g_smem_p0e))) return st;
  // Operand packs: two sets by round parity (so that phases 1-3 of round
  // r+1 can pack while phase 4 of round r still reads), each R column-panel
  // packs (A operands) and R row-panel packs (B operands).
  struct PackSet {
    Pack *A, *B;
  } ps[2]{};
  char *scratch = nullptr;
  if (R > 1) {
    if (cudaMallocAsync((void **)&scratch, sizeof(Pack) * 2 * (2 * (size_t)R), s) != cudaSuccess) {
      cudaGetLastError();
      return APSP_ENOMEM;
    }
    for (int q = 0; q < 2; ++q) {
      Pack *base = reinterpret_cast<Pack *>(scratch) + (size_t)q * (2 * R);
      ps[q] = {base, base + R};
    }
  }
  auto diag_and_panels = [&](int r, cudaStream_t stm) {
    const PackSet &p = ps[r & 1];
    {
      PhaseScope sc(1, stm);
      fw64_diag<<<1, K1_THREADS, smem1, stm>>>(D, ld, P, n, r, R, p.A, p.B);
    }
    if (R > 1) {
      PhaseScope sc(2, stm);
      fw64_lines<<<2 * (R - 1) * k2::PARTS, k2::K2_THREADS, k2::SMEM, stm>>>(D, ld, P, n, r, R, p.A, p.B);
    }
  };
  auto phase4 = [&](int r, int set, int blocks) {
    if (blocks <= 0) return;
    const PackSet &p = ps[r & 1];
    PhaseScope sc(3, s);
    if (r < kEagerRounds64)
      fw64_product<true><<<2 * blocks, THREADS, smemp, s>>>(D, ld, P, n, r, R, p.A, p.B, set);
    else
      fw64_product<false><<<2 * blocks, THREADS, smemp, s>>>(D, ld, P, n, r, R, p.A, p.B, set);
  };
  // Look-ahead as in the FP32 path: phase 4 of round r updates row and
  // column r+1 first; phases 1-3 of round r+1 then run on a second stream of
  // higher priority beside the rest of phase 4 (disjoint blocks, the other
  // pack set).
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
  for (int r = 0; R > 1 && r < R; ++r) {
    if (r + 1 < R && s2) {
      phase4(r, kSetNext, 2 * R - 3);
      cudaEventRecord(ev_next, s);
      cudaStreamWaitEvent(s2, ev_next, 0);
      diag_and_panels(r + 1, s2);
      cudaEventRecord(ev_panels, s2);
      phase4(r, kSetRest, (R - 2) * (R - 2));
      cudaStreamWaitEvent(s, ev_panels, 0);
    } else {
      phase4(r, kSetAll, (R - 1) * (R - 1));
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

int take_device_error_f64() { return take_tu_device_error(); }

}  // namespace apsp
