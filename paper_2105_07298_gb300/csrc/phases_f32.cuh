// Device code of the FP32 phases 2/3 (lines) and phase 4 (block product).
// The line code is shared by the single-graph kernel (fw_single.cu) and the
// batched persistent kernel (fw_batched.cu); the phase-4 block product here
// is the batched kernel's copy of the single-graph phase-4 kernel
// (fw_phase3_minplus_f32 in fw_single.cu), written as a device function so
// that one CTA can run many of them (the single-graph kernel keeps its own
// body: as a device function its code measured 5 % slower).  Internal header.
#pragma once
#include <stdint.h>

#include "bulk.cuh"
#include "common.cuh"
#include "minplus_f32.cuh"

namespace apsp {

// --------------------------------------------------------------------------
// K2: phases 2 and 3.  Blocks b < R-1 of the grid cover row block (r, J),
// the others column block (I, r); four CTAs share a block, 32 lines each.
// Within a row block every column evolves on its own, within a column block
// every row does:
//   row block, column j:  own[i][j] = min(own[i][j], diag[i][k] + own[k][j])
//   column block, row i:  own[i][j] = min(own[i][j], own[i][k] + diag[k][j])
// for k ascending over the round's vertices (the diagonal block is final
// after K1).  A warp keeps four such lines in registers, lane l holding
// positions 2l, 2l+1, 2l+64, 2l+65 of each; at step k the owner of position k
// broadcasts the line's current value with a shuffle, and the diagonal
// entries come from shared memory (M[k][pos], transposed for row blocks) as
// pairs, so one add.rn.f32x2 forms two candidates.  No barrier per step.
// The finished blocks are also written, padded with +inf to T x T, in the
// layouts phase 4 reads this round:
//   row block (r,J):    Bpan[J][j/64][kp][j%64] = (own[2kp][j], own[2kp+1][j]),
//                       Bt[J][j][k] = own[k][j]
//   column block (I,r): Apan[I][kp][i] = (own[i][2kp], own[i][2kp+1]),
//                       Acp[I][i][k] = own[i][k]
// --------------------------------------------------------------------------
struct Panels {
  unsigned long long *Apan, *Bpan;
  float *Acp, *Bt;
};

namespace k2 {
constexpr int T = mp32::T, THREADS = 256, LINES = 4, PARTS = T / (THREADS / 32 * LINES), MS = T + 2;
constexpr int SMEM = T * MS * 4;
}  // namespace k2

// Fills M[k][pos] (the launch's dynamic shared memory from offset 0) with the
// diagonal block of round r (transposed for row blocks, +inf outside the
// matrix).  The caller synchronises before use.
__device__ __forceinline__ void lines_load_diag(const float *__restrict__ D, int64_t ld, int n, int r, bool is_row) {
  using namespace k2;
  extern __shared__ __align__(16) float M[];  // [T][MS], the launch's dynamic shared memory
  const int base_r = r * T, m_r = min(T, n - base_r);
  const float INF = inf<float>();
  for (int e = threadIdx.x; e < T * T; e += THREADS) {
    const int i = e / T, k = e % T;
    const float x = (i < m_r && k < m_r) ? D[(int64_t)(base_r + i) * ld + base_r + k] : INF;
    M[is_row ? k * MS + i : i * MS + k] = x;  // M[k][pos]
  }
}

// Lines 32 part .. 32 part + 31 of the row block (r, other) (is_row) or the
// column block (other, r), with M holding the diagonal block in that block
// type's layout (lines_load_diag).
__device__ __forceinline__ void lines_part_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n,
                                               int r, int other, bool is_row, int part, const Panels &pan) {
  using namespace k2;
  extern __shared__ __align__(16) float M[];  // [T][MS], filled by lines_load_diag
  const int base_r = r * T, m_r = min(T, n - base_r);
  const int base_o = other * T, m_o = min(T, n - base_o);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float INF = inf<float>();
  const int line0 = part * (T / PARTS) + w * LINES;
  // Element (line, pos) of the own block sits at D[g0 + line * sl + pos * sp].
  const int64_t g0 = is_row ? (int64_t)base_r * ld + base_o : (int64_t)base_o * ld + base_r;
  const int64_t sl = is_row ? 1 : ld, sp = is_row ? ld : 1;
  // lane's positions along a line: pos(s) = 2 lane + (s & 1) + 64 (s >> 1)
  float v[LINES][4];
  unsigned pk[LINES];  // byte q: round-local k of the last improvement of slot q, 0xFF: none
#pragma unroll
  for (int c = 0; c < LINES; ++c) {
    pk[c] = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int line = line0 + c, pos = 2 * lane + (q & 1) + 64 * (q >> 1);
      v[c][q] = (line < m_o && pos < m_r) ? D[g0 + line * sl + pos * sp] : INF;
    }
  }
  // Step k: owner lane (k mod 64) / 2, slot 2 (k / 64) + (k mod 2).
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll 1
    for (int kk = 0; kk < 32; ++kk) {
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        const int k = 64 * h + 2 * kk + par;
        const unsigned long long m01 = *reinterpret_cast<const unsigned long long *>(&M[k * MS + 2 * lane]);
        const unsigned long long m23 = *reinterpret_cast<const unsigned long long *>(&M[k * MS + 64 + 2 * lane]);
#pragma unroll
        for (int c = 0; c < LINES; ++c) {
          const float vk = __shfl_sync(kFullMask, v[c][2 * h + par], kk);
          const unsigned long long vv = mp32::pack2(vk, vk);
          const float2 c01 = mp32::sum2(m01, vv), c23 = mp32::sum2(m23, vv);
          const float cand[4] = {c01.x, c01.y, c23.x, c23.y};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (cand[q] < v[c][q]) {
              v[c][q] = cand[q];
              pk[c] = __byte_perm(pk[c], (unsigned)k, 0x3210 ^ ((0x3210 & (0xF << (4 * q))) ^ (4 << (4 * q))));
            }
        }
      }
    }
  }
  // D and P where the line improved; the phase-4 panels everywhere (padded).
  const int64_t blk = other;
#pragma unroll
  for (int c = 0; c < LINES; ++c) {
    const int line = line0 + c;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pos = 2 * lane + (q & 1) + 64 * (q >> 1);
      const unsigned kq = (pk[c] >> (8 * q)) & 0xFFu;
      if (kq != 0xFFu) {  // improved: inside the matrix
        const int64_t g = g0 + line * sl + pos * sp;
        D[g] = v[c][q];
        if (P) P[g] = base_r + (int)kq;
      }
    }
#pragma unroll
    for (int hq = 0; hq < 2; ++hq) {  // positions 2 lane + 64 hq + {0, 1}: k-pair kp = lane + 32 hq
      const int kp = lane + 32 * hq;
      const unsigned long long pr = mp32::pack2(v[c][2 * hq], v[c][2 * hq + 1]);
      if (is_row) {
        pan.Bpan[((blk * 2 + (line >> 6)) * (T / 2) + kp) * (T / 2) + (line & 63)] = pr;
        *reinterpret_cast<float2 *>(&pan.Bt[(blk * T + line) * T + 2 * kp]) = make_float2(v[c][2 * hq], v[c][2 * hq + 1]);
      } else {
        pan.Apan[(blk * (T / 2) + kp) * T + line] = pr;
        *reinterpret_cast<float2 *>(&pan.Acp[(blk * T + line) * T + 2 * kp]) = make_float2(v[c][2 * hq], v[c][2 * hq + 1]);
      }
    }
  }
}

// K3 (FP32): one CTA computes one 128 x 64 half of an output block (two CTAs
// per block; three CTAs per SM, two for the eager instance); each thread owns
// an 8 x 4 register tile.  The operands come from the panel buffers K2 wrote
// (already in the paired shared-memory layout and padded with +inf, so the
// main loop needs no bounds checks): per 32-k slab one 16 KiB bulk copy of A
// and one 8 KiB copy of B into a two-stage ring, completion tracked by an
// mbarrier per stage.  Path recovery (lazy instance) reads the paired panels
// lane-parallel for dense row groups, and the row-contiguous copies Acp/Bt
// otherwise (one float4 of each per lane: the 128 candidate sums of an output
// in one memory round trip); the eager instance reads one operand pair per
// improved output.
namespace k3 {
constexpr int T = mp32::T, KS = mp32::KS, KP = mp32::KP, STAGES = 2, H = T / 2;
// Block sets of one phase-4 launch (grid: 2 CTAs per block).
constexpr int kSetAll = 0;   // all (R-1)^2 blocks off row/column r
constexpr int kSetNext = 1;  // the 2R-3 blocks in row r+1 or column r+1
constexpr int kSetRest = 2;  // the (R-2)^2 blocks off rows/columns r and r+1
constexpr uint32_t A_SLAB = KP * T * 8, B_SLAB = KP * H * 8;
#ifndef APSP_K3_DENSE_MIN
#define APSP_K3_DENSE_MIN 96
#endif
// Improved outputs (of 512) above which an 8-row group takes recovery pass 2a.
constexpr int kDenseMin = APSP_K3_DENSE_MIN;
struct Smem {
  unsigned long long As[STAGES][KP][T];  // As[kp][i] = (A[i][2kp], A[i][2kp+1])
  unsigned long long Bs[STAGES][KP][H];  // Bs[kp][j] = (B[2kp][j], B[2kp+1][j]), this half
  uint64_t bar[STAGES];
};
}  // namespace k3

#ifndef APSP_K3_MIN_BLOCKS
#define APSP_K3_MIN_BLOCKS 3
#endif
#ifndef APSP_K3_EAGER_ROUNDS
#define APSP_K3_EAGER_ROUNDS 16
#endif
// Rounds that track P in the main loop (EAGER): in the first rounds nearly
// every output improves, and one compare and one byte permute per k-pair
// (per two k-pairs in the single-graph kernel) cost less than recomputing
// every candidate afterwards.
constexpr int kEagerRounds = APSP_K3_EAGER_ROUNDS;

#ifndef APSP_K3_EAGER_MIN_BLOCKS
#define APSP_K3_EAGER_MIN_BLOCKS 2
#endif
template <bool NC, typename V>
__device__ __forceinline__ V ld_panel(const V *p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// One 128 x 64 half (hJ) of output block (I, J) of phase 4 in round r from
// the round's panels (both final).  NC: the panels were written by an earlier
// launch, so the recovery may read them through the non-coherent path; a
// caller that wrote them earlier in the same launch passes NC = false.
// Returns false if a bounded wait for a copy ran out (the block is then left
// unchanged and the error word is set).  Uses the launch's dynamic shared
// memory from offset 0 (sizeof(k3::Smem) bytes).
template <bool EAGER, bool NC>
__device__ __forceinline__ bool minplus_half_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n,
                                                 int I, int J, int hJ, int r, int vec_ok, const Panels &pan) {
  using namespace k3;
  using mp32::col_at;
  using mp32::row_at;
  // The launch's dynamic shared memory (declared here, not passed, so that
  // every access compiles as a shared-memory access).
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  const int baseI = I * T, baseJ = J * T + hJ * H, baseK = r * T;
  const int mI = min(T, n - baseI), mJ = min(H, n - baseJ), mK = min(T, n - baseK);
  if (mJ <= 0) return true;  // empty half of the last (narrow) block; uniform exit
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
      return false;
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
#pragma unroll 1
    for (int kp = 0; kp < KP; kp += 2) {
      load_b(kp + 1, b1);
      compute(kp, b0);
      if (kp + 2 < KP) load_b(kp + 2, b0);
      compute(kp + 1, b1);
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
  if (tid == 0)  // every phase of the ring completed; the barriers may be set up again
    for (int st = 0; st < STAGES; ++st) mbar_inval(&sm.bar[st]);
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
  if (!P) return true;
  if constexpr (EAGER) {
    // The k inside each improved output's last decreasing pair: the lower one
    // if its candidate equals the new value (the sequential loop keeps the
    // first k reaching a minimum).
#pragma unroll 1
    for (int t = 0; t < 16; ++t)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!((flags >> (2 * t + q)) & 1u)) continue;
        const int i = i0 + t, j = j0 + q;
        const int kp = Ks[i * H + j];  // an improved output has one
        const float2 c = mp32::sum2(srcA[(int64_t)kp * T + i], srcB[(int64_t)kp * H + j]);
        P[(int64_t)(baseI + i) * ld + baseJ + j] = baseK + (c.x == Cs[i * H + j] ? 2 * kp : 2 * kp + 1);
      }
    return true;
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
        for (int q = 0; q < 4; ++q) b[q] = ld_panel<NC>(reinterpret_cast<const ulonglong2 *>(pb + (4 * c + q) * H));
        const unsigned bit = 1u << c;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          unsigned long long a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = ld_panel<NC>(pa + (4 * c + q) * T + tg0 + t);
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
            av[q2][q] = ld_panel<NC>(pa + (4 * c[q2] + q) * T + tg0 + t);
            bv[q2][q] = ld_panel<NC>(pb + (4 * c[q2] + q) * H + q2);
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
  return true;
}

}  // namespace apsp
