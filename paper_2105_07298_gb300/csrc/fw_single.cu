// Single-graph blocked Floyd-Warshall for sm_103a.
//
// Schedule (§2.2 "Blocked FW Algorithm", kernels as in §3.2): the n x n
// matrix is cut into TB x TB blocks; each of the R = ceil(n / TB) rounds runs
//   K1  fw_phase1_diag      phase 1: the diagonal block (r,r), k sequential;
//   K2  fw_phase2_panels    phases 2+3: the row blocks (r,J) and the column
//                           blocks (I,r), k sequential inside each block;
//   K3  fw_phase3_minplus   phase 4: every other block (I,J) gets
//                           C = min(C, A (x) B) with A = block (I,r) and
//                           B = block (r,J), a min-plus product over the
//                           round's TB values of k.
// Relaxation rule: Algorithm 1 with a strict "<" (see apsp_fw.h).
//
// Differences from the Pascal design of §3.2 (one output per thread, TB <= 32):
//  * K3 computes an 8 x 8 register tile per thread (FP32, TB = 128) and pairs
//    consecutive k: one packed add.rn.f32x2 forms the two candidates of an
//    output and one three-input min.f32 folds both into the accumulator, so a
//    relaxation costs one issue slot (FADD2 and FMNMX3 run on different pipes).
//  * K3 keeps no path state in its inner loop.  After the loop, outputs that
//    improved (new < old) recover the first k that attains the new minimum:
//    the 32 lanes of a warp test 32 values of k at a time and take the lowest
//    hit.  This gives exactly the P of the sequential loop (ascending k,
//    strict "<" keeps the first k reaching the final minimum) at a cost paid
//    only by improved outputs.
//  * Nothing reads P: K1/K2/K3 write P only where D strictly improved.
#include <stdint.h>

#include "common.cuh"
#include "minplus_f32.cuh"

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

// --------------------------------------------------------------------------
// K1: phase 1 on the diagonal block (r,r).  One CTA; the block lives in shared
// memory; T sequential steps separated by barriers.  Step k reads row k and
// column k of the block, which step k itself never changes (D[k][k] = 0).
// --------------------------------------------------------------------------
template <typename Real, int T, int THREADS>
__global__ void __launch_bounds__(THREADS) fw_phase1_diag(Real *__restrict__ D, int64_t ld,
                                                          int32_t *__restrict__ P, int n, int r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *s = reinterpret_cast<Real *>(smem_raw);
  constexpr int EPT = T * T / THREADS;
  const int base = r * T;
  const int m = min(T, n - base);
  const int tid = threadIdx.x;
  for (int e = tid; e < T * T; e += THREADS) {
    const int i = e / T, j = e % T;
    s[e] = (i < m && j < m) ? D[(int64_t)(base + i) * ld + base + j] : inf<Real>();
  }
  int pk[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) pk[q] = -1;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * THREADS;
      const int i = e / T, j = e % T;
      const Real cand = add_rn(s[i * T + k], s[k * T + j]);
      if (cand < s[e]) {
        s[e] = cand;
        pk[q] = base + k;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * THREADS;
    const int i = e / T, j = e % T;
    if (i < m && j < m && pk[q] >= 0) {
      const int64_t g = (int64_t)(base + i) * ld + base + j;
      D[g] = s[e];
      if (P) P[g] = pk[q];
    }
  }
}

// --------------------------------------------------------------------------
// K2: phases 2 and 3.  CTA b < R-1 owns row block (r, J), the others column
// block (I, r).  The diagonal block (final after K1) and the own block sit in
// shared memory; k runs sequentially over the round's vertices.
//   row block:    own[i][j] = min(own[i][j], diag[i][k] + own[k][j])
//   column block: own[i][j] = min(own[i][j], own[i][k] + diag[k][j])
// --------------------------------------------------------------------------
template <typename Real, int T, int THREADS>
__global__ void __launch_bounds__(THREADS) fw_phase2_panels(Real *__restrict__ D, int64_t ld,
                                                            int32_t *__restrict__ P, int n, int r,
                                                            int R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real *diag = reinterpret_cast<Real *>(smem_raw);
  Real *own = diag + T * T;
  constexpr int EPT = T * T / THREADS;
  const int b = blockIdx.x;
  const bool is_row = b < R - 1;
  int other = is_row ? b : b - (R - 1);
  other += (other >= r);
  const int base_r = r * T, m_r = min(T, n - base_r);
  const int base_o = other * T, m_o = min(T, n - base_o);
  // own block: rows x cols = (m_r x m_o) for a row block, (m_o x m_r) for a column block
  const int rows = is_row ? m_r : m_o, cols = is_row ? m_o : m_r;
  const int64_t row0 = is_row ? base_r : base_o, col0 = is_row ? base_o : base_r;
  const int tid = threadIdx.x;
  for (int e = tid; e < T * T; e += THREADS) {
    const int i = e / T, j = e % T;
    diag[e] = (i < m_r && j < m_r) ? D[(int64_t)(base_r + i) * ld + base_r + j] : inf<Real>();
    own[e] = (i < rows && j < cols) ? D[(row0 + i) * ld + col0 + j] : inf<Real>();
  }
  int pk[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) pk[q] = -1;
  __syncthreads();
  if (is_row) {
    for (int k = 0; k < m_r; ++k) {
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * THREADS;
        const int i = e / T, j = e % T;
        const Real cand = add_rn(diag[i * T + k], own[k * T + j]);
        if (cand < own[e]) {
          own[e] = cand;
          pk[q] = base_r + k;
        }
      }
      __syncthreads();
    }
  } else {
    for (int k = 0; k < m_r; ++k) {
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = tid + q * THREADS;
        const int i = e / T, j = e % T;
        const Real cand = add_rn(own[i * T + k], diag[k * T + j]);
        if (cand < own[e]) {
          own[e] = cand;
          pk[q] = base_r + k;
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * THREADS;
    const int i = e / T, j = e % T;
    if (i < rows && j < cols && pk[q] >= 0) {
      const int64_t g = (row0 + i) * ld + col0 + j;
      D[g] = own[e];
      if (P) P[g] = pk[q];
    }
  }
}

// --------------------------------------------------------------------------
// Lazy argmin recovery (shared by the K3 variants).  All 32 lanes of a warp
// call it with the same (gi, gj, target): target is min over the round's k of
// fl(D[gi][baseK+k] + D[baseK+k][gj]).  Lanes test 32 consecutive k at a time;
// the lowest k whose sum equals target (bit for bit, same rounding) is the k
// the sequential loop would have recorded.
// --------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void recover_argmin(const Real *__restrict__ D, int64_t ld,
                                               int32_t *__restrict__ P, int64_t gi, int64_t gj,
                                               Real target, int baseK, int mK, int lane) {
  const Real *arow = D + gi * ld + baseK;
  const Real *bcol = D + (int64_t)baseK * ld + gj;
  for (int k0 = 0; k0 < mK; k0 += 32) {
    const int k = k0 + lane;
    bool hit = false;
    if (k < mK) hit = (add_rn(arow[k], bcol[(int64_t)k * ld]) == target);
    const unsigned bal = __ballot_sync(kFullMask, hit);
    if (bal) {
      if (lane == 0) P[gi * ld + gj] = baseK + k0 + (__ffs(bal) - 1);
      return;
    }
  }
}

// --------------------------------------------------------------------------
// K1 (FP32): phase 1 with the register-resident closure of minplus_f32.cuh.
// K3 (FP32): phase 4, one 128 x 128 block product per CTA (minplus_f32.cuh).
// Grid: (R-1)^2 CTAs in row-major (I', J') order over the blocks I, J != r,
// so consecutive CTAs share the column-panel block A and sweep the row panel.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(mp32::THREADS)
    fw_phase1_diag_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r) {
  __shared__ mp32::DiagSmem sm;
  const int base = r * mp32::T;
  mp32::diag_closure(D, ld, P, base, min(mp32::T, n - base), sm);
}

__global__ void __launch_bounds__(mp32::THREADS, 2)
    fw_phase3_minplus_f32(float *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r,
                          int R, int vec_ok) {
  using mp32::T;
  __shared__ __align__(16) mp32::Smem sm;
  const int Rm = R - 1;
  int I = blockIdx.x / Rm, J = blockIdx.x % Rm;
  I += (I >= r);
  J += (J >= r);
  const int baseI = I * T, baseJ = J * T, baseK = r * T;
  mp32::block_product(D, ld, P, baseI, baseJ, baseK, min(T, n - baseI), min(T, n - baseJ),
                      min(T, n - baseK), vec_ok, sm);
}

// --------------------------------------------------------------------------
// K3 (FP64): phase 4 with native FP64 add and min.  TB = 64, 256 threads,
// 4 x 4 outputs per thread (rows ty + 16 r, cols tx + 16 c), k slabs of 16
// staged k-major in shared memory.  Same epilogue and P recovery as FP32.
// --------------------------------------------------------------------------
namespace k3f64 {
constexpr int T = 64;
constexpr int THREADS = 256;
constexpr int KS = 16;
}  // namespace k3f64

__global__ void __launch_bounds__(k3f64::THREADS)
    fw_phase3_minplus_f64(double *__restrict__ D, int64_t ld, int32_t *__restrict__ P, int n, int r,
                          int R) {
  using namespace k3f64;
  __shared__ double As[KS][T + 1];
  __shared__ double Bs[KS][T];
  const int Rm = R - 1;
  int I = blockIdx.x / Rm, J = blockIdx.x % Rm;
  I += (I >= r);
  J += (J >= r);
  const int baseI = I * T, baseJ = J * T, baseK = r * T;
  const int mI = min(T, n - baseI), mJ = min(T, n - baseJ), mK = min(T, n - baseK);
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 4, tx = tid & 15;
  const double INF = inf<double>();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = INF;

  for (int k0 = 0; k0 < mK; k0 += KS) {
    __syncthreads();
    for (int e = tid; e < T * KS; e += THREADS) {
      const int i = e / KS, k = e % KS;  // A[i][k0+k] -> As[k][i]
      As[k][i] = (i < mI && k0 + k < mK) ? D[(int64_t)(baseI + i) * ld + baseK + k0 + k] : INF;
      const int kb = e / T, j = e % T;  // B[k0+kb][j] -> Bs[kb][j]
      Bs[kb][j] = (j < mJ && k0 + kb < mK) ? D[(int64_t)(baseK + k0 + kb) * ld + baseJ + j] : INF;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KS; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty + 16 * q];
        b[q] = Bs[k][tx + 16 * q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmin(acc[x][y], __dadd_rn(a[x], b[y]));
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = ty + 16 * x;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int j = tx + 16 * y;
      bool imp = false;
      if (i < mI && j < mJ) {
        double *dst = D + (int64_t)(baseI + i) * ld + baseJ + j;
        imp = acc[x][y] < *dst;
        if (imp) *dst = acc[x][y];
      }
      if (P) {
        unsigned bal = __ballot_sync(kFullMask, imp);
        while (bal) {
          const int src = __ffs(bal) - 1;
          bal &= bal - 1;
          const double tgt = __shfl_sync(kFullMask, acc[x][y], src);
          const int si = __shfl_sync(kFullMask, i, src), sj = __shfl_sync(kFullMask, j, src);
          recover_argmin<double>(D, ld, P, baseI + si, baseJ + sj, tgt, baseK, mK, lane);
        }
      }
    }
  }
}

// --------------------------------------------------------------------------
// Phase timing hook: when enabled, each phase launch is bracketed by two CUDA
// events recorded on the launch stream; apsp_profile_collect sums them.
// --------------------------------------------------------------------------
}  // namespace apsp
#include <mutex>
#include <vector>
namespace apsp {
struct PhaseRec {
  int phase;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<PhaseRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII bracket around one launch (no-op when profiling is off).
struct PhaseScope {
  bool on;
  PhaseRec rec;
  cudaStream_t s;
  PhaseScope(int phase, cudaStream_t st) : on(false), s(st) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on) return;
    on = true;
    rec.phase = phase;
    rec.a = prof_event();
    rec.b = prof_event();
    cudaEventRecord(rec.a, s);
  }
  ~PhaseScope() {
    if (!on) return;
    cudaEventRecord(rec.b, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_recs.push_back(rec);
  }
};

// --------------------------------------------------------------------------
// Host side: argument checks and the round loop (all launches on `stream`).
// --------------------------------------------------------------------------
constexpr int kMaxN = 65536;

template <typename Real> struct Cfg;
template <> struct Cfg<float> {
  static constexpr int T = mp32::T, T2 = 1024;
};
template <> struct Cfg<double> {
  static constexpr int T = 64, T2 = 512;
};

static int g_smem_p2f[64], g_smem_p2d[64];

static int launch_phase3(float *D, int64_t ld, int32_t *P, int n, int r, int R, cudaStream_t s) {
  const int vec_ok = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
  fw_phase3_minplus_f32<<<(R - 1) * (R - 1), mp32::THREADS, 0, s>>>(D, ld, P, n, r, R, vec_ok);
  return APSP_OK;
}
static void launch_phase1(float *D, int64_t ld, int32_t *P, int n, int r, cudaStream_t s) {
  fw_phase1_diag_f32<<<1, mp32::THREADS, 0, s>>>(D, ld, P, n, r);
}
static void launch_phase1(double *D, int64_t ld, int32_t *P, int n, int r, cudaStream_t s) {
  constexpr int T = 64, T1 = 512;
  fw_phase1_diag<double, T, T1><<<1, T1, T * T * sizeof(double), s>>>(D, ld, P, n, r);
}
static int launch_phase3(double *D, int64_t ld, int32_t *P, int n, int r, int R, cudaStream_t s) {
  fw_phase3_minplus_f64<<<(R - 1) * (R - 1), k3f64::THREADS, 0, s>>>(D, ld, P, n, r, R);
  return APSP_OK;
}

template <typename Real>
static int run_fw(Real *D, int64_t n64, int64_t ld, int32_t *P, void *stream) {
  if (n64 < 0 || n64 > kMaxN) return APSP_EINVAL;
  if (n64 == 0) return APSP_OK;
  if (!D || ld < n64) return APSP_EINVAL;
  const int n = (int)n64;
  constexpr int T = Cfg<Real>::T, T2 = Cfg<Real>::T2;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int smem2 = 2 * T * T * (int)sizeof(Real);
  auto k2 = fw_phase2_panels<Real, T, T2>;
  const int st = ensure_smem(k2, smem2, sizeof(Real) == 4 ? g_smem_p2f : g_smem_p2d);
  if (st) return st;
  cudaGetLastError();  // clear any stale error so the checks below are ours
  if (P) {
    const int64_t total = n64 * n64;
    const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
    PhaseScope ps(0, s);
    fw_path_init<<<blocks, 256, 0, s>>>(P, n64, ld);
  }
  const int R = (n + T - 1) / T;
  for (int r = 0; r < R; ++r) {
    {
      PhaseScope ps(1, s);
      launch_phase1(D, ld, P, n, r, s);
    }
    if (R > 1) {
      {
        PhaseScope ps(2, s);
        k2<<<2 * (R - 1), T2, smem2, s>>>(D, ld, P, n, r, R);
      }
      PhaseScope ps(3, s);
      launch_phase3(D, ld, P, n, r, R, s);
    }
  }
  return status_from(cudaGetLastError());
}

}  // namespace apsp

APSP_EXPORT int apsp_fw_f32(float *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream) {
  return apsp::run_fw<float>(d_dist, n, ld, d_path, stream);
}

APSP_EXPORT int apsp_fw_f64(double *d_dist, int64_t n, int64_t ld, int32_t *d_path, void *stream) {
  return apsp::run_fw<double>(d_dist, n, ld, d_path, stream);
}

APSP_EXPORT int apsp_fw_block_size(int elem_bytes) {
  return elem_bytes == 4 ? apsp::Cfg<float>::T : elem_bytes == 8 ? apsp::Cfg<double>::T : 0;
}

APSP_EXPORT const char *apsp_status_string(int status) {
  switch (status) {
    case APSP_OK: return "APSP_OK";
    case APSP_EINVAL: return "APSP_EINVAL: invalid argument";
    case APSP_ECUDA: return "APSP_ECUDA: CUDA call or launch failed";
    case APSP_ENOMEM: return "APSP_ENOMEM: device allocation failed";
    case APSP_EUNSUPPORTED: return "APSP_EUNSUPPORTED: outside supported sizes";
    case APSP_ETOODEEP: return "APSP_ETOODEEP: path recursion deeper than the walk stack";
    default: return "APSP: unknown status";
  }
}

APSP_EXPORT int apsp_version(void) { return 100; }

APSP_EXPORT int apsp_profile_enable(int on) {
  std::lock_guard<std::mutex> g(apsp::g_prof_mu);
  for (auto &r : apsp::g_prof_recs) {
    apsp::g_prof_pool.push_back(r.a);
    apsp::g_prof_pool.push_back(r.b);
  }
  apsp::g_prof_recs.clear();
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
