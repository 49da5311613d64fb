// Batched Floyd-Warshall: thousands of independent graphs of uneven size in
// one persistent launch (an extension; the paper solves one matrix at a time).
//
// Work distribution: the plan orders the graphs largest first (longest
// processing time first) and the CTAs of a grid sized to fill every SM pop
// graph indices from one atomic counter.  A CTA solves its graph alone, so no
// CTA ever waits on another.
//
// Per graph (n_g <= 1024, row-major, ld = n_g) the CTA runs the blocked FW of
// §2.2 with TB = 128 on the matrix in global memory (it stays in L2):
//   phase 1     register-resident closure of the diagonal block (Algorithm 1
//               restricted to the block, k sequential);
//   phases 2+3  row block (r,J) <- min(C, D*(r,r) (x) C) and column block
//               (I,r) <- min(C, C (x) D*(r,r)): once the diagonal block is
//               closed, the sequential k loop over a panel block equals one
//               min-plus product with the closed block, so these phases use
//               the same register-blocked product as phase 4;
//   phase 4     (I,J) <- min(C, D(I,r) (x) D(r,J)).
// On integer-valued weights all sums are exact and D equals every other
// correct FW; on real weights the phase-2/3 products round differently from
// the sequential loop (one sum through the closed block instead of a chain of
// sums), within the same error bound.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "minplus_f32.cuh"

namespace apsp {

constexpr int kBatchedMaxN = 1024;

// Size classes and their kernel variants (chosen by the autotuner, see
// apsp_batched_set_variant).  A variant fixes the block edge and register
// tile used for the class's graphs inside the one launch:
//   variant 0: TB = 128, 8 x 8 outputs per thread
//   variant 1: TB = 64,  4 x 4 outputs per thread (less padding for small n)
constexpr int kNumClasses = 4;
static const int32_t kClassLo[kNumClasses] = {1, 65, 129, 257};
static const int32_t kClassHi[kNumClasses] = {64, 128, 256, kBatchedMaxN};
__host__ __device__ constexpr int class_of_n(int32_t n) {
  return n <= 64 ? 0 : n <= 128 ? 1 : n <= 256 ? 2 : 3;
}
constexpr int kNumVariants = 2;
static int g_variant[kNumClasses] = {1, 0, 0, 0};

static int class_of(int32_t n) { return class_of_n(n); }

union BatchedSmem {
  mp32::SmemT<128> prod128;
  mp32::SmemT<64> prod64;
  mp32::DiagSmemT<128> diag128;
  mp32::DiagSmemT<64> diag64;
};

template <int TM>
__device__ __forceinline__ void solve_graph_f32(float *__restrict__ D, int32_t *__restrict__ P,
                                                int n, BatchedSmem &smu) {
  constexpr int T = 16 * TM;
  auto &prod = *reinterpret_cast<mp32::SmemT<T> *>(&smu);
  auto &diag = *reinterpret_cast<mp32::DiagSmemT<T> *>(&smu);
  const int ld = n;
  const int vec_ok = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
  const int R = (n + T - 1) / T;
  for (int r = 0; r < R; ++r) {
    const int base = r * T, m = min(T, n - base);
    __syncthreads();
    mp32::diag_closure<TM>(D, ld, P, base, m, diag);
    __syncthreads();
    for (int J = 0; J < R; ++J) {
      if (J == r) continue;
      mp32::block_product<TM>(D, ld, P, base, J * T, base, m, min(T, n - J * T), m, vec_ok, prod);
    }
    for (int I = 0; I < R; ++I) {
      if (I == r) continue;
      mp32::block_product<TM>(D, ld, P, I * T, base, base, min(T, n - I * T), m, m, vec_ok, prod);
    }
    __syncthreads();
    for (int I = 0; I < R; ++I) {
      if (I == r) continue;
      for (int J = 0; J < R; ++J) {
        if (J == r) continue;
        mp32::block_product<TM>(D, ld, P, I * T, J * T, base, min(T, n - I * T), min(T, n - J * T), m,
                                vec_ok, prod);
      }
    }
  }
  __syncthreads();
}

// Work item t: graph order[t] & 0x3fffffff, variant order[t] >> 30.
__global__ void __launch_bounds__(mp32::THREADS, 2)
    fw_batched_persistent_f32(float *__restrict__ Dp, int32_t *__restrict__ Pp,
                              const int32_t *__restrict__ order, const int32_t *__restrict__ ns,
                              const int64_t *__restrict__ offs, int num, int *__restrict__ counter) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchedSmem &sm = *reinterpret_cast<BatchedSmem *>(smem_raw);
  __shared__ int s_next;
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
    if (variant == 1)
      solve_graph_f32<4>(D, P, n, sm);
    else
      solve_graph_f32<8>(D, P, n, sm);
  }
}

}  // namespace apsp

struct apsp_batched_plan {
  int32_t num;
  int32_t *d_order;
  int32_t *d_n;
  int64_t *d_off;
  int *d_counter;
  int grid;
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
// the variant of its size class in bits 30-31.
std::vector<int32_t> lpt_order(const int32_t *h_n, int32_t num) {
  std::vector<int32_t> order(num);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return h_n[a] > h_n[b]; });
  for (auto &g : order) g |= apsp::g_variant[apsp::class_of(h_n[g])] << 30;
  return order;
}

int g_smem_batched[64];

int grid_for(int32_t num) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (apsp::ensure_smem(apsp::fw_batched_persistent_f32, (int)sizeof(apsp::BatchedSmem), g_smem_batched))
    return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, apsp::fw_batched_persistent_f32,
                                                    apsp::mp32::THREADS,
                                                    sizeof(apsp::BatchedSmem)) != cudaSuccess)
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
    std::vector<int32_t> order = lpt_order(h_n, num);
    if (cudaMemcpy(p->d_order, order.data(), (size_t)num * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      apsp_batched_plan_destroy(p);
      return APSP_ECUDA;
    }
  }
  p->grid = grid_for(num);
  if (p->grid < 0) {
    apsp_batched_plan_destroy(p);
    return APSP_ECUDA;
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
  apsp::fw_batched_persistent_f32<<<p->grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
      d_dist, d_path, p->d_order, p->d_n, p->d_off, p->num, p->d_counter);
  return apsp::status_from(cudaGetLastError());
}

APSP_EXPORT int apsp_fw_batched_f32(float *d_dist, int32_t *d_path, const int32_t *h_n,
                                    const int64_t *h_off, int32_t num, void *stream) {
  int st = validate(h_n, h_off, num);
  if (st) return st;
  if (num == 0) return APSP_OK;
  if (!d_dist) return APSP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int32_t> order = lpt_order(h_n, num);
  // one scratch block: counter | order | n | offsets (stream-ordered allocation)
  const size_t bytes = 16 + (size_t)num * 8 + (size_t)num * 8 + (size_t)num * 8;
  char *scratch = nullptr;
  cudaGetLastError();
  if (cudaMallocAsync((void **)&scratch, bytes, s) != cudaSuccess) return APSP_ENOMEM;
  int *d_counter = reinterpret_cast<int *>(scratch);
  int32_t *d_order = reinterpret_cast<int32_t *>(scratch + 16);
  int32_t *d_n = d_order + num;
  int64_t *d_off = reinterpret_cast<int64_t *>(scratch + 16 + (((size_t)num * 8 + 15) & ~(size_t)15));
  // offsets region starts 16-byte aligned after order and n (2 * 4 * num bytes)
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_order, order.data(), (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice, s);
  int grid = grid_for(num);
  if (e == cudaSuccess && grid > 0) {
    apsp::fw_batched_persistent_f32<<<grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
        d_dist, d_path, d_order, d_n, d_off, num, d_counter);
    e = cudaGetLastError();
  }
  // Copies from pageable host memory have consumed their sources when they
  // return, so `order` may go out of scope; the scratch is freed in stream order.
  cudaFreeAsync(scratch, s);
  if (grid <= 0) return APSP_ECUDA;
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
// a device address): the first call on each device looks its address up with
// cudaGetSymbolAddress while that device is current and caches it.  All calls
// share the array and it keeps the previous call's contents; each call
// resets the counter it needs.  Calls that overlap on the GPU (other streams,
// other host threads) race on the array and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace apsp {

constexpr int kNoAllocMaxGraphs = 65536;
constexpr size_t kNoAllocBytes = 16 + (size_t)kNoAllocMaxGraphs * (4 + 4 + 8);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static unsigned char *g_noalloc_addr[64];  // device address of g_noalloc_scratch, per device

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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APSP_ECUDA;
  if (!apsp::g_noalloc_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, apsp::g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return APSP_ECUDA;
    }
    apsp::g_noalloc_addr[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *base = apsp::g_noalloc_addr[dev];
  int *d_counter = reinterpret_cast<int *>(base);
  int32_t *d_order = reinterpret_cast<int32_t *>(base + 16);
  int32_t *d_n = d_order + apsp::kNoAllocMaxGraphs;
  int64_t *d_off = reinterpret_cast<int64_t *>(d_n + apsp::kNoAllocMaxGraphs);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = grid_for(num);
  if (grid <= 0) return APSP_ECUDA;
  cudaGetLastError();
  cudaError_t e = cudaMemcpyAsync(d_n, h_n, (size_t)num * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_off, (size_t)num * 8, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return APSP_ECUDA;
  apsp::fw_batched_order<<<1, 1024, 0, s>>>(d_n, num, d_order, d_counter, apsp::g_variant[0],
                                            apsp::g_variant[1], apsp::g_variant[2], apsp::g_variant[3]);
  apsp::fw_batched_persistent_f32<<<grid, apsp::mp32::THREADS, sizeof(apsp::BatchedSmem), s>>>(
      d_dist, d_path, d_order, d_n, d_off, num, d_counter);
  return apsp::status_from(cudaGetLastError());
}
