// Bulk asynchronous copies (TMA engine, 1-D form) and mbarrier helpers for
// sm_103a, as inline PTX.  Internal header.
//
// A copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory completes on an mbarrier as transaction bytes.
// Every wait is bounded: after kWaitLimit polls it reports failure, and the
// caller records APSP_ETIMEOUT in the translation unit's error word
// (report_wait_timeout) and leaves instead of spinning forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/apsp_fw.h"

namespace apsp {

constexpr uint32_t kWaitLimit = 1u << 22;

// Error word the kernels of a translation unit set when a bounded wait runs
// out (read back by apsp_device_status).
static __device__ int g_device_error = 0;

// Records that a bounded wait ran out (any thread may call it).
__device__ __forceinline__ void report_wait_timeout() { atomicExch(&g_device_error, APSP_ETIMEOUT); }

// Host side: returns and clears this translation unit's error word (APSP_OK if
// no wait ran out since the last call; APSP_ECUDA if the copy itself failed).
static inline int take_tu_device_error() {
  int v = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_device_error, sizeof(int)) != cudaSuccess) return APSP_ECUDA;
  if (v != 0 && cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int)) != cudaSuccess) return APSP_ECUDA;
  return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Invalidates a barrier whose phases have all completed, so that its memory
// can be initialised again (or used for anything else).
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Makes barrier initialisation visible to the async proxy (the copy engine).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy writes of global memory before
// later async-proxy (bulk copy) reads of it.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Orders earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete; false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace apsp
