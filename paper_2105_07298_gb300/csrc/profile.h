// Host-side phase timing shared by the translation units (internal).  When
// enabled through apsp_profile_enable, each bracketed launch gets two CUDA
// events on its stream; apsp_profile_collect sums them per phase.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

namespace apsp {

struct PhaseRec {
  int phase;
  cudaEvent_t a, b;
};

// State lives in fw_single.cu.
extern std::mutex g_prof_mu;
extern bool g_prof_on;
extern std::vector<PhaseRec> g_prof_recs;
extern std::vector<cudaEvent_t> g_prof_pool;

inline cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII bracket around the launches of one phase (no-op when profiling is off).
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

}  // namespace apsp
