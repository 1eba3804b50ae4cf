// vof_prof.cu -- optional per-launch timing of the library's own kernels.
//
// Between vof_profile_begin() and vof_profile_end() every launch the library
// makes is followed by a CUDA event recorded on the launching stream; the
// times between consecutive events are the launches' durations (each
// includes the small gap before the launch starts).  The paper has no
// counterpart; this is instrumentation for roofline measurements.
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {
namespace {

struct Profiler {
  std::mutex mu;
  bool active = false;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> events;  // recorded this session
  std::vector<const char*> names;
  std::vector<cudaEvent_t> pool;    // created once, reused
};

Profiler& prof() {
  static Profiler p;
  return p;
}

std::atomic<bool> g_prof_on{false};  // fast path: no lock while not profiling

cudaEvent_t take_event(Profiler& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

void prof_mark(const char* name, cudaStream_t st) {
  if (!g_prof_on.load(std::memory_order_acquire)) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.active) return;
  cudaEvent_t e = take_event(p);
  if (!e) return;
  if (cudaEventRecord(e, st) != cudaSuccess) {
    p.pool.push_back(e);
    return;
  }
  p.events.push_back(e);
  p.names.push_back(name);
}

}  // namespace vofgb

using namespace vofgb;

extern "C" {

vof_status vof_profile_begin(void* stream) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (p.active) return VOF_EINVAL;
  for (cudaEvent_t e : p.events) p.pool.push_back(e);
  p.events.clear();
  p.names.clear();
  if (!p.start && cudaEventCreate(&p.start) != cudaSuccess) return VOF_ECUDA;
  if (cudaEventRecord(p.start, (cudaStream_t)stream) != cudaSuccess) return VOF_ECUDA;
  p.active = true;
  g_prof_on.store(true, std::memory_order_release);
  return VOF_OK;
}

int vof_profile_end(float* ms, const char** names, int max_entries) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.active) return -1;
  p.active = false;
  g_prof_on.store(false, std::memory_order_release);
  const int n = (int)p.events.size();
  if (n > 0 && cudaEventSynchronize(p.events.back()) != cudaSuccess) return -1;
  cudaEvent_t prev = p.start;
  for (int i = 0; i < n; ++i) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, prev, p.events[i]) != cudaSuccess) t = -1.0f;
    if (i < max_entries) {
      if (ms) ms[i] = t;
      if (names) names[i] = p.names[i];
    }
    prev = p.events[i];
  }
  return n;
}

}  // extern "C"
