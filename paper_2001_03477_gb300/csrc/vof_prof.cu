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

// ---------------------------------------------------------------------------
// FP64 issue-rate probe (instrumentation): every thread runs 8 independent
// chains of `iters` dependent FP64 operations -- fused multiply-adds
// (op 0, two flops each) or adds (op 1, one flop) -- and stores one value,
// so the FP64 pipes of every SM stay busy and nothing else is on the
// critical path.  Timed by the caller with CUDA events, it gives the
// part's measured FP64 rate for the roofline of FP64-bound kernels.
// ---------------------------------------------------------------------------
namespace vofgb {
__global__ void __launch_bounds__(256) k_fp64_probe(int op, long iters, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = 1.0 + 1e-9 * t, a1 = a0 + 1e-3, a2 = a0 + 2e-3, a3 = a0 + 3e-3;
  double a4 = a0 + 4e-3, a5 = a0 + 5e-3, a6 = a0 + 6e-3, a7 = a0 + 7e-3;
  const double x = 0.9999999, y = 1e-7;
  if (op == 0) {
#pragma unroll 4
    for (long i = 0; i < iters; ++i) {
      a0 = fma(a0, x, y); a1 = fma(a1, x, y); a2 = fma(a2, x, y); a3 = fma(a3, x, y);
      a4 = fma(a4, x, y); a5 = fma(a5, x, y); a6 = fma(a6, x, y); a7 = fma(a7, x, y);
    }
  } else {
#pragma unroll 4
    for (long i = 0; i < iters; ++i) {
      a0 += y; a1 += y; a2 += y; a3 += y; a4 += y; a5 += y; a6 += y; a7 += y;
    }
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}
}  // namespace vofgb

extern "C" vof_status vof_fp64_probe(int op, long iters, int blocks, double* out, void* stream) {
  if ((op != 0 && op != 1) || iters < 1 || blocks < 1 || !out) return VOF_EINVAL;
  vofgb::k_fp64_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(op, iters, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vofgb::set_last_cuda_error((int)e);
    return VOF_ECUDA;
  }
  return VOF_OK;
}
