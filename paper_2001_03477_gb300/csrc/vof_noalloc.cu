// vof_noalloc.cu -- a time step that allocates nothing and takes no
// workspace from the caller.
//
// Some callers cannot allocate device memory when they step the solver:
// code that runs inside a host callback or another library's error path
// where the CUDA allocator must not be entered, embedders whose memory is
// fully reserved up front by their own pool and who cannot hand out an
// extra buffer, or tools that drive a few steps on a small grid and have no
// allocator of their own.  For them vof_step_noalloc() runs the same time
// step as vof_step() (in place on the caller's c and e), but its scratch
// space (the frozen-state flags and Theta, the per-sweep lists, planes and
// face fluxes, the per-CTA partial sums) lives in one fixed array in device
// memory that the library reserves when it is loaded.
//
// Limits and rules for callers:
//   * the grid may have at most VOF_NOALLOC_MAX_CELLS cells (64^3), and its
//     step workspace must fit the array (it does for every such grid with
//     at least 8 cells along each axis; thinner grids need more list space);
//     other grids are rejected with VOF_EINVAL before anything is launched;
//   * every GPU on which the library is loaded holds the array (40 MiB)
//     until the process exits;
//   * all calls share the one array per device: two calls whose kernels
//     overlap on the GPU (different streams, or different host threads on
//     the same device without ordering) race on it and give wrong results;
//     order them on one stream or synchronise between them;
//   * the array keeps whatever the previous call left in it; the step
//     itself clears the parts that must start at zero (the frozen-state
//     flags) and overwrites the rest before reading it;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it; make
//     that first call before any stream capture is started on the device.
// The paper has no counterpart to this entry point.
#include <cstring>
#include <mutex>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(40) << 20;  // 40 MiB

// the scratch array; in host code this name is only a stand-in for the
// device symbol, never a usable address
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {nullptr};

// device address of the scratch array on the current device (looked up
// once per device, with that device current); nullptr on failure
void* scratch_on_current_device(int* cuda_err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    *cuda_err = (int)(e != cudaSuccess ? e : cudaErrorInvalidDevice);
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      *cuda_err = (int)(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" {

size_t vof_noalloc_scratch_bytes(void) { return kNoAllocBytes; }

vof_status vof_step_noalloc(const vof_grid* g, double* c, double* e, const double* u, const double* v,
                            const double* w, double dt, long step_index, const double* dd, double dd_uniform,
                            double* sums, void* stream) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return VOF_EINVAL;
  const long long cells = (long long)g->nx * g->ny * g->nz;
  if (cells > VOF_NOALLOC_MAX_CELLS) return VOF_EINVAL;
  const size_t need = vof_step_workspace_bytes(g);
  if (need == 0 || need > kNoAllocBytes) return VOF_EINVAL;
  int err = 0;
  void* ws = scratch_on_current_device(&err);
  if (!ws) {
    vofgb::set_last_cuda_error(err);
    return VOF_ECUDA;
  }
  return vof_step(g, c, e, u, v, w, dt, step_index, dd, dd_uniform, sums, ws, kNoAllocBytes, stream);
}

}  // extern "C"
