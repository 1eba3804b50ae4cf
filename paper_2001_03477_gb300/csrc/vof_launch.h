// vof_launch.h -- internal launchers shared by the library's translation
// units (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "vof_device.cuh"

namespace vofgb {

// Per-block partial sums: a kernel either writes its block's partials to
// `partials[block * stride + k]` (deterministic, reduced later in a fixed
// order) or, when partials == nullptr, adds them to `diag[k]` with atomics.
struct SumOut {
  double* partials;
  int stride;
  double* diag;
};

int sweep_blocks(int axis, const GridDev& g);
int shift_blocks(const GridDev& g);

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SumOut sums, cudaStream_t st);

cudaError_t launch_energy(int axis, const GridDev& g, const double* c_before, const double* c_after,
                          const double* e_in, double* e_out, const double* F, const double* uf, uint8_t* state,
                          double* theta, cudaStream_t st);

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, SumOut sums, cudaStream_t st);

cudaError_t launch_reconstruct(const GridDev& g, const double* c, double* m, double* alpha, uint8_t* mixed,
                               cudaStream_t st);

cudaError_t launch_reduce(const double* partials, int nblocks, int stride, int k0, int nk, double* out,
                          cudaStream_t st);

cudaError_t launch_sum_fields(const GridDev& g, const double* c, const double* e, double* partials,
                              int* nblocks_out, cudaStream_t st);

// sticky device status word (iteration caps, CFL > 1): bit flags
enum : int { DEV_CFL = 1 };
int* device_status_ptr();

}  // namespace vofgb
