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

// Scratch of one sweep (kernel A -> kernel B): T of the cells whose (c, e)
// differs from the previous cell of their line, the per-warp lists of cells
// that are not no-ops with their counts, and per-CTA partial sums of the
// clipped volume (or, when partial is null, atomics into diag).
struct SweepScratch {
  double* T;
  uint32_t* list;
  int* count;
  double* partial;
  double* diag;
  uint32_t* mlist;  // per-warp lists of mixed cells
  int* mcount;
  double* plane;    // [N][4]: m0, m1, m2, alpha of the listed mixed cells
};

struct SweepPlan {
  dim3 gridA, blockA;
  int cap;          // list capacity per warp of kernel A
  long long nsub;   // number of lists (warps of kernel A)
  unsigned gridB;   // CTAs of kernel B (8 lists each)
};

SweepPlan sweep_plan(int axis, const GridDev& g);
size_t sweep_scratch_bytes(const GridDev& g);
SweepScratch carve_sweep_scratch(int axis, const GridDev& g, void* ws, double* partials, double* diag);

int sweep_blocks(int axis, const GridDev& g);

// Scratch of the shift: per-warp lists of moving mixed cells with their
// counts, and the plane (m0, m1, m2, alpha) and shift |m|_2 dd of every
// listed cell, stored densely at the cell's index.
struct ShiftScratch {
  uint32_t* list;
  int* count;
  double* plane;  // [N][4]
  double* shift;  // [N]
};

// CTAs of each of the three shift kernels; their partial sums take
// 3 * shift_blocks rows of the SumOut
int shift_blocks(const GridDev& g);
size_t shift_scratch_bytes(const GridDev& g);
ShiftScratch carve_shift_scratch(const GridDev& g, void* ws);

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SweepScratch sc, cudaStream_t st);

cudaError_t launch_energy(int axis, const GridDev& g, const double* c_before, const double* c_after,
                          const double* e_in, double* e_out, const double* F, const double* uf, uint8_t* state,
                          double* theta, cudaStream_t st);

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, ShiftScratch sc, SumOut sums,
                         cudaStream_t st);

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
