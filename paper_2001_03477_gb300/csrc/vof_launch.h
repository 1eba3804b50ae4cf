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

// Scratch of one sweep (kernel A -> kernels M, F, U): T of the cells whose
// (c, e) differs from the previous cell of their line (kernel F adds the
// listed others), the per-warp lists of cells that are not no-ops with their
// counts, per-CTA partial sums of the clipped volume (or, when partial is
// null, atomics into diag), per-warp staging of mixed cells and run ends,
// the grid-wide lists of mixed cells and of face items with their counters,
// the planes of the mixed cells and the face fluxes F, G.
struct SweepScratch {
  double* T;
  uint32_t* list;
  int* count;
  double* partial;
  double* diag;
  uint32_t* mlist;   // per-warp staging lists of mixed cells
  uint32_t* rlist;   // per-warp staging lists of run ends
  int* counters;     // [0] mixed cells, [1] face items (zeroed before kernel A)
  uint32_t* gmix;    // grid-wide list of mixed cells, in no fixed order
  uint32_t* gface;   // grid-wide face items (cell << 1 | side), no fixed order
  double* plane;     // [N][4]: m0, m1, m2, alpha of the listed mixed cells
  double* F;         // face arrays of the axis (face layout of the velocities)
  double* G;
};

struct SweepPlan {
  dim3 gridA, blockA;
  int cap;          // list capacity per warp of kernel A
  long long nsub;   // number of lists (warps of kernel A)
  unsigned gridB;   // CTAs of kernel U (8 lists each)
};

SweepPlan sweep_plan(int axis, const GridDev& g);
size_t sweep_scratch_bytes(const GridDev& g);
SweepScratch carve_sweep_scratch(int axis, const GridDev& g, void* ws, double* partials, double* diag);

int sweep_blocks(int axis, const GridDev& g);

// Scratch of the shift: per-warp lists of moving mixed cells with their
// counts (fixed order), a grid-wide list of the same cells and one of the
// receivers (no fixed order) with their counters, and per cell: the plane
// (m0, m1, m2, alpha) and shift |m|_2 dd of a moving mixed cell, the mask of
// receivers it settles, and the volume swept into a receiver.
struct ShiftScratch {
  uint32_t* list;
  int* count;
  int* counters;  // [0] non-edge cells, [1] edge cells, [2] receivers
  uint32_t* gmix; // non-edge cells from the front, edge cells from the back
  uint32_t* recv;
  double* plane;  // [N][4]
  double* shift;  // [N]
  double* sweep;  // [N]
  uint32_t* own;  // [N]
};

// CTAs of the shift's stream and sums kernels; their partial sums take
// kShiftPartialSets * shift_blocks rows of the SumOut
constexpr int kShiftPartialSets = 2;
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
