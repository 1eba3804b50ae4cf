// vof_launch.h -- internal launchers shared by the library's translation
// units (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/vofgb.h"
#include "vof_device.cuh"

namespace vofgb {

// Programmatic dependent launch between the kernels of one time step.  A
// kernel launched by launch_pdl may be scheduled before the kernel ahead of it
// on the stream has completed: once every CTA of that kernel has exited, its
// launch and CTA placement overlap the previous grid's completion and memory
// flush.  The wrapper of every such kernel calls pdl_wait() as its first
// statement: griddepcontrol.wait blocks until the previous grid has completed
// and its writes are visible, the same ordering as a plain launch, so nothing
// is read early.  It returns at once when the kernel was launched without the
// attribute.  No kernel signals its dependents before it exits
// (griddepcontrol.launch_dependents): on the 256^3 step that placed the next
// kernel's waiting CTAs on the SMs that happened to be free, unevenly, and the
// step took 1.05 ms instead of 0.83 ms (0.88 ms with plain launches).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);  // errors: cudaGetLastError()
}

// Virtual block index of a kernel body: the hardware's for a launch over one
// grid; in a grouped launch over many boxes (vof_batched_step without lanes)
// the CTA's box and its block within the box's own launch shape, from the
// group map.  Bodies use vb.b* / vb.g* where a single launch uses blockIdx /
// gridDim.
struct VB {
  unsigned bx, by, bz, gx, gy, gz;
};
__device__ __forceinline__ VB vb_self() { return VB{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z}; }

// Grouped launch: cta_box[blockIdx.x] = the box of the CTA, box_first[b] =
// its first CTA, gdim[b] = the box's own launch shape (x fastest).
struct GroupMap {
  const uint32_t* cta_box;
  const uint32_t* box_first;
  const uint3* gdim;
};
__device__ __forceinline__ VB vb_group(const GroupMap& m, unsigned& b) {
  b = __ldg(m.cta_box + blockIdx.x);
  const unsigned l = blockIdx.x - __ldg(m.box_first + b);
  const uint3 d = m.gdim[b];
  return VB{l % d.x, (l / d.x) % d.y, l / (d.x * d.y), d.x, d.y, d.z};
}

// A grouped launch's per-box arguments, copied once per CTA into shared
// memory (the struct's words spread over the threads) instead of loaded
// whole by every thread.
template <class T>
__device__ __forceinline__ const T& cta_args(const T* __restrict__ args, unsigned b, T& smem) {
  static_assert(sizeof(T) % 8 == 0 && alignof(T) >= 8, "argument structs are whole 8-byte words");
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(args + b);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&smem);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  for (int i = tid; i < (int)(sizeof(T) / 8); i += nthr) dst[i] = __ldg(src + i);
  __syncthreads();
  return smem;
}

// Sums.  Every kernel that sums produces one row of kNSums values per CTA,
// in one layout:
//   [kSumC] sum of c contributions   [kSumE] sum of e contributions
//   [kSumClip] clipped volume of the sweeps
//   [kSumShDc] shift: sum Delta c    [kSumUnpl] shift: volume clamped away
//   [kSumShDe] shift: sum Delta e
// and either writes it to partials[block * stride] (deterministic, reduced
// later in a fixed order) or, when partials == nullptr, adds each value k
// with map[k] >= 0 to diag[map[k]] with an atomic (nothing when diag is
// null too).
enum { kSumC = 0, kSumE, kSumClip, kSumShDc, kSumUnpl, kSumShDe, kNSums };
struct SumOut {
  double* partials;
  int stride;
  double* diag;
  signed char map[kNSums];
};
__host__ __device__ inline SumOut sums_to_partials(double* p, int stride) {
  SumOut s{p, stride, nullptr, {-1, -1, -1, -1, -1, -1}};
  return s;
}
inline SumOut sums_to_diag(double* diag, const signed char (&map)[kNSums]) {
  SumOut s{nullptr, kNSums, diag, {map[0], map[1], map[2], map[3], map[4], map[5]}};
  return s;
}

// Quiet tiles: 8^3 tiles whose cells, with a 3-cell halo, all hold the same
// (c, e) bits with c exactly 0 or 1 at the start of a time step.  No cell of
// such a tile changes in any of the step's three sweeps (each sweep's 7-cell
// window stays inside the uniform box, and the cells of the box outside the
// tile that the earlier sweeps' windows reach are themselves no-ops), and none
// is mixed when the shift runs, so the streaming kernels of an in-place step
// skip them.  quiet == nullptr: no tile is skipped.
constexpr int kTile = 8;
struct TileMap {
  const uint8_t* quiet;
  int nt[3];  // tiles per axis
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
  SumOut sums;       // per-CTA sums of kernel U: Delta c, Delta e, clipped volume
  TileMap tiles;     // quiet tiles (in-place steps only)
  int* stats;        // nullable: kernel U copies counters[0..1] here
  uint32_t* mlist;   // per-warp staging lists of mixed cells
  uint32_t* rlist;   // per-warp staging lists of run ends
  int* counters;     // [0] mixed cells, [1] face items at the front, [2] at the
                     // back (faces next to a mixed cell), [3] learned normals
                     // replaced by MYC; zeroed before kernel A
  uint32_t* gmix;    // grid-wide list of mixed cells, in no fixed order
  uint32_t* gface;   // grid-wide face items (cell << 1 | side), no fixed order
  uint32_t gface_cap;  // entries of gface (2 N)
  double* plane;     // [N][4]: m0, m1, m2, alpha of the listed mixed cells
  double* gplane;    // [2][N / n_axis][4]: planes of the ghost donors beyond the
                     // low / high zero-gradient end of each line (boundary
                     // cells that are mixed only)
  int* mlp_stat;     // nullable: kernel U copies counters[3] (learned normals
                     // replaced by MYC in this sweep) here
  double* F;         // face arrays of the axis (face layout of the velocities)
  double* G;
};

// kernel U walks the kernel-A lists in groups of this many consecutive
// lists, each group as one sequence of cells
constexpr int kUpdLists = 8;
constexpr int kUpdBatch = 4;  // groups a CTA of kernel U walks per scan

struct SweepPlan {
  dim3 gridA, blockA;
  int cap;          // list capacity per warp of kernel A
  long long nsub;   // number of lists (warps of kernel A)
  unsigned gridB;   // CTAs of kernel U (lpc lists each)
  int lpc;          // kernel-A lists per CTA of kernel U (groups of kUpdLists)
};

SweepPlan sweep_plan(int axis, const GridDev& g);
size_t sweep_scratch_bytes(const GridDev& g);
SweepScratch carve_sweep_scratch(int axis, const GridDev& g, void* ws, SumOut sums);

int sweep_blocks(int axis, const GridDev& g);

// Scratch of the shift: per-warp lists of moving mixed cells with their
// counts (fixed order; a warp owns up to 256 cells of one x row), a
// grid-wide list of the same cells and one of the receivers (no fixed order)
// with their counters, and per cell: the plane (m0, m1, m2, alpha), shift
// |m|_2 dd and shifted volume of a moving mixed cell, the mask of receivers
// it settles, and the volume swept into a receiver.
struct ShiftScratch {
  uint32_t* list;
  int* count;
  int* counters;  // [0] non-edge cells, [1] edge cells, [2] receivers
  uint32_t* gmix; // non-edge cells from the front, edge cells from the back
  uint32_t* recv;
  double* plane;  // [N][4]
  double* shift;  // [N]
  double* sweep;  // [N]
  double* cnew;   // [N] shifted volume of a moving mixed cell
  uint32_t* own;  // [N]
  // reach and claim are written (and cleared) by the stream kernel for
  // every cell it visits; the cells of quiet tiles it skips are never read
  uint8_t* reach; // [N] 1: moving mixed cell with shift < 0, 2: > 0, else 0
  uint32_t* claim;  // [N] receivers: bit 31 - b set by the reaching neighbour at offset index b
  TileMap tiles;  // quiet tiles (in-place steps only)
  int* stats;     // nullable: the sums kernel copies counters[0..2] here
};

// The shift's kernels: stream (lists; out of place also copies; sums c, e
// when `stream_sums` is given) and sums (applies and sums the changes).
// sum_blocks: CTAs of the sums kernel (rows it writes to its SumOut).
int shift_sum_blocks(const GridDev& g);
int shift_stream_blocks(const GridDev& g);
size_t shift_scratch_bytes(const GridDev& g);
ShiftScratch carve_shift_scratch(const GridDev& g, void* ws);

// Tiles: per-tile uniform flag and values, then the quiet map; the tile
// pass also sums c and e over the grid (per-CTA rows).
struct TileScratch {
  uint8_t* uni;
  double* vc;
  double* ve;
  uint8_t* quiet;
};
void tile_counts(const GridDev& g, int nt[3]);
bool tiles_usable(const GridDev& g);
int tile_blocks(const GridDev& g);
size_t tile_scratch_bytes(const GridDev& g);
TileScratch carve_tile_scratch(const GridDev& g, void* ws);
// The tile pass of a time step also clears the step's frozen-state flags
// (state[N], nullable) and its list counters (counters[kStepCounters],
// nullable), so that the step needs no memset.
constexpr int kStepCounters = 16;  // 4 per sweep axis, then the shift's 3; the last: the reduction's ticket
cudaError_t launch_tiles(const GridDev& g, const double* c, const double* e, TileScratch ts, SumOut sums,
                         uint8_t* state, int* counters, cudaStream_t st);

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SweepScratch sc, bool zero_counters, cudaStream_t st);

cudaError_t launch_energy(int axis, const GridDev& g, const double* c_before, const double* c_after,
                          const double* e_in, double* e_out, const double* F, const double* uf, uint8_t* state,
                          double* theta, cudaStream_t st);

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, ShiftScratch sc, SumOut stream_sums,
                         SumOut sums, bool zero_counters, cudaStream_t st);

cudaError_t launch_reconstruct(const GridDev& g, const double* c, double* m, double* alpha, uint8_t* mixed,
                               cudaStream_t st);

// out[k] = sum over b < nblocks of partials[b * stride + k0 + k], k < nk
struct ReduceJob {
  const double* partials;
  int nblocks, stride, k0, nk;
  double* out;
};
constexpr int kMaxReduceJobs = 4;
constexpr int kMaxReduceK = 8;      // outputs per job at most
constexpr int kReduceCTAs = 152;    // first-level CTAs per job
struct ReduceJobs {
  ReduceJob job[kMaxReduceJobs];
};
size_t reduce_scratch_bytes();
// one job's two levels in one launch; *ticket is zero before and after
cudaError_t launch_reduce_fused(const ReduceJob& job, double* scratch, int* ticket, cudaStream_t st);

// ---------------------------------------------------------------------------
// Grouped launches: one launch runs one kernel of the time step for every box
// of a batch (vof_group_*), each CTA on its box's arguments (from a table in
// device memory) with its virtual block index in the box's own launch shape.
// ---------------------------------------------------------------------------
struct SweepArgs {  // one box's in-place sweep along one axis
  GridDev g;
  double* c;
  double* e;
  const double* uf;
  uint8_t* state;
  double* theta;
  SweepScratch sc;
  int cap, nsub, ngrp;
  int* status;
};
struct TileArgs {
  GridDev g;
  const double* c;
  const double* e;
  TileScratch ts;
  int nt[3];
  SumOut sums;
  uint8_t* state;  // cleared by the tile pass
  int* counters;   // kStepCounters, cleared by the tile pass
};
struct ShiftArgs {
  GridDev g;
  double* c;
  double* e;
  const double* dd;
  double dd_uniform;
  ShiftScratch sc;
  SumOut sums;
  long long nw;
};
struct ReduceBox {  // one box's sum rows and its output
  const double* rows;
  int nblocks;
  double* out;
  double* scratch;  // kReduceCTAs x kMaxReduceK partials
};
cudaError_t launch_tiles_grp(const GroupMap& mt, const GroupMap& mq, const TileArgs* a, unsigned ct, unsigned cq,
                             cudaStream_t st);
// maps / ctas: [0] kernel A, [1] prep, [2] faces, [3] update
cudaError_t launch_sweep_grp(int axis, int f32, int youngs, const GroupMap* maps, const SweepArgs* a,
                             const unsigned* ctas, cudaStream_t st);
// maps / ctas: [0] stream, [1] planes, [2] own, [3] receivers, [4] sums
cudaError_t launch_shift_grp(const GroupMap* maps, const ShiftArgs* a, const unsigned* ctas, cudaStream_t st);
// m1: (box, part) CTAs of the first level; the second level runs one CTA per box
cudaError_t launch_reduce_grp(const GroupMap& m1, const ReduceBox* rb, unsigned ctas1, unsigned nbox,
                              cudaStream_t st);
// One box's arguments and launch shapes for every kernel of a grouped time
// step (vof_api.cu builds them exactly as vof_step carves its workspace).
struct StepBox {
  size_t cells;
  TileArgs tiles;
  SweepArgs sweep[3];
  ShiftArgs shift;
  ReduceBox red;
  dim3 grid_tiles, grid_stream[3], grid_shift_stream;
  unsigned grid_quiet, grid_update[3], grid_shift_sums;
};
// false for a grid vof_step refuses; ws: the box's step workspace
// (vof_step_workspace_bytes), sums: device double[VOF_NSUMS] or null
bool step_box(const vof_grid* g, double* c, double* e, const double* u, const double* v, const double* w,
              double dt, const double* dd, double dd_uniform, double* sums, char* ws, StepBox* out);
int shift_list_ctas();
long long shift_warps_of(const GridDev& g);
int prep_ctas();
dim3 shift_stream_grid_of(const GridDev& g);
unsigned quiet_blocks(const GridDev& g);

// per-launch timing (vof_profile_begin/end): records an event after a launch
void prof_mark(const char* name, cudaStream_t st);

// records the cudaError_t that vof_last_cuda_error() reports (for entry
// points outside vof_api.cu that return VOF_ECUDA)
void set_last_cuda_error(int err);

// sticky device status word (iteration caps, CFL > 1): bit flags
enum : int { DEV_CFL = 1, DEV_WAIT = 2 };
int* device_status_ptr();

// Mass transfer rate (vof_mdot.cu): workspace size, the launch of its four
// kernels, and its counters ([0] mixed cells, [1] band cells) in a workspace.
size_t mdot_scratch_bytes(size_t N);
cudaError_t launch_mass_transfer(const GridDev& g, double h, const double* c, const double* e, double k_l, double k_g,
                                 double h_fg, double dd_per_mdot, double* mdot, double* d_gamma, double* grad_n,
                                 double* dd, void* workspace, cudaStream_t st);
int* mdot_counters(const GridDev& g, void* workspace);

// Velocity extension (vof_ext.cu): workspace size and the whole solve;
// *status: 0 ok, 1 no free-flow face (nothing written), 2 not converged.
size_t ext_scratch_bytes(size_t N);
cudaError_t launch_velocity_extension(const GridDev& g, double h, const double* c, const double* mdot, double rho_l,
                                      double rho_g, double dt, double tol, int max_iter, double* u, double* v,
                                      double* w, double* ut, double* vt, double* wt, void* workspace,
                                      cudaStream_t st, int* iters_out, double* res_out, int* status);

// Learned interface normal (vof_mlp.cu): packed parameter size, packing of
// the FP32 master parameters, forward pass and normals (with MYC fallback)
// on explicit stencils, the normals of a sweep's mixed cells, and one
// training step (forward, backward, Adam).
size_t mlp_packed_bytes();
int mlp_param_count();
cudaError_t launch_mlp_pack(const float* master, void* packed, cudaStream_t st);
cudaError_t launch_mlp_forward(const void* params, const double* X, long n, float* y, cudaStream_t st);
cudaError_t launch_mlp_normals(const void* params, const double* X, long n, double* m, uint8_t* flag,
                               int* nfallback, cudaStream_t st);
cudaError_t launch_mlp_sweep_normals(const GridDev& g, const double* c, const SweepScratch& sc, cudaStream_t st);
cudaError_t launch_mlp_train_step(const double* X, const double* N, long ntrain, int batch, unsigned long long seed,
                                  long step, float* master, float* mom, float* vel, void* packed, float* partial,
                                  float* loss_part, const long* idx_fixed, float lr, float beta1, float beta2,
                                  float eps, float* grad_out, float* loss_out, cudaStream_t st);

// Heat diffusion (vof_diffuse.cu): workspace size and the whole solve;
// *status: 0 converged, 2 not converged within max_iter.
size_t dif_scratch_bytes(size_t N);
cudaError_t launch_heat_diffusion(const GridDev& g, double h, const double* c, double* e, double k_l, double k_g,
                                  double dt, double tol, int max_iter, int phase_cp, const double* wall_T,
                                  void* workspace, cudaStream_t st, int* iters_out, double* change_out,
                                  int* status);

}  // namespace vofgb
