// vof_api.cu -- C ABI of the library (declared in include/vofgb.h): argument
// checks, parameter marshalling and the stream-ordered time step.
#include <cstring>
#include <mutex>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {

__device__ int g_vof_status;

static thread_local int t_last_cuda = 0;

void set_last_cuda_error(int err) { t_last_cuda = err; }

int* device_status_ptr() {
  static std::mutex mu;
  static int* ptrs[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_vof_status) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

static bool grid_ok(const vof_grid* g) {
  if (!g) return false;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  // cell lists hold 32-bit entries (cell index << 1 | face side)
  if ((long long)g->nx * g->ny * g->nz >= (1LL << 31)) return false;
  for (int d = 0; d < 3; ++d)
    if (g->bc[d] != 0 && g->bc[d] != 1) return false;
  if (!(g->h > 0.0) || !(g->Cp_l > 0.0) || !(g->Cp_g > 0.0)) return false;
  if (!(g->eps_mixed >= 0.0 && g->eps_mixed < 0.5)) return false;
  if (g->precision != VOF_F64 && g->precision != VOF_F32_FLUX) return false;
  if (g->scheme != VOF_SCHEME_WY && g->scheme != VOF_SCHEME_LE) return false;
  if (g->normal != VOF_NORMAL_MYC && g->normal != VOF_NORMAL_MLP && g->normal != VOF_NORMAL_YOUNGS) return false;
  if (g->normal == VOF_NORMAL_MLP && (!g->mlp || ((uintptr_t)g->mlp & 15) != 0)) return false;
  return true;
}

static GridDev to_dev(const vof_grid* g, double dt) {
  GridDev d;
  d.n[0] = g->nx; d.n[1] = g->ny; d.n[2] = g->nz;
  d.bc[0] = g->bc[0]; d.bc[1] = g->bc[1]; d.bc[2] = g->bc[2];
  d.lam = dt / g->h;
  d.Cp_l = g->Cp_l; d.Cp_g = g->Cp_g; d.T_sat = g->T_sat; d.eps = g->eps_mixed;
  d.rCp_l = 1.0 / g->Cp_l;
  d.rCp_g = 1.0 / g->Cp_g;
  double ome = 1.0 - g->eps_mixed;
  std::memcpy(&d.eps_bits, &g->eps_mixed, 8);
  std::memcpy(&d.one_m_eps, &ome, 8);
  d.f32 = g->precision == VOF_F32_FLUX ? 1 : 0;
  d.le = g->scheme == VOF_SCHEME_LE ? 1 : 0;
  d.mlp = g->normal == VOF_NORMAL_MLP ? 1 : (g->normal == VOF_NORMAL_YOUNGS ? 2 : 0);
  d.mlp_params = d.mlp == 1 ? g->mlp : nullptr;
  return d;
}

static size_t cells(const vof_grid* g) { return (size_t)g->nx * g->ny * g->nz; }

static size_t face_count(const vof_grid* g, int axis) {
  size_t nx = g->nx, ny = g->ny, nz = g->nz;
  if (axis == 0) return nz * ny * (nx + 1);
  if (axis == 1) return nz * (ny + 1) * nx;
  return (nz + 1) * ny * nx;
}

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b) return false;
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

static vof_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return VOF_OK;
  t_last_cuda = (int)e;
  return VOF_ECUDA;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace vofgb

using namespace vofgb;

extern "C" {

vof_status vof_reconstruct(const vof_grid* g, const double* c, double* m, double* alpha, uint8_t* mixed,
                           void* stream) {
  if (!grid_ok(g) || !c || !m || !alpha || !mixed) return VOF_EINVAL;
  size_t N = cells(g);
  if (overlap(c, N * 8, m, 3 * N * 8) || overlap(c, N * 8, alpha, N * 8) || overlap(c, N * 8, mixed, N))
    return VOF_EINVAL;
  return cuda_status(launch_reconstruct(to_dev(g, 0.0), c, m, alpha, mixed, (cudaStream_t)stream));
}

size_t vof_sweep_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return sweep_scratch_bytes(to_dev(g, 0.0));
}

static vof_status sweep_common(int axis, const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                               double* e_out, const double* uf, double dt, uint8_t* state, double* theta,
                               double* flux_out, double* diag, void* workspace, size_t workspace_bytes,
                               void* stream) {
  if (!grid_ok(g) || !c_in || !c_out || !uf || !workspace) return VOF_EINVAL;
  if (e_in && (!e_out || (state && !theta))) return VOF_EINVAL;
  if (!(dt >= 0.0)) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  const GridDev d = to_dev(g, dt);
  const size_t need = sweep_scratch_bytes(d);
  if (workspace_bytes < need) return VOF_EINVAL;
  size_t N = cells(g), B = N * 8;
  // either fully in place (c_out == c_in and e_out == e_in) or no overlap
  const bool inplace = c_out == c_in && (!e_in || e_out == e_in);
  if (!inplace) {
    if (overlap(c_in, B, c_out, B)) return VOF_EINVAL;
    if (e_in && (overlap(e_in, B, e_out, B) || overlap(c_in, B, e_out, B) || overlap(e_in, B, c_out, B)))
      return VOF_EINVAL;
  }
  if (e_in && (overlap(c_out, B, e_out, B) || overlap(c_in, B, e_in, B))) return VOF_EINVAL;
  if (flux_out && (overlap(flux_out, face_count(g, axis) * 8, c_out, B) ||
                   (e_out && overlap(flux_out, face_count(g, axis) * 8, e_out, B))))
    return VOF_EINVAL;
  if (overlap(workspace, need, c_in, B) || overlap(workspace, need, c_out, B) ||
      (e_in && (overlap(workspace, need, e_in, B) || overlap(workspace, need, e_out, B))))
    return VOF_EINVAL;
  // stand-alone sweep: diag[0] += clipped volume
  static const signed char kMap[kNSums] = {-1, -1, 0, -1, -1, -1};
  SweepScratch sc = carve_sweep_scratch(axis, d, workspace, sums_to_diag(diag, kMap));
  return cuda_status(launch_sweep(axis, d, c_in, e_in, c_out, e_in ? e_out : nullptr, uf, state, theta, flux_out, sc, true,
                                  (cudaStream_t)stream));
}

vof_status vof_advect_sweep_x(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                              double* e_out, const double* u_face, double dt, uint8_t* state, double* theta,
                              double* flux_out, double* diag, void* workspace, size_t workspace_bytes,
                              void* stream) {
  return sweep_common(0, g, c_in, e_in, c_out, e_out, u_face, dt, state, theta, flux_out, diag, workspace,
                      workspace_bytes, stream);
}
vof_status vof_advect_sweep_y(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                              double* e_out, const double* v_face, double dt, uint8_t* state, double* theta,
                              double* flux_out, double* diag, void* workspace, size_t workspace_bytes,
                              void* stream) {
  return sweep_common(1, g, c_in, e_in, c_out, e_out, v_face, dt, state, theta, flux_out, diag, workspace,
                      workspace_bytes, stream);
}
vof_status vof_advect_sweep_z(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                              double* e_out, const double* w_face, double dt, uint8_t* state, double* theta,
                              double* flux_out, double* diag, void* workspace, size_t workspace_bytes,
                              void* stream) {
  return sweep_common(2, g, c_in, e_in, c_out, e_out, w_face, dt, state, theta, flux_out, diag, workspace,
                      workspace_bytes, stream);
}

vof_status energy_advect_consistent(const vof_grid* g, int axis, const double* c_before, const double* c_after,
                                    const double* e_in, double* e_out, const double* flux_F, const double* u_face,
                                    double dt, uint8_t* state, double* theta, void* stream) {
  if (!grid_ok(g) || axis < 0 || axis > 2 || !c_before || !c_after || !e_in || !e_out || !flux_F || !u_face)
    return VOF_EINVAL;
  if (state && !theta) return VOF_EINVAL;
  if (!(dt >= 0.0)) return VOF_EINVAL;
  size_t B = cells(g) * 8;
  if (overlap(e_in, B, e_out, B) || overlap(c_before, B, e_out, B) || overlap(c_after, B, e_out, B)) return VOF_EINVAL;
  return cuda_status(launch_energy(axis, to_dev(g, dt), c_before, c_after, e_in, e_out, flux_F, u_face, state, theta,
                                   (cudaStream_t)stream));
}

size_t vof_shift_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return shift_scratch_bytes(to_dev(g, 0.0));
}

vof_status vof_phase_change_shift(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                                  double* e_out, const double* dd, double dd_uniform, uint8_t* state, double* diag,
                                  void* workspace, size_t workspace_bytes, void* stream) {
  if (!grid_ok(g) || !c_in || !e_in || !c_out || !e_out || !workspace) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  const GridDev d = to_dev(g, 0.0);
  const size_t need = shift_scratch_bytes(d);
  if (workspace_bytes < need) return VOF_EINVAL;
  size_t B = cells(g) * 8;
  // either fully in place (c_out == c_in and e_out == e_in) or no overlap
  const bool inplace = c_out == c_in && e_out == e_in;
  if (!inplace && (overlap(c_in, B, c_out, B) || overlap(e_in, B, e_out, B) || overlap(c_in, B, e_out, B) ||
                   overlap(e_in, B, c_out, B)))
    return VOF_EINVAL;
  if (overlap(c_out, B, e_out, B) || overlap(c_in, B, e_in, B)) return VOF_EINVAL;
  if (overlap(workspace, need, c_in, B) || overlap(workspace, need, c_out, B) || overlap(workspace, need, e_in, B) ||
      overlap(workspace, need, e_out, B) || (dd && overlap(workspace, need, dd, B)) ||
      (state && overlap(workspace, need, state, cells(g))) || (diag && overlap(workspace, need, diag, 5 * 8)))
    return VOF_EINVAL;
  // diag = {sum dc, clamped, sum de, sum c_out, sum e_out}
  static const signed char kMap[kNSums] = {3, 4, -1, 0, 1, 2};
  const SumOut so = sums_to_diag(diag, kMap);
  return cuda_status(launch_shift(d, c_in, e_in, c_out, e_out, dd, dd_uniform, state, carve_shift_scratch(d, workspace),
                                  so, so, true, (cudaStream_t)stream));
}

// workspace layout: theta | state | sum rows (tile pass, the three sweeps'
// update kernels, the shift's sums kernel; kNSums doubles per CTA) |
// reduction scratch | work counts (12 ints) and, 128 bytes in, the passes'
// list counters (kStepCounters ints, cleared by the tile pass) | tiles |
// scratch (reused by the three sweeps, then the shift).  The sweeps and the
// shift all run in place on c and e; the tile pass sums c and e at the start
// and every later kernel adds the changes it makes, so one fixed-order
// reduction of all rows gives the sums at the end of the step.
struct StepLayout {
  size_t off_th, off_st, off_rows, off_red, off_stats, off_tiles, off_sw, total;
  int nb_tiles, nb_sw[3], nb_sh, nrows;
};

static StepLayout step_layout(const vof_grid* g) {
  StepLayout L;
  GridDev d = to_dev(g, 0.0);
  size_t N = cells(g);
  L.off_th = 0;
  L.off_st = L.off_th + align256(N * 8);
  L.off_rows = L.off_st + align256(N);
  L.nb_tiles = tile_blocks(d);
  L.nrows = L.nb_tiles;
  for (int a = 0; a < 3; ++a) {
    L.nb_sw[a] = sweep_blocks(a, d);
    L.nrows += L.nb_sw[a];
  }
  L.nb_sh = shift_sum_blocks(d);
  L.nrows += L.nb_sh;
  L.off_red = L.off_rows + align256((size_t)L.nrows * kNSums * 8);
  L.off_stats = L.off_red + align256(reduce_scratch_bytes());
  L.off_tiles = L.off_stats + 256;
  L.off_sw = L.off_tiles + align256(tile_scratch_bytes(d));
  const size_t sw = sweep_scratch_bytes(d), sh = shift_scratch_bytes(d);
  L.total = L.off_sw + align256(sw > sh ? sw : sh);
  return L;
}

// the passes' list counters: 128 bytes into the work-count block
static int* step_counters(char* ws, const StepLayout& L) {
  return reinterpret_cast<int*>(ws + L.off_stats + 128);
}

size_t vof_step_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return step_layout(g).total;
}

}  // extern "C"

namespace vofgb {

// One box's arguments for the grouped step: the same carving, sum rows and
// launch shapes as vof_step below (keep the two in step).
bool step_box(const vof_grid* g, double* c, double* e, const double* u, const double* v, const double* w,
              double dt, const double* dd, double dd_uniform, double* sums, char* ws, StepBox* out) {
  if (!grid_ok(g) || !c || !e || !u || !v || !w || !(dt >= 0.0) || !ws) return false;
  if (g->normal == VOF_NORMAL_MLP) return false;  // the learned normal runs per grid (vof_step)
  const StepLayout L = step_layout(g);
  const GridDev d = to_dev(g, dt);
  const size_t N = cells(g);
  StepBox& B = *out;
  B.cells = N;
  double* th = reinterpret_cast<double*>(ws + L.off_th);
  uint8_t* state = reinterpret_cast<uint8_t*>(ws + L.off_st);
  double* rows = reinterpret_cast<double*>(ws + L.off_rows);
  int* cnt = step_counters(ws, L);
  // tile pass
  const TileScratch ts = carve_tile_scratch(d, ws + L.off_tiles);
  int nt[3];
  tile_counts(d, nt);
  B.tiles.g = d;
  B.tiles.c = c;
  B.tiles.e = e;
  B.tiles.ts = ts;
  B.tiles.nt[0] = nt[0]; B.tiles.nt[1] = nt[1]; B.tiles.nt[2] = nt[2];
  B.tiles.sums = sums_to_partials(rows, kNSums);
  B.tiles.state = state;
  B.tiles.counters = cnt;
  B.grid_tiles = dim3((unsigned)((nt[0] + 3) / 4), (unsigned)nt[1], (unsigned)nt[2]);
  B.grid_quiet = quiet_blocks(d);
  size_t r = (size_t)L.nb_tiles;
  TileMap tm{nullptr, {0, 0, 0}};
  if (tiles_usable(d)) {
    tm.quiet = ts.quiet;
    tile_counts(d, tm.nt);
  }
  const double* uf[3] = {u, v, w};
  // sum rows in the order of the axes of an even step (x, y, z): the rows of
  // a sweep belong to its axis, as in vof_step
  size_t row_of_axis[3];  // fixed per axis, as in vof_step
  {
    size_t rr = r;
    for (int a = 0; a < 3; ++a) {
      row_of_axis[a] = rr;
      rr += (size_t)L.nb_sw[a];
    }
  }
  for (int a = 0; a < 3; ++a) {
    SweepScratch sc = carve_sweep_scratch(a, d, ws + L.off_sw, sums_to_partials(rows + row_of_axis[a] * kNSums, kNSums));
    sc.tiles = tm;
    sc.stats = reinterpret_cast<int*>(ws + L.off_stats) + 2 * a;
    sc.mlp_stat = reinterpret_cast<int*>(ws + L.off_stats) + 9 + a;
    sc.counters = cnt + 4 * a;
    const SweepPlan p = sweep_plan(a, d);
    SweepArgs& A = B.sweep[a];
    A.g = d;
    A.c = c;
    A.e = e;
    A.uf = uf[a];
    A.state = state;
    A.theta = th;
    A.sc = sc;
    A.cap = p.cap;
    A.nsub = (int)p.nsub;
    A.ngrp = p.lpc / kUpdLists;
    A.status = device_status_ptr();
    B.grid_stream[a] = p.gridA;
    B.grid_update[a] = p.gridB;
    r += (size_t)L.nb_sw[a];
  }
  ShiftScratch shs = carve_shift_scratch(d, ws + L.off_sw);
  shs.tiles = tm;
  shs.stats = reinterpret_cast<int*>(ws + L.off_stats) + 6;
  shs.counters = cnt + 12;
  ShiftArgs& S = B.shift;
  S.g = d;
  S.c = c;
  S.e = e;
  S.dd = dd;
  S.dd_uniform = dd_uniform;
  S.sc = shs;
  S.sums = sums_to_partials(rows + r * kNSums, kNSums);
  S.nw = shift_warps_of(d);
  B.grid_shift_stream = shift_stream_grid_of(d);
  B.grid_shift_sums = (unsigned)shift_sum_blocks(d);
  r += (size_t)L.nb_sh;
  B.red = ReduceBox{rows, (int)r, sums, reinterpret_cast<double*>(ws + L.off_red)};
  return true;
}

}  // namespace vofgb

extern "C" {

vof_status vof_step(const vof_grid* g, double* c, double* e, const double* u, const double* v, const double* w,
                    double dt, long step_index, const double* dd, double dd_uniform, double* sums, void* workspace,
                    size_t workspace_bytes, void* stream) {
  if (!grid_ok(g) || !c || !e || !u || !v || !w || !workspace) return VOF_EINVAL;
  if (!(dt >= 0.0) || step_index < 0) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  StepLayout L = step_layout(g);
  if (workspace_bytes < L.total) return VOF_EINVAL;
  size_t N = cells(g), B = N * 8;
  if (overlap(c, B, e, B) || overlap(c, B, workspace, L.total) || overlap(e, B, workspace, L.total))
    return VOF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = static_cast<char*>(workspace);
  double* th = reinterpret_cast<double*>(ws + L.off_th);
  uint8_t* state = reinterpret_cast<uint8_t*>(ws + L.off_st);
  double* rows = reinterpret_cast<double*>(ws + L.off_rows);
  GridDev d = to_dev(g, dt);
  const double* uf[3] = {u, v, w};
  int* cnt = step_counters(ws, L);
  // tile pass: quiet tiles and the sums of c, e at the start of the step;
  // it also clears the frozen-state flags and the passes' list counters
  const TileScratch ts = carve_tile_scratch(d, ws + L.off_tiles);
  size_t r = 0;
  cudaError_t err = launch_tiles(d, c, e, ts, sums_to_partials(rows, kNSums), state, cnt, st);
  if (err != cudaSuccess) return cuda_status(err);
  r += (size_t)L.nb_tiles;
  TileMap tm{nullptr, {0, 0, 0}};
  if (tiles_usable(d)) {
    tm.quiet = ts.quiet;
    tile_counts(d, tm.nt);
  }
  // each axis' sum rows have a fixed place (x, y, z after the tile rows),
  // whatever the order the sweeps run in
  size_t row_of_axis[3];
  for (int a = 0; a < 3; ++a) {
    row_of_axis[a] = r;
    r += (size_t)L.nb_sw[a];
  }
  for (int s = 0; s < 3; ++s) {
    const int ax = (step_index % 2 == 0) ? s : 2 - s;
    SweepScratch sc =
        carve_sweep_scratch(ax, d, ws + L.off_sw, sums_to_partials(rows + row_of_axis[ax] * kNSums, kNSums));
    sc.tiles = tm;
    sc.stats = reinterpret_cast<int*>(ws + L.off_stats) + 2 * ax;
    sc.mlp_stat = reinterpret_cast<int*>(ws + L.off_stats) + 9 + ax;
    sc.counters = cnt + 4 * ax;
    err = launch_sweep(ax, d, c, e, c, e, uf[ax], state, th, nullptr, sc, false, st);
    if (err != cudaSuccess) return cuda_status(err);
  }
  ShiftScratch shs = carve_shift_scratch(d, ws + L.off_sw);
  shs.tiles = tm;
  shs.stats = reinterpret_cast<int*>(ws + L.off_stats) + 6;
  shs.counters = cnt + 12;
  const SumOut none = sums_to_partials(nullptr, kNSums);
  err = launch_shift(d, c, e, c, e, dd, dd_uniform, nullptr, shs, none, sums_to_partials(rows + r * kNSums, kNSums),
                     false, st);
  if (err != cudaSuccess) return cuda_status(err);
  r += (size_t)L.nb_sh;
  if (sums) {
    // sums[0..1] = sum c, sum e; sums[2] = clip; sums[3..5] = shift diagnostics
    err = launch_reduce_fused(ReduceJob{rows, (int)r, kNSums, 0, kNSums, sums},
                              reinterpret_cast<double*>(ws + L.off_red), cnt + (kStepCounters - 1), st);
    if (err != cudaSuccess) return cuda_status(err);
  }
  return VOF_OK;
}

vof_status vof_step_work_counts(const vof_grid* g, const void* workspace, int* counts, void* stream) {
  if (!grid_ok(g) || !workspace || !counts) return VOF_EINVAL;
  const StepLayout L = step_layout(g);
  const char* ws = static_cast<const char*>(workspace);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t err = cudaMemcpyAsync(counts, ws + L.off_stats, VOF_NCOUNTS * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  return cuda_status(err);
}

size_t vof_mass_transfer_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return mdot_scratch_bytes(cells(g));
}

vof_status vof_mass_transfer(const vof_grid* g, const double* c, const double* e, double k_l, double k_g,
                             double h_fg, double* mdot, double* d_gamma, double* grad_n, double dd_per_mdot,
                             double* dd, void* workspace, size_t workspace_bytes, void* stream) {
  if (!grid_ok(g) || !c || !e || !mdot || !workspace) return VOF_EINVAL;
  if (!(h_fg > 0.0) || !(k_l >= 0.0) || !(k_g >= 0.0) || !(dd_per_mdot == dd_per_mdot)) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  const size_t N = cells(g), B = N * 8;
  const size_t need = mdot_scratch_bytes(N);
  if (workspace_bytes < need) return VOF_EINVAL;
  const void* outs[4] = {mdot, d_gamma, grad_n, dd};
  for (int a = 0; a < 4; ++a) {
    if (!outs[a]) continue;
    if (overlap(outs[a], B, c, B) || overlap(outs[a], B, e, B) || overlap(outs[a], B, workspace, need))
      return VOF_EINVAL;
    for (int b = a + 1; b < 4; ++b)
      if (overlap(outs[a], B, outs[b], B)) return VOF_EINVAL;
  }
  if (overlap(workspace, need, c, B) || overlap(workspace, need, e, B)) return VOF_EINVAL;
  return cuda_status(launch_mass_transfer(to_dev(g, 0.0), g->h, c, e, k_l, k_g, h_fg, dd_per_mdot, mdot, d_gamma,
                                          grad_n, dd, workspace, (cudaStream_t)stream));
}

vof_status vof_mass_transfer_work_counts(const vof_grid* g, const void* workspace, int* counts, void* stream) {
  if (!grid_ok(g) || !workspace || !counts) return VOF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t err = cudaMemcpyAsync(counts, mdot_counters(to_dev(g, 0.0), const_cast<void*>(workspace)),
                                    2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  return cuda_status(err);
}

size_t vof_velocity_extension_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return ext_scratch_bytes(cells(g));
}

vof_status vof_velocity_extension(const vof_grid* g, const double* c, const double* mdot, double rho_l,
                                  double rho_g, double dt, double tol, int max_iter, double* u, double* v,
                                  double* w, double* ut, double* vt, double* wt, int* iterations,
                                  double* residual, void* workspace, size_t workspace_bytes, void* stream) {
  if (!grid_ok(g) || !c || !mdot || !workspace) return VOF_EINVAL;
  if (!(rho_l > 0.0) || !(rho_g > 0.0) || !(dt >= 0.0) || !(tol > 0.0) || max_iter < 1) return VOF_EINVAL;
  const bool add = u || v || w, put = ut || vt || wt;
  if ((add && !(u && v && w)) || (put && !(ut && vt && wt)) || (!add && !put)) return VOF_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  const size_t N = cells(g), B = N * 8;
  const size_t need = ext_scratch_bytes(N);
  if (workspace_bytes < need) return VOF_EINVAL;
  const void* outs[6] = {u, v, w, ut, vt, wt};
  for (int a = 0; a < 6; ++a) {
    if (!outs[a]) continue;
    const size_t fa = face_count(g, a % 3) * 8;
    if (overlap(outs[a], fa, c, B) || overlap(outs[a], fa, mdot, B) || overlap(outs[a], fa, workspace, need))
      return VOF_EINVAL;
    for (int b = a + 1; b < 6; ++b)
      if (outs[b] && overlap(outs[a], fa, outs[b], face_count(g, b % 3) * 8)) return VOF_EINVAL;
  }
  if (overlap(workspace, need, c, B) || overlap(workspace, need, mdot, B)) return VOF_EINVAL;
  int it = 0, st = 0;
  double res = 0.0;
  cudaError_t err = launch_velocity_extension(to_dev(g, 0.0), g->h, c, mdot, rho_l, rho_g, dt, tol, max_iter, u, v,
                                              w, ut, vt, wt, workspace, (cudaStream_t)stream, &it, &res, &st);
  if (err != cudaSuccess) return cuda_status(err);
  if (iterations) *iterations = it;
  if (residual) *residual = res;
  return st ? VOF_ESOLVE : VOF_OK;
}

size_t vof_heat_diffusion_workspace_bytes(const vof_grid* g) {
  if (!grid_ok(g)) return 0;
  return dif_scratch_bytes(cells(g));
}

vof_status vof_heat_diffusion(const vof_grid* g, const double* c, double* e, double k_l, double k_g, double dt,
                              double tol, int max_iter, int heat_capacity, const double* wall_T, int* iterations,
                              double* change, void* workspace, size_t workspace_bytes, void* stream) {
  if (!grid_ok(g) || !c || !e || !workspace) return VOF_EINVAL;
  if (!(k_l >= 0.0) || !(k_g >= 0.0) || !(dt > 0.0) || !(tol > 0.0) || max_iter < 1) return VOF_EINVAL;
  if (heat_capacity != VOF_CP_PHASE && heat_capacity != VOF_CP_MIXTURE) return VOF_EINVAL;
  if (wall_T) {
    for (int f = 0; f < 6; ++f) {
      const double Tw = wall_T[f];
      if (Tw != Tw) continue;                                   // NaN: no wall temperature on this face
      if (g->bc[f / 2] != 1 || !(Tw > -1e300 && Tw < 1e300)) return VOF_EINVAL;  // finite, zero-gradient axis
    }
  }
  if (((uintptr_t)workspace & 255) != 0) return VOF_EINVAL;
  const size_t N = cells(g), B = N * 8;
  const size_t need = dif_scratch_bytes(N);
  if (workspace_bytes < need) return VOF_EINVAL;
  if (overlap(c, B, e, B) || overlap(workspace, need, c, B) || overlap(workspace, need, e, B)) return VOF_EINVAL;
  int it = 0, st = 0;
  double ch = 0.0;
  cudaError_t err = launch_heat_diffusion(to_dev(g, 0.0), g->h, c, e, k_l, k_g, dt, tol, max_iter,
                                          heat_capacity == VOF_CP_PHASE ? 1 : 0, wall_T, workspace,
                                          (cudaStream_t)stream, &it, &ch, &st);
  if (err != cudaSuccess) return cuda_status(err);
  if (iterations) *iterations = it;
  if (change) *change = ch;
  return st ? VOF_ESOLVE : VOF_OK;
}

vof_status vof_get_device_status(void) {
  int* p = device_status_ptr();
  if (!p) return VOF_ECUDA;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, p, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  int z = 0;
  e = cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  if (h & DEV_WAIT) return VOF_EWAIT;
  return (h & DEV_CFL) ? VOF_ECFL : VOF_OK;
}

const char* vof_status_string(int status) {
  switch (status) {
    case VOF_OK: return "ok";
    case VOF_EINVAL: return "invalid argument";
    case VOF_ECUDA: return "CUDA error";
    case VOF_ECFL: return "face CFL number above 1";
    case VOF_ESOLVE: return "iterative solve not converged (or no free-flow face for the velocity extension)";
    case VOF_EWAIT: return "a bounded device wait gave up (tensor-core completion not seen in time)";
    default: return "unknown status";
  }
}

int vof_last_cuda_error(void) { return t_last_cuda; }

}  // extern "C"
