// vof_diffuse.cu -- implicit heat diffusion with the interface as a
// Dirichlet boundary (Malan et al., arXiv:2001.03477, Sec. 3.4.2: Eqs.
// T_diff_disc and mod_branchesT, after Sato and Niceno).
//
// A node is liquid when c >= 1/2, else gas; each phase diffuses with its own
// conductivity and T_Gamma = T_sat on the interface.  Along each axis the
// gradient towards a same-phase neighbour is the plain difference over h;
// towards the other phase it is (T_Gamma - T) / theta, theta the distance
// from the node to the interface along that axis, and the axis' second
// difference is divided by (d_- + d_+) / 2 (d = h or theta).  theta is the
// height function of the 7 cells centred on the node along the axis when
// the column ends in pure cells of the node's phase behind and the other
// phase beyond (the interface H - 3.5 cells ahead of a liquid node, 3.5 - H
// of a gas node), else the distance along the axis to the PLIC plane of the
// pair's mixed cell (the node's own if mixed, else the neighbour's), half a
// cell when both are pure or the plane is parallel to the axis; capped to
// [1e-3 h, h].  Zero-gradient walls carry no flux unless the caller fixes
// their temperature T_w: the node then sees the wall half a cell away,
// gradient (T_w - T) / (h / 2), d = h / 2 (the heated wall of Sec. 4.3).
// Periodic axes wrap.  Backward Euler with the heat capacity of the
// reading chosen:
//   phase (the default): every node diffuses with the constant C_p of its
//     phase, C_p,node (T' - T) / dt = k_p sum L(T'), and the cell's energy
//     changes by the heat conducted into it, e' = e + C_p,node (T' - T)
//     (Sec. 3.4.2 solves phase by phase with constant properties);
//   mixture: C_p(c) (T' - T) / dt = k_p sum L(T'), e' = C_p(c) T'.
// T = e / C_p(c) in both.
//
// Kernels: k_dif_planes (MYC normal and plane constant of the mixed cells),
// k_dif_assemble (per cell: the six couplings, the diagonal and the right
// side), k_dif_jacobi (one Jacobi sweep; the system is strictly diagonally
// dominant -- C_p / dt sits on the diagonal alone -- so the iteration
// converges; the largest change per sweep is reduced per CTA and read on the
// host every few sweeps), k_dif_store (e' = C_p T').
#include <algorithm>
#include <vector>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {

namespace {

constexpr int kDifThreads = 256;
constexpr int kDifCTAs = 152 * 8;
constexpr double kThetaEps = 1e-3;

__device__ __forceinline__ size_t dcid(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

// coordinate p + k along an axis of n cells: wrapped (periodic) or -1 off a
// zero-gradient wall
__device__ __forceinline__ int step_coord(int p, int k, int n, int bc) {
  int q = p + k;
  if (q < 0 || q >= n) {
    if (bc != 0) return -1;
    q %= n;
    if (q < 0) q += n;
  }
  return q;
}

// the same, clamped to the boundary cell on a zero-gradient axis (the
// height function's column extends by its boundary values)
__device__ __forceinline__ int clamp_coord(int p, int k, int n, int bc) {
  int q = p + k;
  if (bc != 0) return q < 0 ? 0 : (q >= n ? n - 1 : q);
  q %= n;
  return q < 0 ? q + n : q;
}

__global__ void k_dif_planes(GridDev g, const double* __restrict__ c, double4* __restrict__ plane, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const double cv = __ldg(c + i);
    if (!is_mixed_b(cv, g)) continue;
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    double s[27];
    for (int oz = 0; oz < 3; ++oz)
      for (int oy = 0; oy < 3; ++oy)
        for (int ox = 0; ox < 3; ++ox)
          s[(oz * 3 + oy) * 3 + ox] = __ldg(c + dcid(g, map_idx(x + ox - 1, g.n[0], g.bc[0]),
                                                      map_idx(y + oy - 1, g.n[1], g.bc[1]),
                                                      map_idx(z + oz - 1, g.n[2], g.bc[2])));
    double m[3];
    myc_normal(s, m);
    double4 p;
    p.x = m[0]; p.y = m[1]; p.z = m[2];
    p.w = plane_alpha(m[0], m[1], m[2], cv);
    plane[i] = p;
  }
}

// theta (cell units) from node (x, y, z) towards its neighbour in direction
// s along axis, the two being of different phases
__device__ double interface_theta(const GridDev& g, const double* __restrict__ c, const double4* __restrict__ plane,
                                  int x, int y, int z, int axis, int s, bool liquid_p) {
  const int pc[3] = {x, y, z};
  const int n = g.n[axis], bc = g.bc[axis];
  double col[7];
  for (int k = -3; k <= 3; ++k) {
    int q[3] = {x, y, z};
    q[axis] = clamp_coord(pc[axis], s * k, n, bc);
    col[k + 3] = __ldg(c + dcid(g, q[0], q[1], q[2]));
  }
  const double back = col[0], front = col[6];
  const double one_m_eps = 1.0 - g.eps;
  const bool ok = liquid_p ? (back >= one_m_eps && front <= g.eps) : (back <= g.eps && front >= one_m_eps);
  double theta;
  if (ok) {
    double H = 0.0;
    for (int k = 0; k < 7; ++k) H += col[k];
    theta = liquid_p ? H - 3.5 : 3.5 - H;
  } else {
    theta = 0.5;
    const size_t pid = dcid(g, x, y, z);
    int q[3] = {x, y, z};
    q[axis] = step_coord(pc[axis], s, n, bc);
    int mcell = -1;  // 0: the node's own cell, 1: the neighbour
    if (is_mixed_b(__ldg(c + pid), g)) mcell = 0;
    else if (q[axis] >= 0 && is_mixed_b(__ldg(c + dcid(g, q[0], q[1], q[2])), g)) mcell = 1;
    if (mcell >= 0) {
      const double4 p = plane[mcell == 0 ? pid : dcid(g, q[0], q[1], q[2])];
      // the node in the mixed cell's local coordinates
      double x0[3] = {0.5, 0.5, 0.5};
      if (mcell == 1) x0[axis] = 0.5 - (double)s;
      const double mm[3] = {p.x, p.y, p.z};
      const double ma = mm[axis] * (double)s;
      if (ma != 0.0) {
        const double t = (p.w - ((mm[0] * x0[0] + mm[1] * x0[1]) + mm[2] * x0[2])) / ma;
        theta = fabs(t);
      }
    }
  }
  return fmin(fmax(theta, kThetaEps), 1.0);
}

// walls at fixed temperature, per face x-, x+, y-, y+, z-, z+
struct DifWalls {
  double T[6];
  int on[6];
};

struct DifVec {
  double* off;    // [6 N]: coupling to the neighbour (face order -x, +x, -y, +y, -z, +z)
  double* diag;   // [N] reciprocal of the diagonal
  double* rhs;    // [N]
  double* Ta;     // [N] the two Jacobi iterates
  double* Tb;
  double* part;   // [kDifCTAs] per-CTA largest change
};

__global__ void __launch_bounds__(kDifThreads)
k_dif_assemble(GridDev g, double h, double inv_h, double inv_dt, double k_l, double k_g,
               const double* __restrict__ c, const double* __restrict__ e, const double4* __restrict__ plane,
               DifVec v, size_t N, DifWalls walls, int phase_cp) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    const double cv = __ldg(c + i);
    const bool liq = cv >= 0.5;
    const double kp = liq ? k_l : k_g;
    const double Cp = g.Cp_l * cv + g.Cp_g * (1.0 - cv);
    const double T0 = temp_of(g, __ldg(e + i), cv);
    const double Cd = phase_cp ? (liq ? g.Cp_l : g.Cp_g) : Cp;
    // a same-phase neighbour couples by k_p / h^2 (no division); only the
    // interface and heated-wall sides need their own distances
    const double kq = kp * (inv_h * inv_h);
    double diag = Cd * inv_dt, rhs = Cd * inv_dt * T0;
    const int pc[3] = {x, y, z};
    for (int axis = 0; axis < 3; ++axis) {
      double cs[2], cq[2], cst[2], d[2];
      bool reg[2];  // the side's distance is h (same phase or a wall without flux)
      for (int side = 0; side < 2; ++side) {
        reg[side] = true;
        const int s = side ? 1 : -1;
        int q[3] = {x, y, z};
        q[axis] = step_coord(pc[axis], s, g.n[axis], g.bc[axis]);
        if (q[axis] < 0 && walls.on[2 * axis + side]) {  // a wall at fixed T, half a cell away
          const double Tw = walls.T[2 * axis + side];
          cs[side] = 2.0 * inv_h; cq[side] = 0.0; cst[side] = Tw * 2.0 * inv_h; d[side] = 0.5 * h;
          reg[side] = false;
        } else if (q[axis] < 0) {  // a wall: no flux
          cs[side] = 0.0; cq[side] = 0.0; cst[side] = 0.0; d[side] = h;
        } else if ((__ldg(c + dcid(g, q[0], q[1], q[2])) >= 0.5) == liq) {
          cs[side] = inv_h; cq[side] = inv_h; cst[side] = 0.0; d[side] = h;
        } else {
          const double th = interface_theta(g, c, plane, x, y, z, axis, s, liq) * h;
          cs[side] = 1.0 / th; cq[side] = 0.0; cst[side] = g.T_sat / th; d[side] = th;
          reg[side] = false;
        }
      }
      if (reg[0] && reg[1]) {
        // both sides h: k_p / h^2 each (walls without flux contribute 0)
        for (int side = 0; side < 2; ++side) {
          const double o = dnz(cq[side]) ? kq : 0.0;
          diag += o;
          v.off[6 * i + 2 * axis + side] = o;
        }
      } else {
        const double kd = kp / (0.5 * (d[0] + d[1]));
        for (int side = 0; side < 2; ++side) {
          diag += kd * cs[side];
          v.off[6 * i + 2 * axis + side] = kd * cq[side];
          rhs += kd * cst[side];
        }
      }
    }
    v.diag[i] = 1.0 / diag;  // stored as its reciprocal: the sweeps multiply
    v.rhs[i] = rhs;
    v.Ta[i] = T0;
  }
}

// one Jacobi sweep Tout = (rhs + sum off T_nb(in)) / diag; per-CTA largest
// |Tout - Tin|
__global__ void __launch_bounds__(kDifThreads)
k_dif_jacobi(GridDev g, DifVec v, const double* __restrict__ Tin, double* __restrict__ Tout, size_t N) {
  __shared__ double red[kDifThreads];
  double dmax = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    const int pc[3] = {x, y, z};
    double acc = v.rhs[i];
    for (int f = 0; f < 6; ++f) {
      const int axis = f >> 1, s = (f & 1) ? 1 : -1;
      int q[3] = {x, y, z};
      q[axis] = step_coord(pc[axis], s, g.n[axis], g.bc[axis]);
      if (q[axis] < 0) continue;  // a wall: its coupling is 0
      acc = fma(v.off[6 * i + f], Tin[dcid(g, q[0], q[1], q[2])], acc);
    }
    const double t = acc * v.diag[i];
    Tout[i] = t;
    dmax = fmax(dmax, fabs(t - Tin[i]));
  }
  red[threadIdx.x] = dmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) v.part[blockIdx.x] = red[0];
}

__global__ void k_dif_store(GridDev g, const double* __restrict__ c, const double* __restrict__ T,
                            double* __restrict__ e, size_t N, int phase_cp) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const double cv = __ldg(c + i);
    const double Cp = g.Cp_l * cv + g.Cp_g * (1.0 - cv);
    if (phase_cp) {
      // e' = e + C_p,node (T' - T), T = e / C_p(c)
      const double ev = e[i];
      const double Cd = cv >= 0.5 ? g.Cp_l : g.Cp_g;
      e[i] = ev + Cd * (T[i] - temp_of(g, ev, cv));  // the T the assembly started from
    } else {
      e[i] = Cp * T[i];
    }
  }
}

struct DifLayout {
  size_t plane, off, diag, rhs, Ta, Tb, part, total;
};

DifLayout dif_layout(size_t N) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  DifLayout L;
  size_t o = 0;
  L.plane = o; o += a(N * 32);
  L.off = o; o += a(N * 6 * 8);
  L.diag = o; o += a(N * 8);
  L.rhs = o; o += a(N * 8);
  L.Ta = o; o += a(N * 8);
  L.Tb = o; o += a(N * 8);
  L.part = o; o += a(kDifCTAs * 8);
  L.total = o;
  return L;
}

}  // namespace

size_t dif_scratch_bytes(size_t N) { return dif_layout(N).total; }

cudaError_t launch_heat_diffusion(const GridDev& g, double h, const double* c, double* e, double k_l, double k_g,
                                  double dt, double tol, int max_iter, int phase_cp, const double* wall_T,
                                  void* workspace, cudaStream_t st, int* iters_out, double* change_out,
                                  int* status) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const DifLayout L = dif_layout(N);
  char* ws = static_cast<char*>(workspace);
  double4* plane = reinterpret_cast<double4*>(ws + L.plane);
  DifVec v;
  v.off = reinterpret_cast<double*>(ws + L.off);
  v.diag = reinterpret_cast<double*>(ws + L.diag);
  v.rhs = reinterpret_cast<double*>(ws + L.rhs);
  v.Ta = reinterpret_cast<double*>(ws + L.Ta);
  v.Tb = reinterpret_cast<double*>(ws + L.Tb);
  v.part = reinterpret_cast<double*>(ws + L.part);
  *status = 0;
  const int grid = (int)std::min<size_t>((N + kDifThreads - 1) / kDifThreads, (size_t)kDifCTAs);
  k_dif_planes<<<grid, kDifThreads, 0, st>>>(g, c, plane, N);
  DifWalls walls;
  for (int f = 0; f < 6; ++f) {
    walls.on[f] = wall_T && wall_T[f] == wall_T[f] ? 1 : 0;  // NaN: no wall temperature
    walls.T[f] = walls.on[f] ? wall_T[f] : 0.0;
  }
  k_dif_assemble<<<grid, kDifThreads, 0, st>>>(g, h, 1.0 / h, 1.0 / dt, k_l, k_g, c, e, plane, v, N, walls,
                                                phase_cp);
  prof_mark("diffuse.assemble", st);
  std::vector<double> part(grid);
  double* Tin = v.Ta;
  double* Tout = v.Tb;
  int it = 0;
  double change = 0.0;
  bool done = false;
  cudaError_t err = cudaSuccess;
  while (!done && it < max_iter) {
    k_dif_jacobi<<<grid, kDifThreads, 0, st>>>(g, v, Tin, Tout, N);
    std::swap(Tin, Tout);
    ++it;
    if (it % 4 == 0 || it == max_iter) {
      err = cudaMemcpyAsync(part.data(), v.part, grid * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) return err;
      change = 0.0;
      for (int b = 0; b < grid; ++b) change = std::max(change, part[b]);
      done = change <= tol;
    }
  }
  prof_mark("diffuse.jacobi", st);
  if (!done) *status = 2;
  k_dif_store<<<grid, kDifThreads, 0, st>>>(g, c, Tin, e, N, phase_cp);
  prof_mark("diffuse.store", st);
  if (iters_out) *iters_out = it;
  if (change_out) *change_out = change;
  return cudaGetLastError();
}

}  // namespace vofgb
