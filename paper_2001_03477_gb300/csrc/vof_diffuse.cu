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
// Kernels: k_dif_mlist (list of the mixed cells), k_dif_planes (MYC normal
// and plane constant of each listed cell), k_dif_classify (per cell: its
// class; every cell whose sides all couple by k_p / h^2 takes its diagonal
// from a per-phase table), k_dif_irregular (the listed cells next to the
// interface or a heated wall: the six couplings and the diagonal), k_dif_jacobi (one Jacobi sweep; the
// system is strictly diagonally dominant -- C_p / dt sits on the diagonal
// alone -- so the iteration converges; on every fourth sweep the largest
// change is reduced per CTA and read on the host), k_dif_store (e' from T').
#include <algorithm>
#include <cstring>
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

// the mixed cells of the grid, appended to a list (one atomic per warp);
// the list's order varies from run to run, and nothing depends on it
__global__ void __launch_bounds__(kDifThreads)
k_dif_mlist(GridDev g, const double* __restrict__ c, uint32_t* __restrict__ mlist, int* __restrict__ count,
            size_t N) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t n_iter = (N + stride - 1) / stride;  // whole warps iterate together
  const int lane = threadIdx.x & 31;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t it = 0; it < n_iter; ++it, i += stride) {
    const bool mx = i < N && is_mixed_b(__ldg(c + i), g);
    const unsigned mask = __ballot_sync(0xffffffffu, mx);
    if (!mask) continue;
    int base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (mx) mlist[base + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// MYC normal and plane constant of each listed mixed cell (lanes dense over
// the list: the FP64 work of a warp serves 32 cells)
__global__ void __launch_bounds__(kDifThreads)
k_dif_planes(GridDev g, const double* __restrict__ c, const uint32_t* __restrict__ mlist,
             const int* __restrict__ count, double4* __restrict__ plane) {
  const int nm = *count;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nm; k += gridDim.x * blockDim.x) {
    const size_t i = mlist[k];
    const double cv = __ldg(c + i);
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    double s[27];
#pragma unroll
    for (int oz = 0; oz < 3; ++oz)
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
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

// Per-phase constants of the assembled system (index 0 gas, 1 liquid),
// computed on the host in the order the per-cell assembly would use:
// k_p / h^2, C_p / dt (phase heat capacity), and the reciprocal of the
// diagonal C_p / dt + n k_p / h^2 of a cell with n same-phase sides.
struct DifConst {
  double kq[2];
  double cdt[2];
  double rdiag[2][7];
};

// Cell classes: bits 0..5 the sides (-x, +x, -y, +y, -z, +z) with a
// neighbour in the grid; kDifLiq the node is liquid (c >= 1/2); kDifIrr
// the cell has an interface or heated-wall side, so its couplings and
// diagonal are stored.  Every other cell couples by k_p / h^2 to each
// neighbour and, with the phase heat capacity, takes its diagonal from the
// table: the sweeps then read no coupling for it.
constexpr uint8_t kDifLiq = 0x40, kDifIrr = 0x80;

struct DifVec {
  double* off;    // [6 N]: coupling to the neighbour (face order -x, +x, -y, +y, -z, +z); kDifIrr cells only
  double* diag;   // [N] reciprocal of the diagonal; kDifIrr cells (all cells with the mixture heat capacity)
  double* rhs;    // [N]; kDifIrr cells (all cells with the mixture heat capacity)
  double* T0;     // [N] T at the start (the first iterate)
  double* Ta;     // [N] the two later Jacobi iterates
  double* Tb;
  double* part;   // [1] the largest change of a checked sweep
  uint8_t* cls;   // [N] cell class
};

constexpr long long kHalfBits = 0x3FE0000000000000LL;  // 0.5: c >= 1/2 on the integer pipe (c >= +0)

// The six sides of node (x, y, z): in the grid (inm), with a node of the
// same phase (same), and whether a side is a wall at fixed temperature.
__device__ __forceinline__ void dif_sides(const GridDev& g, const double* __restrict__ c, const DifWalls& walls,
                                          int x, int y, int z, bool liq, unsigned& inm, unsigned& same,
                                          bool& hot_wall) {
  const int pc[3] = {x, y, z};
  inm = 0u;
  same = 0u;
  hot_wall = false;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int axis = f >> 1, s = (f & 1) ? 1 : -1;
    int q[3] = {x, y, z};
    q[axis] = step_coord(pc[axis], s, g.n[axis], g.bc[axis]);
    if (q[axis] < 0) {
      hot_wall = hot_wall || walls.on[f] != 0;
      continue;
    }
    inm |= 1u << f;
    if ((dbits(__ldg(c + dcid(g, q[0], q[1], q[2]))) >= kHalfBits) == liq) same |= 1u << f;
  }
}

// Per cell: its class and T; every cell that couples by k_p / h^2 on all
// sides also gets its right side (and, with the mixture heat capacity, its
// diagonal); the others -- next to the interface or a heated wall -- are
// listed for k_dif_irregular (one atomic per warp; the list's order varies
// from run to run, and nothing depends on it).
// the sweep's CTAs: 32 x 8 cells of every plane each, enough z shares for
// a few waves
static dim3 dif_sweep_grid(const GridDev& g) {
  const unsigned gx = (unsigned)((g.n[0] + 31) / 32), gy = (unsigned)((g.n[1] + 7) / 8);
  unsigned gz = (unsigned)std::max(1, std::min(g.n[2], (int)(152u * 16u / std::max(1u, gx * gy))));
  return dim3(gx, gy, gz);
}

template <bool PHASE>
__global__ void __launch_bounds__(kDifThreads)
k_dif_classify(GridDev g, const double* __restrict__ c, const double* __restrict__ e, DifVec v, DifWalls walls,
               double inv_dt, DifConst K, uint32_t* __restrict__ ilist, int* __restrict__ icount) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (y >= g.n[1]) return;  // whole warps (a warp is one row segment)
  const bool in_x = x < g.n[0];
  const int lane = threadIdx.x;
  for (int z = blockIdx.z; z < g.n[2]; z += gridDim.z) {
    const size_t i = ((size_t)z * g.n[1] + y) * g.n[0] + x;
    bool irr = false;
    if (in_x) {
      const double cv = __ldg(c + i);
      const bool liq = dbits(cv) >= kHalfBits;
      const double T0 = temp_of(g, __ldg(e + i), cv);
      unsigned inm, same;
      bool hot_wall;
      dif_sides(g, c, walls, x, y, z, liq, inm, same, hot_wall);
      const int li = liq ? 1 : 0;
      v.T0[i] = T0;
      irr = hot_wall || same != inm;
      v.cls[i] = (uint8_t)(inm | (liq ? kDifLiq : 0) | (irr ? kDifIrr : 0));
      if (!irr && !PHASE) {
        // every side in the grid couples by k_p / h^2 (walls without flux:
        // 0); with the phase heat capacity the sweeps form the right side
        // C_p / dt T0 and take the diagonal from the table themselves
        const double cdt = (g.Cp_l * cv + g.Cp_g * (1.0 - cv)) * inv_dt;
        v.rhs[i] = cdt * T0;
        const double kq = li ? K.kq[1] : K.kq[0];
        double diag = cdt;
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (inm & (1u << f)) diag += kq;
        v.diag[i] = 1.0 / diag;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, irr);
    if (!mask) continue;
    int base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(icount, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (irr) ilist[base + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// Per listed cell (lanes dense over the list): the six couplings (heights
// or plane distances on the interface sides), the diagonal and the right
// side.
__global__ void __launch_bounds__(kDifThreads)
k_dif_irregular(GridDev g, double h, double inv_h, double inv_dt, double k_l, double k_g,
                const double* __restrict__ c, const double* __restrict__ e, const double4* __restrict__ plane,
                DifVec v, DifWalls walls, int phase_cp, DifConst K, const uint32_t* __restrict__ ilist,
                const int* __restrict__ icount) {
  const int ni = *icount;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ni; k += gridDim.x * blockDim.x) {
    const size_t i = ilist[k];
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    const double cv = __ldg(c + i);
    const bool liq = dbits(cv) >= kHalfBits;
    const double T0 = temp_of(g, __ldg(e + i), cv);
    unsigned inm, same;
    bool hot_wall;
    dif_sides(g, c, walls, x, y, z, liq, inm, same, hot_wall);
    const int li = liq ? 1 : 0;
    const double cdt = phase_cp ? K.cdt[li] : (g.Cp_l * cv + g.Cp_g * (1.0 - cv)) * inv_dt;
    double diag = cdt, rhs = cdt * T0;
    const double kp = liq ? k_l : k_g;
    // a same-phase neighbour couples by k_p / h^2 (no division); only the
    // interface and heated-wall sides need their own distances
    const double kq = kp * (inv_h * inv_h);
#pragma unroll
    for (int axis = 0; axis < 3; ++axis) {
      double cs[2], cq[2], cst[2], d[2];
      bool reg[2];  // the side's distance is h (same phase or a wall without flux)
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * axis + side;
        reg[side] = true;
        if (!(inm & (1u << f)) && walls.on[f]) {  // a wall at fixed T, half a cell away
          const double Tw = walls.T[f];
          cs[side] = 2.0 * inv_h; cq[side] = 0.0; cst[side] = Tw * 2.0 * inv_h; d[side] = 0.5 * h;
          reg[side] = false;
        } else if (!(inm & (1u << f))) {  // a wall: no flux
          cs[side] = 0.0; cq[side] = 0.0; cst[side] = 0.0; d[side] = h;
        } else if (same & (1u << f)) {
          cs[side] = inv_h; cq[side] = inv_h; cst[side] = 0.0; d[side] = h;
        } else {
          const double th = interface_theta(g, c, plane, x, y, z, axis, side ? 1 : -1, liq) * h;
          cs[side] = 1.0 / th; cq[side] = 0.0; cst[side] = g.T_sat / th; d[side] = th;
          reg[side] = false;
        }
      }
      if (reg[0] && reg[1]) {
        // both sides h: k_p / h^2 each (walls without flux contribute 0)
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const double o = dnz(cq[side]) ? kq : 0.0;
          diag += o;
          v.off[6 * i + 2 * axis + side] = o;
        }
      } else {
        const double kd = kp / (0.5 * (d[0] + d[1]));
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          diag += kd * cs[side];
          v.off[6 * i + 2 * axis + side] = kd * cq[side];
          rhs += kd * cst[side];
        }
      }
    }
    v.diag[i] = 1.0 / diag;  // stored as its reciprocal: the sweeps multiply
    v.rhs[i] = rhs;
  }
}

// The Jacobi update of one cell from its neighbours' values t0..t5 (sides
// not in the grid skipped): (rhs + sum off T_nb) / diag, the right side
// C_p / dt T0 and the couplings k_p / h^2 unless the cell's are stored.  Not
// inlined, and called only by warps with a cell that needs it, so that the
// other warps issue none of its FP64 instructions.
static __device__ __noinline__ double dif_row(unsigned cls, const double* __restrict__ off6,
                                              const double* __restrict__ rhs_i, const double* __restrict__ diag_i,
                                              double kq, double cdt, double rdt, double T0, int phase_cp, double t0,
                                              double t1, double t2, double t3, double t4, double t5) {
  const bool irr = (cls & kDifIrr) != 0;
  const bool stored = irr || !phase_cp;
  double acc = stored ? __ldg(rhs_i) : cdt * T0;
  const double tn[6] = {t0, t1, t2, t3, t4, t5};
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if (cls & (1u << f)) acc = fma(irr ? __ldg(off6 + f) : kq, tn[f], acc);
  return acc * (stored ? __ldg(diag_i) : rdt);
}

// Neighbour index of cell i at (x, y, z) across side f (its class bit set):
// the next cell along the axis, or across a periodic boundary the first or
// last of the line.
__device__ __forceinline__ size_t dif_nb(const GridDev& g, size_t i, int x, int y, int z, int f) {
  const size_t sx = 1, sy = (size_t)g.n[0], sz = (size_t)g.n[0] * g.n[1];
  switch (f) {
    case 0: return x > 0 ? i - sx : i + (size_t)(g.n[0] - 1) * sx;
    case 1: return x < g.n[0] - 1 ? i + sx : i - (size_t)(g.n[0] - 1) * sx;
    case 2: return y > 0 ? i - sy : i + (size_t)(g.n[1] - 1) * sy;
    case 3: return y < g.n[1] - 1 ? i + sy : i - (size_t)(g.n[1] - 1) * sy;
    case 4: return z > 0 ? i - sz : i + (size_t)(g.n[2] - 1) * sz;
    default: return z < g.n[2] - 1 ? i + sz : i - (size_t)(g.n[2] - 1) * sz;
  }
}

// One Jacobi sweep Tout = (rhs + sum off T_nb(in)) / diag; with CHECK the
// largest |Tout - Tin| into *change (non-negative doubles order like their
// bits: an integer atomic max, the same whatever the order).  A cell
// coupled by k_p / h^2 whose own and neighbours' values all equal its T0 is
// the sweep's fixed point, (C_p/dt T0 + n k_p/h^2 T0) / (C_p/dt + n k_p/h^2)
// = T0, and keeps T0 without arithmetic.  CTAs of 32 x 8 threads over x and
// y, each walking its share of the z planes (no index division).
template <bool CHECK>
__global__ void __launch_bounds__(kDifThreads)
k_dif_jacobi(GridDev g, DifVec v, DifConst K, const double* __restrict__ Tin, double* __restrict__ Tout,
             unsigned long long* __restrict__ change, int phase_cp) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  double dmax = 0.0;
  if (x < g.n[0] && y < g.n[1]) {
    for (int z = blockIdx.z; z < g.n[2]; z += gridDim.z) {
      const size_t i = ((size_t)z * g.n[1] + y) * g.n[0] + x;
      const unsigned cls = __ldg(v.cls + i);
      const double T0 = __ldg(v.T0 + i), tin = Tin[i];
      const long long b0 = dbits(T0);
      double tn[6];
      bool fixed = (cls & kDifIrr) == 0 && dbits(tin) == b0;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        tn[f] = 0.0;
        if (!(cls & (1u << f))) continue;  // a wall: its coupling is 0
        tn[f] = Tin[dif_nb(g, i, x, y, z, f)];
        fixed = fixed && dbits(tn[f]) == b0;
      }
      double t = T0;
      if (__any_sync(__activemask(), !fixed)) {
        const int li = (cls & kDifLiq) ? 1 : 0;
        const double r = dif_row(cls, v.off + 6 * i, v.rhs + i, v.diag + i, li ? K.kq[1] : K.kq[0],
                                 li ? K.cdt[1] : K.cdt[0], K.rdiag[li][__popc(cls & 63u)], T0, phase_cp, tn[0],
                                 tn[1], tn[2], tn[3], tn[4], tn[5]);
        if (!fixed) t = r;
      }
      Tout[i] = t;
      if (CHECK) dmax = fmax(dmax, fabs(t - tin));
    }
  }
  if constexpr (CHECK) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dnz(dmax)) atomicMax(change, (unsigned long long)dbits(dmax));
  }
}


__global__ void k_dif_store(GridDev g, const double* __restrict__ c, const DifVec v, const double* __restrict__ T,
                            double* __restrict__ e, size_t N, int phase_cp) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const double Tn = T[i];
    if (phase_cp) {
      // e' = e + C_p,node (T' - T0); a node whose T came back unchanged
      // keeps its e
      const double T0 = __ldg(v.T0 + i);
      if (dbits(Tn) == dbits(T0)) continue;
      const double Cd = (__ldg(v.cls + i) & kDifLiq) ? g.Cp_l : g.Cp_g;
      e[i] = e[i] + Cd * (Tn - T0);
    } else {
      const double cv = __ldg(c + i);
      const double Cp = g.Cp_l * cv + g.Cp_g * (1.0 - cv);
      e[i] = Cp * Tn;
    }
  }
}

struct DifLayout {
  size_t plane, off, diag, rhs, T0, Ta, Tb, part, cls, mlist, count, total;
};

DifLayout dif_layout(size_t N) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  DifLayout L;
  size_t o = 0;
  L.plane = o; o += a(N * 32);
  L.off = o; o += a(N * 6 * 8);
  L.diag = o; o += a(N * 8);
  L.rhs = o; o += a(N * 8);
  L.T0 = o; o += a(N * 8);
  L.Ta = o; o += a(N * 8);
  L.Tb = o; o += a(N * 8);
  L.part = o; o += 256;  // the largest change (bits of a non-negative double)
  L.cls = o; o += a(N);
  L.mlist = o; o += a(N * 4);
  L.count = o; o += 256;
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
  v.T0 = reinterpret_cast<double*>(ws + L.T0);
  v.Ta = reinterpret_cast<double*>(ws + L.Ta);
  v.Tb = reinterpret_cast<double*>(ws + L.Tb);
  v.part = reinterpret_cast<double*>(ws + L.part);
  v.cls = reinterpret_cast<uint8_t*>(ws + L.cls);
  uint32_t* mlist = reinterpret_cast<uint32_t*>(ws + L.mlist);
  int* count = reinterpret_cast<int*>(ws + L.count);
  *status = 0;
  const int grid = (int)std::min<size_t>((N + kDifThreads - 1) / kDifThreads, (size_t)kDifCTAs);
  cudaError_t err = cudaMemsetAsync(count, 0, 2 * sizeof(int), st);
  if (err != cudaSuccess) return err;
  k_dif_mlist<<<grid, kDifThreads, 0, st>>>(g, c, mlist, count, N);
  k_dif_planes<<<grid, kDifThreads, 0, st>>>(g, c, mlist, count, plane);
  prof_mark("diffuse.planes", st);
  DifWalls walls;
  for (int f = 0; f < 6; ++f) {
    walls.on[f] = wall_T && wall_T[f] == wall_T[f] ? 1 : 0;  // NaN: no wall temperature
    walls.T[f] = walls.on[f] ? wall_T[f] : 0.0;
  }
  // the per-phase constants, in the order of the per-cell assembly
  const double inv_h = 1.0 / h, inv_dt = 1.0 / dt;
  DifConst K;
  const double kp[2] = {k_g, k_l}, Cph[2] = {g.Cp_g, g.Cp_l};
  for (int p = 0; p < 2; ++p) {
    K.kq[p] = kp[p] * (inv_h * inv_h);
    K.cdt[p] = Cph[p] * inv_dt;
    double d = K.cdt[p];
    for (int n = 0; n <= 6; ++n) {
      K.rdiag[p][n] = 1.0 / d;
      d += K.kq[p];
    }
  }
  // the cells next to the interface or a heated wall are listed in the
  // mixed-cell list's storage (k_dif_planes is done with it)
  uint32_t* ilist = mlist;
  const dim3 sgrid = dif_sweep_grid(g);
  if (phase_cp) k_dif_classify<true><<<sgrid, dim3(32, 8), 0, st>>>(g, c, e, v, walls, inv_dt, K, ilist, count + 1);
  else k_dif_classify<false><<<sgrid, dim3(32, 8), 0, st>>>(g, c, e, v, walls, inv_dt, K, ilist, count + 1);
  k_dif_irregular<<<grid, kDifThreads, 0, st>>>(g, h, inv_h, inv_dt, k_l, k_g, c, e, plane, v, walls, phase_cp, K,
                                                 ilist, count + 1);
  prof_mark("diffuse.assemble", st);
  unsigned long long* chg = reinterpret_cast<unsigned long long*>(v.part);
  // T0 is the first iterate; Ta and Tb take turns after it
  const double* Tin = v.T0;
  double* Tout = v.Ta;
  double* Tnext = v.Tb;
  int it = 0;
  double change = 0.0;
  bool done = false;
  while (!done && it < max_iter) {
    const bool check = (it + 1) % 4 == 0 || it + 1 == max_iter;
    if (check) {
      err = cudaMemsetAsync(chg, 0, sizeof(unsigned long long), st);
      if (err != cudaSuccess) return err;
      k_dif_jacobi<true><<<sgrid, dim3(32, 8), 0, st>>>(g, v, K, Tin, Tout, chg, phase_cp);
    } else {
      k_dif_jacobi<false><<<sgrid, dim3(32, 8), 0, st>>>(g, v, K, Tin, Tout, chg, phase_cp);
    }
    Tin = Tout;
    std::swap(Tout, Tnext);
    ++it;
    if (check) {
      unsigned long long hb = 0ull;
      err = cudaMemcpyAsync(&hb, chg, sizeof(hb), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) return err;
      std::memcpy(&change, &hb, sizeof(change));
      done = change <= tol;
    }
  }
  prof_mark("diffuse.jacobi", st);
  if (!done) *status = 2;
  k_dif_store<<<grid, kDifThreads, 0, st>>>(g, c, v, Tin, e, N, phase_cp);
  prof_mark("diffuse.store", st);
  if (iters_out) *iters_out = it;
  if (change_out) *change_out = change;
  return cudaGetLastError();
}

}  // namespace vofgb
