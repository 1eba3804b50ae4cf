// vof_mdot.cu -- mass transfer rate from PLIC interface distances (Malan et
// al., arXiv:2001.03477, Sec. 3.2 "Calculating the mass transfer rate":
// Eqs. mdot_calc, grad_n_T, plane_m, cell_d, dint_trans, the collinearity
// xi, normTgrad and the weights chi, gamma).
//
// For every mixed cell M the plane is put in Hessian form: unit normal
// n = m / |m| (m the MYC normal, pointing from liquid into gas) and distance
// d = alpha / |m| from M's low corner (Eq. cell_d).  Every pure cell P within
// two cells of a mixed cell (Chebyshev distance <= 2, the 3D reading of the
// 5 x 5 stencil) takes, among its mixed neighbours, the one of largest
// collinearity xi = |n . dx| (dx from that neighbour's low corner to P's
// centre; the first in z-, y-, x-order on ties) and the normal distance
// |d_Gamma| = |d - n . dx| h (Eq. dint_trans); its temperature gradient
// along n is (T_Gamma - T) / |d_Gamma| on the liquid side and
// (T - T_Gamma) / |d_Gamma| on the gas side (Eq. grad_n_T with n pointing
// into the gas).  Each mixed cell averages its pure neighbours' gradients
// per phase with weights gamma = |n . dx| / |dx|^2, dx the offset between
// the two centres (Eq. normTgrad), and mdot = (k_g grad_g - k_l grad_l) /
// h_fg (Eq. mdot_calc).  On a zero-gradient axis, offsets that leave the
// grid are not cells; periodic axes wrap.
//
// Five kernels, all over compact lists except the first:
//   k_md_list    stream c once: zero the outputs, list the mixed cells;
//   k_md_planes  a thread per mixed cell: MYC normal, plane constant (FP64),
//                Hessian plane;
//   k_md_band    a warp per mixed cell, its lanes over the 124 offsets: the
//                pure neighbours join the band (an atomic OR on one bit per
//                cell; the lane that sets the bit lists the cell);
//   k_md_grad    a warp per band cell: the most collinear mixed neighbour's
//                plane (warp argmax), |d_Gamma|, grad_n T;
//   k_md_avg     a warp per mixed cell: the weighted averages (lane sums and
//                a shuffle tree) and mdot.
// A warp per stencil spreads the 124 dependent neighbour loads over 32
// lanes: the lists are short (1e4-1e5 cells) and a thread per cell walking
// its 124 neighbours leaves the GPU waiting on load latency.
#include <algorithm>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {

namespace {

constexpr int kMdThreads = 128;
constexpr int kMdCTAs = 152 * 8;
constexpr int kListThreads = 256;

// a gradient that does not exist (a node on its plane): a quiet NaN pattern,
// tested on the integer pipe
constexpr long long kNoGrad = 0x7FF8DEAD00000000LL;

// 0.5 - d for the offsets d = -2 .. 2 (index d + 2): the node of a cell at
// offset -d from a mixed cell, from that cell's low corner
__constant__ double c_half_minus[5] = {2.5, 1.5, 0.5, -0.5, -1.5};
// offsets d = -2 .. 2 as doubles (index d + 2)
__constant__ double c_off[5] = {-2.0, -1.0, 0.0, 1.0, 2.0};

// 1 / |dx|^2 for the squared offsets 0 .. 12 of the 5 x 5 x 5 stencil
__constant__ double c_rinv[13] = {0.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0, 0.0, 0.125, 1.0 / 9.0, 0.0, 0.0,
                                  1.0 / 12.0};

// per axis: the neighbour coordinate of offset o in [-2, 2], or -1 where a
// zero-gradient axis has no cell
__device__ __forceinline__ int nb_coord(int x, int o, int n, int bc) {
  const int p = x + o;
  if (bc == 0) {
    int r = p % n;
    return r < 0 ? r + n : r;
  }
  return (p < 0 || p >= n) ? -1 : p;
}

__device__ __forceinline__ size_t nb_id(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

// grid-wide list append, one atomic per warp
__device__ __forceinline__ void warp_append(bool take, uint32_t v, uint32_t* list, int* counter) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (take) list[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

__global__ void __launch_bounds__(kListThreads)
k_md_list(GridDev g, const double* __restrict__ c, double* __restrict__ mdot, double* __restrict__ d_gamma,
          double* __restrict__ grad_n, double* __restrict__ dd, uint32_t* __restrict__ mlist,
          int* __restrict__ counters, size_t N) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  // whole warps iterate together (the append is warp-collective)
  const size_t n_iter = (N + stride - 1) / stride;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t it = 0; it < n_iter; ++it, i += stride) {
    const bool in = i < N;
    bool mx = false;
    if (in) {
      mx = is_mixed_b(__ldg(c + i), g);
      mdot[i] = 0.0;
      if (d_gamma) d_gamma[i] = -1.0;
      if (grad_n) grad_n[i] = 0.0;
      if (dd) dd[i] = 0.0;
    }
    warp_append(mx, (uint32_t)i, mlist, counters);
  }
}

__global__ void __launch_bounds__(kMdThreads)
k_md_planes(GridDev g, const double* __restrict__ c, const uint32_t* __restrict__ mlist,
            const int* __restrict__ counters, double4* __restrict__ plane) {
  const int nm = counters[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
    const uint32_t id = mlist[i];
    int x, y, z;
    cell_xyz(g, id, x, y, z);
    double s[27];
#pragma unroll
    for (int oz = 0; oz < 3; ++oz) {
      const int zz = map_idx(z + oz - 1, g.n[2], g.bc[2]);
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        const int yy = map_idx(y + oy - 1, g.n[1], g.bc[1]);
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          const int xx = map_idx(x + ox - 1, g.n[0], g.bc[0]);
          s[(oz * 3 + oy) * 3 + ox] = __ldg(c + nb_id(g, xx, yy, zz));
        }
      }
    }
    double m[3];
    myc_normal(s, m);
    const double al = plane_alpha(m[0], m[1], m[2], s[13]);
    const double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    double4 p;
    p.x = m[0] / len;
    p.y = m[1] / len;
    p.z = m[2] / len;
    p.w = al / len;
    plane[id] = p;
  }
}

// The 124 offsets of the 5 x 5 x 5 stencil (all but the centre, index 62)
// are spread over a warp's lanes: lane l takes the indices l, l + 32, l + 64
// and l + 96 below 125, in increasing order; index o is the offset
// (o % 5 - 2, o / 5 % 5 - 2, o / 25 - 2), so increasing indices visit z
// outer, then y, then x.
constexpr int kOffRounds = 4;

// the neighbour of (x, y, z) at stencil index o, or -1 (the centre, or off a
// zero-gradient axis); its offset in dx, dy, dz
__device__ __forceinline__ long long stencil_nb(const GridDev& g, int x, int y, int z, int o, int& dx, int& dy,
                                                int& dz) {
  dx = o % 5 - 2;
  dy = (o / 5) % 5 - 2;
  dz = o / 25 - 2;
  if (o >= 125 || o == 62) return -1;
  const int xx = nb_coord(x, dx, g.n[0], g.bc[0]);
  const int yy = nb_coord(y, dy, g.n[1], g.bc[1]);
  const int zz = nb_coord(z, dz, g.n[2], g.bc[2]);
  if (xx < 0 || yy < 0 || zz < 0) return -1;
  return (long long)nb_id(g, xx, yy, zz);
}

// one warp per mixed cell: its pure neighbours join the band; the lane that
// sets a cell's bit lists it
__global__ void __launch_bounds__(kMdThreads)
k_md_band(GridDev g, const double* __restrict__ c, const uint32_t* __restrict__ mlist, uint32_t* __restrict__ blist,
          int* __restrict__ counters, uint32_t* __restrict__ bits) {
  const int nm = counters[0];
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nm; i += nwarps) {
    int x, y, z;
    cell_xyz(g, mlist[i], x, y, z);
#pragma unroll
    for (int r = 0; r < kOffRounds; ++r) {
      int dx, dy, dz;
      const long long q = stencil_nb(g, x, y, z, lane + 32 * r, dx, dy, dz);
      bool take = false;
      if (q >= 0 && !is_mixed_b(__ldg(c + q), g)) {
        const uint32_t bit = 1u << ((uint32_t)q & 31u);
        take = (atomicOr(bits + (q >> 5), bit) & bit) == 0u;
      }
      warp_append(take, (uint32_t)q, blist, counters + 1);
    }
  }
}

// A warp takes kBatch consecutive list entries at a time and treats them
// one after the other, all lanes on one stencil; lane j keeps the result of
// entry j, and the per-cell tail (FP64 divisions) then runs on kBatch lanes
// at once.  8: enough lanes to share the divisions, enough warps (lists of
// 1e4-1e5 entries over ~5000 warps) to hide the neighbour loads.
constexpr int kMdWarps = kMdThreads / 32;
constexpr int kBatch = 8;

// one warp per band cell: the mixed neighbour of largest xi (the lowest
// stencil index on ties), |d_Gamma| and grad_n T.  The mixed neighbours are
// first compacted in stencil-index order into the warp's slots, so the FP64
// evaluation of xi runs lane-dense (one round for up to 32 of them).
__global__ void __launch_bounds__(kMdThreads)
k_md_grad(GridDev g, double h, const double* __restrict__ c, const double* __restrict__ e,
          const uint32_t* __restrict__ blist, const int* __restrict__ counters, const double4* __restrict__ plane,
          double* __restrict__ grad, double* __restrict__ d_gamma, double* __restrict__ grad_n) {
  __shared__ uint32_t s_q[kMdWarps][kOffRounds * 32];
  __shared__ unsigned char s_o[kMdWarps][kOffRounds * 32];
  const int nb_count = counters[1];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int b0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kBatch; b0 < nb_count; b0 += nwarps * kBatch) {
    const int nj = min(kBatch, nb_count - b0);
    const uint32_t my_id = lane < nj ? blist[b0 + lane] : 0u;
    double my_s = 0.0;
    for (int j = 0; j < nj; ++j) {
      const uint32_t id = __shfl_sync(0xffffffffu, my_id, j);
      int x, y, z;
      cell_xyz(g, id, x, y, z);
      // compact the mixed neighbours, in increasing stencil index
      int n = 0;
#pragma unroll
      for (int r = 0; r < kOffRounds; ++r) {
        int dx, dy, dz;
        const int o = lane + 32 * r;
        const long long q = stencil_nb(g, x, y, z, o, dx, dy, dz);
        const bool mx = q >= 0 && is_mixed_b(__ldg(c + q), g);
        const unsigned bm = __ballot_sync(0xffffffffu, mx);
        if (mx) {
          s_q[wib][n + __popc(bm & lt)] = (uint32_t)q;
          s_o[wib][n + __popc(bm & lt)] = (unsigned char)o;
        }
        n += __popc(bm);
      }
      __syncwarp();
      // this lane's best over its slots (increasing index: the first wins
      // ties): xi bits (non-negative doubles order as integers), stencil
      // index, signed distance
      long long bxi = -1;
      int bo = 1 << 30;
      double bs = 0.0;
      for (int k = lane; k < n; k += 32) {
        const int o = s_o[wib][k];
        const double4 p = plane[s_q[wib][k]];
        // dx: from the mixed cell's low corner to this cell's centre
        const double ndx =
            (p.x * c_half_minus[o % 5] + p.y * c_half_minus[(o / 5) % 5]) + p.z * c_half_minus[o / 25];
        const long long xb = dbits(fabs(ndx));
        if (xb > bxi) {
          bxi = xb;
          bo = o;
          bs = p.w - ndx;  // Eq. dint_trans, cell units
        }
      }
      __syncwarp();
      // warp argmax: largest xi, then lowest stencil index (band cells have
      // a mixed neighbour, so some lane holds one)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const long long oxi = __shfl_xor_sync(0xffffffffu, bxi, off);
        const int oo = __shfl_xor_sync(0xffffffffu, bo, off);
        const double os = __shfl_xor_sync(0xffffffffu, bs, off);
        if (oxi > bxi || (oxi == bxi && oo < bo)) {
          bxi = oxi;
          bo = oo;
          bs = os;
        }
      }
      if (lane == j) my_s = bs;
    }
    if (lane >= nj) continue;
    const double dist = fabs(my_s) * h;
    if (d_gamma) d_gamma[my_id] = dist;
    if (!dnz(dist)) {
      grad[my_id] = __longlong_as_double(kNoGrad);
      continue;
    }
    const double cv = __ldg(c + my_id);
    const double T = __ldg(e + my_id) / heat_cap(g.Cp_l, g.Cp_g, cv);
    const double gr = dgthalf(cv) ? (g.T_sat - T) / dist : (T - g.T_sat) / dist;
    grad[my_id] = gr;
    if (grad_n) grad_n[my_id] = gr;
  }
}

// one warp per mixed cell: per-phase weighted averages of the pure
// neighbours' gradients (lane partial sums in increasing stencil index,
// then a fixed shuffle tree) and mdot
__global__ void __launch_bounds__(kMdThreads)
k_md_avg(GridDev g, double k_l, double k_g, double h_fg, double dd_per_mdot, const double* __restrict__ c,
         const uint32_t* __restrict__ mlist, const int* __restrict__ counters, const double4* __restrict__ plane,
         const double* __restrict__ grad, double* __restrict__ mdot, double* __restrict__ dd) {
  const int nm = counters[0];
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kBatch; b0 < nm; b0 += nwarps * kBatch) {
    const int nj = min(kBatch, nm - b0);
    const uint32_t my_id = lane < nj ? mlist[b0 + lane] : 0u;
    double s_al = 0.0, s_wl = 0.0, s_ag = 0.0, s_wg = 0.0;
    for (int j = 0; j < nj; ++j) {
      const uint32_t id = __shfl_sync(0xffffffffu, my_id, j);
      int x, y, z;
      cell_xyz(g, id, x, y, z);
      const double4 p = plane[id];
      double acc_l = 0.0, w_l = 0.0, acc_g = 0.0, w_g = 0.0;
#pragma unroll
      for (int r = 0; r < kOffRounds; ++r) {
        int dx, dy, dz;
        const long long q = stencil_nb(g, x, y, z, lane + 32 * r, dx, dy, dz);
        if (q < 0) continue;
        const double cq = __ldg(c + q);
        if (is_mixed_b(cq, g)) continue;
        const double gq = grad[q];
        if (dbits(gq) == kNoGrad) continue;
        const double xi = fabs((p.x * c_off[dx + 2] + p.y * c_off[dy + 2]) + p.z * c_off[dz + 2]);
        const double gam = xi * c_rinv[dx * dx + dy * dy + dz * dz];
        if (dgthalf(cq)) {
          acc_l += gam * gq;
          w_l += gam;
        } else {
          acc_g += gam * gq;
          w_g += gam;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        acc_l += __shfl_xor_sync(0xffffffffu, acc_l, off);
        w_l += __shfl_xor_sync(0xffffffffu, w_l, off);
        acc_g += __shfl_xor_sync(0xffffffffu, acc_g, off);
        w_g += __shfl_xor_sync(0xffffffffu, w_g, off);
      }
      if (lane == j) {
        s_al = acc_l;
        s_wl = w_l;
        s_ag = acc_g;
        s_wg = w_g;
      }
    }
    if (lane >= nj) continue;
    const double gl = dgt0(s_wl) ? s_al / s_wl : 0.0;
    const double gg = dgt0(s_wg) ? s_ag / s_wg : 0.0;
    const double md = (k_g * gg - k_l * gl) / h_fg;
    mdot[my_id] = md;
    if (dd) dd[my_id] = dd_per_mdot * md;
  }
}

}  // namespace

size_t mdot_scratch_bytes(size_t N) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return a(N * sizeof(double4)) + a(N * sizeof(double)) + 2 * a(N * sizeof(uint32_t)) + a(((N + 31) / 32) * 4) +
         a(4 * sizeof(int));
}

struct MdotScratch {
  double4* plane;     // [N]: unit normal and distance of each mixed cell's plane
  double* grad;       // [N]: grad_n T of each band cell
  uint32_t* mlist;    // mixed cells, grid-wide, no fixed order
  uint32_t* blist;    // band cells, grid-wide, no fixed order
  uint32_t* bits;     // [ceil(N / 32)]: band membership
  int* counters;      // [0] mixed cells, [1] band cells
  size_t zero_bytes;  // bits and counters, zeroed by each call
};

static MdotScratch carve_mdot(size_t N, void* workspace) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* w = static_cast<char*>(workspace);
  MdotScratch s;
  s.plane = reinterpret_cast<double4*>(w);
  w += a(N * sizeof(double4));
  s.grad = reinterpret_cast<double*>(w);
  w += a(N * sizeof(double));
  s.mlist = reinterpret_cast<uint32_t*>(w);
  w += a(N * sizeof(uint32_t));
  s.blist = reinterpret_cast<uint32_t*>(w);
  w += a(N * sizeof(uint32_t));
  s.bits = reinterpret_cast<uint32_t*>(w);
  w += a(((N + 31) / 32) * 4);
  s.counters = reinterpret_cast<int*>(w);
  s.zero_bytes = a(((N + 31) / 32) * 4) + 4 * sizeof(int);
  return s;
}

int* mdot_counters(const GridDev& g, void* workspace) {
  return carve_mdot((size_t)g.n[0] * g.n[1] * g.n[2], workspace).counters;
}

cudaError_t launch_mass_transfer(const GridDev& g, double h, const double* c, const double* e, double k_l, double k_g,
                                 double h_fg, double dd_per_mdot, double* mdot, double* d_gamma, double* grad_n,
                                 double* dd, void* workspace, cudaStream_t st) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const MdotScratch s = carve_mdot(N, workspace);
  cudaError_t err = cudaMemsetAsync(s.bits, 0, s.zero_bytes, st);
  if (err != cudaSuccess) return err;
  prof_mark("mdot.memset", st);
  const int list_ctas = (int)std::min<size_t>((N + kListThreads - 1) / kListThreads, (size_t)152 * 16);
  k_md_list<<<list_ctas, kListThreads, 0, st>>>(g, c, mdot, d_gamma, grad_n, dd, s.mlist, s.counters, N);
  prof_mark("mdot.list", st);
  k_md_planes<<<kMdCTAs, kMdThreads, 0, st>>>(g, c, s.mlist, s.counters, s.plane);
  prof_mark("mdot.planes", st);
  k_md_band<<<kMdCTAs, kMdThreads, 0, st>>>(g, c, s.mlist, s.blist, s.counters, s.bits);
  prof_mark("mdot.band", st);
  k_md_grad<<<kMdCTAs, kMdThreads, 0, st>>>(g, h, c, e, s.blist, s.counters, s.plane, s.grad, d_gamma, grad_n);
  prof_mark("mdot.grad", st);
  k_md_avg<<<kMdCTAs, kMdThreads, 0, st>>>(g, k_l, k_g, h_fg, dd_per_mdot, c, s.mlist, s.counters, s.plane, s.grad,
                                           mdot, dd);
  prof_mark("mdot.avg", st);
  return cudaGetLastError();
}

}  // namespace vofgb
