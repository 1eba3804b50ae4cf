// vof_shift.cu -- Step 2 of the two-step VOF advection (Malan et al.,
// arXiv:2001.03477, Sec. 3.3.2, Eqs. vof_step2_full, Delta d and
// alpha^{n+1}) with the energy change Delta e = Delta c (C_pl - C_pg) T_Gamma
// (end of Sec. 3.4.1), and the stand-alone PLIC reconstruction (Sec. 3.2).
//
// The shift moves every mixed cell's plane along its normal:
//   * mixed:  alpha* = alpha + |m|_2 dd capped to the cell, c = V(m, alpha*);
//   * pure, of the receding phase: takes the largest volume swept inside it
//     by the shifted plane of an adjacent mixed cell extended across the
//     shared face, edge or corner (the cap's cut-off movement carried on in
//     the direction the interface moves).
// Only cells at the interface do work, so the kernels after the first one
// visit a compact list of the moving mixed cells instead of the grid.
#include "vof_launch.h"

namespace vofgb {

constexpr int kShBX = 32, kShBY = 4, kShBZ = 2, kShThreads = kShBX * kShBY * kShBZ;

__device__ __forceinline__ bool same_bits_dev(double a, double b) { return dbits(a) == dbits(b); }

template <int K>
__device__ __forceinline__ void block_sums_sh(double (&v)[K], SumOut out, int block_lin) {
  __shared__ double red[K][kShThreads / 32];  // up to 8 warps
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      const int nw = (int)(blockDim.x * blockDim.y * blockDim.z) / 32;
      for (int w = 0; w < nw; ++w) s += red[k][w];
      if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = s;
      else if (out.diag) atomicAdd(out.diag + k, s);
    }
  }
}

// ---------------------------------------------------------------------------
// Shift in three kernels.
//   SA (stream): copies c, e to the output, sums them, and lists the moving
//      mixed cells per warp (256 consecutive cells per warp, fixed order);
//   SM (planes): per moving mixed cell, the plane (MYC normal, plane
//      constant -- by bisection when c is within 1e-3 of 0 or 1, where the
//      plane is extrapolated into neighbours), the shift |m|_2 dd, and the
//      cell's own shifted volume;
//   SR (receivers): per moving mixed cell, the pure neighbours of the
//      receding phase it is the first to reach in the scan order; for each,
//      the largest volume swept in it by the extended planes of all its
//      moving mixed neighbours.
// Sums are per-CTA partials {dc, clamped, de, c, e}.
// ---------------------------------------------------------------------------
constexpr int kWarpCells = 256;

__device__ __forceinline__ void decode(const GridDev& g, size_t id, int& x, int& y, int& z) {
  x = (int)(id % (size_t)g.n[0]);
  const size_t r = id / (size_t)g.n[0];
  y = (int)(r % (size_t)g.n[1]);
  z = (int)(r / (size_t)g.n[1]);
}

__device__ __forceinline__ size_t cell_id(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

__global__ void __launch_bounds__(256)
k_shift_stream(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
               double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, ShiftScratch sc,
               SumOut sums) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int lane = threadIdx.x & 31;
  const size_t w = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  uint32_t* list = sc.list + w * kWarpCells;
  int n = 0;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool uni_moving = dnz(dd_uniform);
  for (int it = 0; it < kWarpCells / 32; ++it) {
    const size_t id = w * kWarpCells + (size_t)it * 32 + lane;
    const bool ok = id < N;
    double c = 0.0, e = 0.0;
    if (ok) {
      c = __ldg(c_in + id);
      e = __ldg(e_in + id);
      c_out[id] = c;
      e_out[id] = e;
      acc[3] += c;
      acc[4] += e;
    }
    bool moving = ok && is_mixed_b(c, g);
    if (moving) moving = dd ? dnz(__ldg(dd + id)) : uni_moving;
    const unsigned m = __ballot_sync(0xffffffffu, moving);
    if (moving) list[n + __popc(m & ((1u << lane) - 1u))] = (uint32_t)id;
    n += __popc(m);
  }
  if (lane == 0) sc.count[w] = n;
  block_sums_sh<5>(acc, sums, blockIdx.x);
}

__global__ void __launch_bounds__(256)
k_shift_planes(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
               double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, ShiftScratch sc,
               long long nwarps, SumOut sums) {
  const int lane = threadIdx.x & 31;
  const size_t w = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if ((long long)w < nwarps) {
    const int cnt = sc.count[w];
    const uint32_t* list = sc.list + w * kWarpCells;
    for (int i = lane; i < cnt; i += 32) {
      const size_t id = list[i];
      int x, y, z;
      decode(g, id, x, y, z);
      double st[27];
#pragma unroll
      for (int oz = 0; oz < 3; ++oz) {
        const int zz = map_idx(z + oz - 1, g.n[2], g.bc[2]);
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
          const int yy = map_idx(y + oy - 1, g.n[1], g.bc[1]);
#pragma unroll
          for (int ox = 0; ox < 3; ++ox) {
            const int xx = map_idx(x + ox - 1, g.n[0], g.bc[0]);
            st[(oz * 3 + oy) * 3 + ox] = __ldg(c_in + cell_id(g, xx, yy, zz));
          }
        }
      }
      const double ct = st[13];
      double m[3];
      myc_normal(st, m);
      const bool edge = dbits(ct) < 0x3F50624DD2F1A9FCLL /* 1e-3 */ || dbits(ct) > 0x3FEFF7CED916872BLL /* 0.999 */;
      const double al = edge ? plane_alpha_bisect(m[0], m[1], m[2], ct) : plane_alpha(m[0], m[1], m[2], ct);
      const double ddv = dd ? __ldg(dd + id) : dd_uniform;
      const double mn2 = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
      const double sft = mn2 * ddv;
      double4 pl;
      pl.x = m[0]; pl.y = m[1]; pl.z = m[2]; pl.w = al;
      reinterpret_cast<double4*>(sc.plane)[id] = pl;
      sc.shift[id] = sft;
      // own shift, capped to the cell
      double lo = 0.0, hi = 0.0;
      if (m[0] < 0.0) lo += m[0]; else hi += m[0];
      if (m[1] < 0.0) lo += m[1]; else hi += m[1];
      if (m[2] < 0.0) lo += m[2]; else hi += m[2];
      double ast = al + sft;
      if (ast < lo) ast = lo;
      if (ast > hi) ast = hi;
      const double cn = volume(m[0], m[1], m[2], ast);
      if (!same_bits_dev(cn, ct)) {
        const double dc = cn - ct;
        const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
        c_out[id] = cn;
        e_out[id] = __ldg(e_in + id) + de;
        acc[0] += dc;
        acc[2] += de;
        acc[3] += dc;  // sum c_out = sum c_in + sum dc
        acc[4] += de;
      }
    }
  }
  block_sums_sh<5>(acc, sums, blockIdx.x);
}

// moving mixed cell whose shift has the sign that reaches a receiver of this kind
__device__ __forceinline__ bool reaches(const GridDev& g, const double* __restrict__ c_in,
                                        const double* __restrict__ dd, double dd_uniform, size_t q, bool full) {
  if (!is_mixed_b(__ldg(c_in + q), g)) return false;
  const double ddv = dd ? __ldg(dd + q) : dd_uniform;
  return dnz(ddv) && (dlt0(ddv) == full);
}

__global__ void __launch_bounds__(256)
k_shift_receivers(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in,
                  double* __restrict__ c_out, double* __restrict__ e_out, const double* __restrict__ dd,
                  double dd_uniform, ShiftScratch sc, long long nwarps, SumOut sums) {
  const int lane = threadIdx.x & 31;
  const size_t w = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if ((long long)w < nwarps) {
    const int cnt = sc.count[w];
    const uint32_t* list = sc.list + w * kWarpCells;
    for (int i = lane; i < cnt; i += 32) {
      const size_t qid = list[i];
      int qx, qy, qz;
      decode(g, qid, qx, qy, qz);
      const double qdd = dd ? __ldg(dd + qid) : dd_uniform;
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            if (!ox && !oy && !oz) continue;
            int px = qx + ox, py = qy + oy, pz = qz + oz;
            if (g.bc[0] != 0 && (px < 0 || px >= nx)) continue;
            if (g.bc[1] != 0 && (py < 0 || py >= ny)) continue;
            if (g.bc[2] != 0 && (pz < 0 || pz >= nz)) continue;
            px = map_idx(px, nx, g.bc[0]);
            py = map_idx(py, ny, g.bc[1]);
            pz = map_idx(pz, nz, g.bc[2]);
            const size_t pid = cell_id(g, px, py, pz);
            const double cp = __ldg(c_in + pid);
            if (is_mixed_b(cp, g)) continue;
            const bool full = is_full_b(cp, g);
            if (dlt0(qdd) != full) continue;
            // this receiver is settled by its first reaching neighbour offset
            // in the scan order (z outer, x inner), which must be the offset
            // back to this cell (on periodic axes of 1 or 2 cells several
            // offsets lead to the same cell; only one of them settles it)
            int first = -1;
            for (int rz = -1; rz <= 1 && first < 0; ++rz)
              for (int ry = -1; ry <= 1 && first < 0; ++ry)
                for (int rx = -1; rx <= 1 && first < 0; ++rx) {
                  if (!rx && !ry && !rz) continue;
                  int sx = px + rx, sy = py + ry, sz = pz + rz;
                  if (g.bc[0] != 0 && (sx < 0 || sx >= nx)) continue;
                  if (g.bc[1] != 0 && (sy < 0 || sy >= ny)) continue;
                  if (g.bc[2] != 0 && (sz < 0 || sz >= nz)) continue;
                  const size_t sid =
                      cell_id(g, map_idx(sx, nx, g.bc[0]), map_idx(sy, ny, g.bc[1]), map_idx(sz, nz, g.bc[2]));
                  if (reaches(g, c_in, dd, dd_uniform, sid, full)) first = ((rz + 1) * 3 + (ry + 1)) * 3 + (rx + 1);
                }
            if (first != ((1 - oz) * 3 + (1 - oy)) * 3 + (1 - ox)) continue;
            // settle the receiver: largest sweep over its reaching neighbours
            double best = 0.0;
            for (int rz = -1; rz <= 1; ++rz)
              for (int ry = -1; ry <= 1; ++ry)
                for (int rx = -1; rx <= 1; ++rx) {
                  if (!rx && !ry && !rz) continue;
                  int sx = px + rx, sy = py + ry, sz = pz + rz;
                  if (g.bc[0] != 0 && (sx < 0 || sx >= nx)) continue;
                  if (g.bc[1] != 0 && (sy < 0 || sy >= ny)) continue;
                  if (g.bc[2] != 0 && (sz < 0 || sz >= nz)) continue;
                  const size_t sid =
                      cell_id(g, map_idx(sx, nx, g.bc[0]), map_idx(sy, ny, g.bc[1]), map_idx(sz, nz, g.bc[2]));
                  if (!reaches(g, c_in, dd, dd_uniform, sid, full)) continue;
                  const double4 pl = reinterpret_cast<const double4*>(sc.plane)[sid];
                  const double sft = sc.shift[sid];
                  const double m0 = pl.x, m1 = pl.y, m2 = pl.z, al = pl.w;
                  // the receiver sits at offset -(rx, ry, rz) from the source
                  const double shiftv = -((m0 * (double)(-rx) + m1 * (double)(-ry)) + m2 * (double)(-rz));
                  const double a_old = al + shiftv;
                  const double a_new = (al + sft) + shiftv;
                  double lo = 0.0, hi = 0.0;
                  if (m0 < 0.0) lo += m0; else hi += m0;
                  if (m1 < 0.0) lo += m1; else hi += m1;
                  if (m2 < 0.0) lo += m2; else hi += m2;
                  // the extended plane stays outside the receiver: both
                  // volumes are exactly 1 (or 0); the margin clears rounding
                  if (full ? (a_new >= hi + 1e-9) : (a_new <= lo - 1e-9)) continue;
                  const double sw = volume(m0, m1, m2, a_new) - volume(m0, m1, m2, a_old);
                  if (fabs(sw) > fabs(best)) best = sw;
                }
            if (dnz(best)) {
              const double v = cp + best;
              const double vc = dlt0(v) ? 0.0 : (dgt1(v) ? 1.0 : v);
              if (!deq(v, vc)) acc[1] += v - vc;
              if (!same_bits_dev(vc, cp)) {
                const double dc = vc - cp;
                const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
                c_out[pid] = vc;
                e_out[pid] = __ldg(e_in + pid) + de;
                acc[0] += dc;
                acc[2] += de;
                acc[3] += dc;
                acc[4] += de;
              }
            }
          }
    }
  }
  block_sums_sh<5>(acc, sums, blockIdx.x);
}

__global__ void __launch_bounds__(kShThreads)
k_reconstruct(GridDev g, const double* __restrict__ c, double* __restrict__ m_out, double* __restrict__ a_out,
              uint8_t* __restrict__ mixed) {
  constexpr int CX = kShBX + 2, CY = kShBY + 2, CZ = kShBZ + 2;
  __shared__ double sc[CZ][CY][CX];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * kShBX, y0 = blockIdx.y * kShBY, z0 = blockIdx.z * kShBZ;
  const int tid = threadIdx.x + kShBX * (threadIdx.y + kShBY * threadIdx.z);
  for (int q = tid; q < CX * CY * CZ; q += kShThreads) {
    int lx = q % CX, ly = (q / CX) % CY, lz = q / (CX * CY);
    int gx = map_idx(x0 + lx - 1, nx, g.bc[0]);
    int gy = map_idx(y0 + ly - 1, ny, g.bc[1]);
    int gz = map_idx(z0 + lz - 1, nz, g.bc[2]);
    sc[lz][ly][lx] = c[((size_t)gz * ny + gy) * nx + gx];
  }
  __syncthreads();
  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  if (gx >= nx || gy >= ny || gz >= nz) return;
  const size_t N = (size_t)nx * ny * nz;
  const size_t id = ((size_t)gz * ny + gy) * nx + gx;
  const double ct = sc[lz + 1][ly + 1][lx + 1];
  double m[3] = {0.0, 0.0, 0.0}, al = 0.0;
  uint8_t mx = 0;
  if (is_mixed(ct, g.eps)) {
    double s[27];
#pragma unroll
    for (int oz = 0; oz < 3; ++oz)
#pragma unroll
      for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) s[(oz * 3 + oy) * 3 + ox] = sc[lz + oz][ly + oy][lx + ox];
    myc_normal(s, m);
    al = plane_alpha(m[0], m[1], m[2], ct);
    mx = 1;
  }
  m_out[id] = m[0];
  m_out[N + id] = m[1];
  m_out[2 * N + id] = m[2];
  a_out[id] = al;
  mixed[id] = mx;
}

static dim3 sh_grid(const GridDev& g) {
  return dim3((g.n[0] + kShBX - 1) / kShBX, (g.n[1] + kShBY - 1) / kShBY, (g.n[2] + kShBZ - 1) / kShBZ);
}

static long long shift_warps(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  return (long long)((N + kWarpCells - 1) / kWarpCells);
}

// CTAs of each shift kernel (8 warps of 256 cells)
int shift_blocks(const GridDev& g) { return (int)((shift_warps(g) + 7) / 8); }

size_t shift_scratch_bytes(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_warps(g);
  size_t b = 0;
  b += (nw * kWarpCells * 4 + 255) & ~(size_t)255;  // lists
  b += (nw * 4 + 255) & ~(size_t)255;               // counts
  b += (N * 32 + 255) & ~(size_t)255;               // planes
  b += (N * 8 + 255) & ~(size_t)255;                // shifts
  return b;
}

ShiftScratch carve_shift_scratch(const GridDev& g, void* ws) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_warps(g);
  char* b = static_cast<char*>(ws);
  ShiftScratch s;
  s.list = reinterpret_cast<uint32_t*>(b);
  b += (nw * kWarpCells * 4 + 255) & ~(size_t)255;
  s.count = reinterpret_cast<int*>(b);
  b += (nw * 4 + 255) & ~(size_t)255;
  s.plane = reinterpret_cast<double*>(b);
  b += (N * 32 + 255) & ~(size_t)255;
  s.shift = reinterpret_cast<double*>(b);
  return s;
}

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, ShiftScratch sc, SumOut sums,
                         cudaStream_t st) {
  const long long nw = shift_warps(g);
  const unsigned nb = (unsigned)((nw + 7) / 8);
  // the three kernels write partials to consecutive regions of nb CTAs
  SumOut s0 = sums, s1 = sums, s2 = sums;
  if (sums.partials) {
    s1.partials = sums.partials + (size_t)nb * sums.stride;
    s2.partials = sums.partials + (size_t)2 * nb * sums.stride;
  }
  k_shift_stream<<<nb, 256, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc, s0);
  k_shift_planes<<<nb, 256, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc, nw, s1);
  k_shift_receivers<<<nb, 256, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc, nw, s2);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && state)
    err = cudaMemsetAsync(state, 0, (size_t)g.n[0] * g.n[1] * g.n[2], st);
  return err;
}

cudaError_t launch_reconstruct(const GridDev& g, const double* c, double* m, double* alpha, uint8_t* mixed,
                               cudaStream_t st) {
  k_reconstruct<<<sh_grid(g), dim3(kShBX, kShBY, kShBZ), 0, st>>>(g, c, m, alpha, mixed);
  return cudaGetLastError();
}

// Deterministic reduction of per-block partials: one CTA, fixed order.
__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ partials, int nblocks, int stride, int k0,
                                                int nk, double* __restrict__ out) {
  __shared__ double red[256];
  for (int k = 0; k < nk; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[(size_t)b * stride + k0 + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}

cudaError_t launch_reduce(const double* partials, int nblocks, int stride, int k0, int nk, double* out,
                          cudaStream_t st) {
  k_reduce<<<1, 256, 0, st>>>(partials, nblocks, stride, k0, nk, out);
  return cudaGetLastError();
}

}  // namespace vofgb
