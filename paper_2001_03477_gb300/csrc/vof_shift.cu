// vof_shift.cu -- Step 2 of the two-step VOF advection (Malan et al.,
// arXiv:2001.03477, Sec. 3.3.2, Eqs. vof_step2_full, Delta d and
// alpha^{n+1}) with the energy change Delta e = Delta c (C_pl - C_pg) T_Gamma
// (end of Sec. 3.4.1), and the stand-alone PLIC reconstruction (Sec. 3.2).
//
// Shift, one fused pass: the CTA stages c with a halo of 2, reconstructs the
// plane (MYC normal + plane constant) of every moving mixed cell of the tile
// and its 1-cell ring, then each cell of the tile
//   * mixed:  alpha* = alpha + |m|_2 dd capped to the cell, c = V(m, alpha*);
//   * pure, of the receding phase: takes the largest volume swept inside it
//     by the shifted plane of an adjacent mixed cell extended across the
//     shared face, edge or corner (the cap's cut-off movement carried on in
//     the direction the interface moves).
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

// Shift kernel: a CTA owns a 32 x kShTY column of cells and walks kShSegZ planes
// along z.  Shared-memory rings hold c of planes z..z+2 (halo 2 in x and y)
// and the plane data (m, alpha, |m|_2 dd) of the moving mixed cells of
// planes z-1..z+1 (halo 1); each thread then settles its cell of plane z.
constexpr int kShSegZ = 8;    // short z segments and small CTAs: the FP64 work of
constexpr int kShTY = 4;      // the interface is spread over many CTAs
constexpr int kShT = 32 * kShTY;
constexpr int kRX = kShBX + 4, kRY = kShTY + 4;   // c plane with halo 2
constexpr int kPX = kShBX + 2, kPY = kShTY + 2;   // plane-data region with halo 1
constexpr int kRP = kRX * kRY, kPP = kPX * kPY;

struct ShiftSmem {
  double c[3][kRP];
  double pd[3][5][kPP];   // m0, m1, m2, alpha, shift
  int any[3];
};

// Plane of a moving mixed cell from its 3x3x3 stencil (three shared-memory
// rows of the c ring, each pointer at the cell's own column): MYC normal,
// plane constant, shift |m|_2 dd.  Writes m0, m1, m2, alpha at out[0],
// out[kPP], out[2 kPP], out[3 kPP]; returns the shift.
__device__ __noinline__ double moving_plane(const double* zm, const double* z0p, const double* zp, double ct,
                                            double ddv, double* out) {
  double st[27];
  const double* rows[3] = {zm, z0p, zp};
#pragma unroll
  for (int oz = 0; oz < 3; ++oz)
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) st[(oz * 3 + oy) * 3 + ox] = rows[oz][(oy - 1) * kRX + (ox - 1)];
  double m[3];
  myc_normal(st, m);
  // nearly empty or full cells: alpha(c) is ill-conditioned and this plane
  // is extrapolated into the neighbours, so take the bisection constant
  const bool edge = dbits(ct) < 0x3F50624DD2F1A9FCLL /* 1e-3 */ || dbits(ct) > 0x3FEFF7CED916872BLL /* 0.999 */;
  const double al = edge ? plane_alpha_bisect(m[0], m[1], m[2], ct) : plane_alpha(m[0], m[1], m[2], ct);
  const double mn2 = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  out[0] = m[0];
  out[kPP] = m[1];
  out[2 * kPP] = m[2];
  out[3 * kPP] = al;
  return mn2 * ddv;
}

// Largest volume swept inside a pure cell by the shifted plane of an
// adjacent moving mixed cell extended into it (26 neighbours, z outer, x
// inner; neighbours beyond a zero-gradient boundary do not count).
// p[0..2]: plane data of planes z-1, z, z+1 (layout [5][kPP]).
__device__ __noinline__ double extended_sweep(GridDev g, const double* pm, const double* p0, const double* pp, int q,
                                              int gx, int gy, int z, bool full) {
  const double* pl[3] = {pm, p0, pp};
  double best = 0.0;
  for (int oz = -1; oz <= 1; ++oz) {
    if (g.bc[2] != 0 && (z + oz < 0 || z + oz >= g.n[2])) continue;
    const double* P = pl[oz + 1];
    for (int oy = -1; oy <= 1; ++oy) {
      if (g.bc[1] != 0 && (gy + oy < 0 || gy + oy >= g.n[1])) continue;
      for (int ox = -1; ox <= 1; ++ox) {
        if (!ox && !oy && !oz) continue;
        if (g.bc[0] != 0 && (gx + ox < 0 || gx + ox >= g.n[0])) continue;
        const int qn = q + oy * kPX + ox;
        const double sft = P[4 * kPP + qn];
        if (!dnz(sft)) continue;
        if (dlt0(sft) != full) continue;
        const double m0 = P[qn], m1 = P[kPP + qn], m2 = P[2 * kPP + qn], al = P[3 * kPP + qn];
        const double shiftv = -((m0 * (double)(-ox) + m1 * (double)(-oy)) + m2 * (double)(-oz));
        const double a_old = al + shiftv;
        const double a_new = (al + sft) + shiftv;
        // the extended plane stays outside this cell (both volumes are
        // exactly 1, or exactly 0): nothing is swept.  The 1e-9 margin keeps
        // the test clear of the rounding of the volume function's own test.
        double lo = 0.0, hi = 0.0;
        if (m0 < 0.0) lo += m0; else hi += m0;
        if (m1 < 0.0) lo += m1; else hi += m1;
        if (m2 < 0.0) lo += m2; else hi += m2;
        if (full ? (a_new >= hi + 1e-9) : (a_new <= lo - 1e-9)) continue;
        const double sw = volume(m0, m1, m2, a_new) - volume(m0, m1, m2, a_old);
        if (fabs(sw) > fabs(best)) best = sw;
      }
    }
  }
  return best;
}

__global__ void __launch_bounds__(kShT, 4)
k_shift(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
        double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, SumOut sums) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ShiftSmem& S = *reinterpret_cast<ShiftSmem*>(smem_raw);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int x0 = blockIdx.x * kShBX, y0 = blockIdx.y * kShTY;
  const int z0 = blockIdx.z * kShSegZ, z1 = min(z0 + kShSegZ, nz);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool cell_ok = gx < nx && gy < ny;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // sum dc, unplaced, sum de, sum c, sum e

  auto load_plane = [&](int z, int slot) {
    const int zz = map_idx(z, nz, g.bc[2]);
    for (int q = tid; q < kRP; q += kShT) {
      const int lx = q % kRX, ly = q / kRX;
      const int xx = map_idx(x0 + lx - 2, nx, g.bc[0]);
      const int yy = map_idx(y0 + ly - 2, ny, g.bc[1]);
      S.c[slot][q] = __ldg(c_in + ((size_t)zz * ny + yy) * nx + xx);
    }
  };
  // plane data of plane z (ring slot z % 3) from c planes z-1, z, z+1
  auto plane_data = [&](int z) {
    const int sl = ((z % 3) + 3) % 3;
    const int sm1 = ((z - 1) % 3 + 3) % 3, sp1 = ((z + 1) % 3 + 3) % 3;
    int any = 0;
    for (int q = tid; q < kPP; q += kShT) {
      const int px = q % kPX, py = q / kPX;
      const int rq = (py + 1) * kRX + (px + 1);
      const double ct = S.c[sl][rq];
      double sft = 0.0;
      if (is_mixed_b(ct, g)) {
        double ddv = dd_uniform;
        if (dd) {
          const int xx = map_idx(x0 + px - 1, nx, g.bc[0]);
          const int yy = map_idx(y0 + py - 1, ny, g.bc[1]);
          const int zz = map_idx(z, nz, g.bc[2]);
          ddv = __ldg(dd + ((size_t)zz * ny + yy) * nx + xx);
        }
        if (dnz(ddv)) {
          sft = moving_plane(S.c[sm1] + rq, S.c[sl] + rq, S.c[sp1] + rq, ct, ddv, &S.pd[sl][0][q]);
          any = 1;
        }
      }
      S.pd[sl][4][q] = sft;
    }
    if (__any_sync(0xffffffffu, any) && (tid & 31) == 0) atomicOr(&S.any[sl], 1);
  };

  // prologue: c planes z0-1, z0, z0+1 and plane data of z0-1 (needs z0-2)
  if (tid < 3) S.any[tid] = 0;
  load_plane(z0 - 2, ((z0 - 2) % 3 + 3) % 3);
  load_plane(z0 - 1, ((z0 - 1) % 3 + 3) % 3);
  load_plane(z0, ((z0) % 3 + 3) % 3);
  __syncthreads();
  plane_data(z0 - 1);
  __syncthreads();
  // now the slot of z0-2 is free: load z0+1, then plane data of z0
  load_plane(z0 + 1, ((z0 + 1) % 3 + 3) % 3);
  __syncthreads();
  plane_data(z0);
  __syncthreads();

  for (int z = z0; z < z1; ++z) {
    // own cell's energy, issued before the plane work to hide its latency
    const size_t id = ((size_t)z * ny + gy) * nx + gx;
    const double ev = cell_ok ? __ldg(e_in + id) : 0.0;
    // c of plane z+2 replaces plane z-1; plane data of z+1 replaces z-2
    const int sz2 = ((z + 2) % 3 + 3) % 3;
    if (tid == 0) S.any[((z + 1) % 3 + 3) % 3] = 0;
    load_plane(z + 2, sz2);
    __syncthreads();
    plane_data(z + 1);
    __syncthreads();
    if (cell_ok) {
      const int sl = ((z % 3) + 3) % 3;
      const int q = (ty + 1) * kPX + (tx + 1);
      const double ct = S.c[sl][(ty + 2) * kRX + (tx + 2)];
      double cn = ct;
      if (is_mixed_b(ct, g)) {
        const double sft = S.pd[sl][4][q];
        if (dnz(sft)) {
          const double m0 = S.pd[sl][0][q], m1 = S.pd[sl][1][q], m2 = S.pd[sl][2][q], al = S.pd[sl][3][q];
          double lo = 0.0, hi = 0.0;
          if (m0 < 0.0) lo += m0; else hi += m0;
          if (m1 < 0.0) lo += m1; else hi += m1;
          if (m2 < 0.0) lo += m2; else hi += m2;
          double ast = al + sft;
          if (ast < lo) ast = lo;
          if (ast > hi) ast = hi;
          cn = volume(m0, m1, m2, ast);
        }
      } else if (S.any[0] | S.any[1] | S.any[2]) {
        const bool full = is_full_b(ct, g);
        const double* pl[3] = {&S.pd[((z - 1) % 3 + 3) % 3][0][0], &S.pd[((z % 3) + 3) % 3][0][0],
                               &S.pd[((z + 1) % 3 + 3) % 3][0][0]};
        const double best = extended_sweep(g, pl[0], pl[1], pl[2], q, gx, gy, z, full);
        if (dnz(best)) {
          const double v = ct + best;
          const double vc = dlt0(v) ? 0.0 : (dgt1(v) ? 1.0 : v);
          if (!deq(v, vc)) acc[1] += v - vc;
          cn = vc;
        }
      }
      double en = ev;
      if (!same_bits_dev(cn, ct)) {
        const double dc = cn - ct;
        const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
        en = ev + de;
        acc[0] += dc;
        acc[2] += de;
      }
      c_out[id] = cn;
      e_out[id] = en;
      acc[3] += cn;
      acc[4] += en;
    }
    __syncthreads();
  }
  block_sums_sh<5>(acc, sums, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
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

static dim3 shm_grid(const GridDev& g) {
  return dim3((g.n[0] + kShBX - 1) / kShBX, (g.n[1] + kShTY - 1) / kShTY, (g.n[2] + kShSegZ - 1) / kShSegZ);
}

int shift_blocks(const GridDev& g) {
  dim3 gr = shm_grid(g);
  return (int)(gr.x * gr.y * gr.z);
}

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, SumOut sums, cudaStream_t st) {
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = sizeof(ShiftSmem);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  k_shift<<<shm_grid(g), dim3(kShBX, kShTY), smem, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sums);
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
