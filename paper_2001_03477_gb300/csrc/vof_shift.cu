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

template <int K>
__device__ __forceinline__ void block_sums_sh(double (&v)[K], SumOut out, int block_lin) {
  __shared__ double red[K][kShThreads / 32];
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
      for (int w = 0; w < kShThreads / 32; ++w) s += red[k][w];
      if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = s;
      else if (out.diag) atomicAdd(out.diag + k, s);
    }
  }
}

__global__ void __launch_bounds__(kShThreads)
k_shift(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
        double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, SumOut sums) {
  constexpr int H = 2;
  constexpr int CX = kShBX + 2 * H, CY = kShBY + 2 * H, CZ = kShBZ + 2 * H;
  constexpr int PX = kShBX + 2, PY = kShBY + 2, PZ = kShBZ + 2;
  constexpr int NP = PX * PY * PZ;
  __shared__ double sc[CZ][CY][CX];
  __shared__ double sm[4][NP];  // m0, m1, m2, alpha of moving mixed cells
  __shared__ double ss[NP];     // |m|_2 dd (0: not moving)

  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * kShBX, y0 = blockIdx.y * kShBY, z0 = blockIdx.z * kShBZ;
  const int tid = threadIdx.x + kShBX * (threadIdx.y + kShBY * threadIdx.z);
  for (int q = tid; q < CX * CY * CZ; q += kShThreads) {
    int lx = q % CX, ly = (q / CX) % CY, lz = q / (CX * CY);
    int gx = map_idx(x0 + lx - H, nx, g.bc[0]);
    int gy = map_idx(y0 + ly - H, ny, g.bc[1]);
    int gz = map_idx(z0 + lz - H, nz, g.bc[2]);
    sc[lz][ly][lx] = c_in[((size_t)gz * ny + gy) * nx + gx];
  }
  __syncthreads();
  for (int q = tid; q < NP; q += kShThreads) {
    int px = q % PX, py = (q / PX) % PY, pz = q / (PX * PY);
    int cx = px + 1, cy = py + 1, cz = pz + 1;  // c-tile coordinates
    double ct = sc[cz][cy][cx];
    double sft = 0.0;
    if (is_mixed(ct, g.eps)) {
      double ddv = dd_uniform;
      if (dd) {
        int gx = map_idx(x0 + px - 1, nx, g.bc[0]);
        int gy = map_idx(y0 + py - 1, ny, g.bc[1]);
        int gz = map_idx(z0 + pz - 1, nz, g.bc[2]);
        ddv = dd[((size_t)gz * ny + gy) * nx + gx];
      }
      if (ddv != 0.0) {
        double s[27];
#pragma unroll
        for (int oz = 0; oz < 3; ++oz)
#pragma unroll
          for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) s[(oz * 3 + oy) * 3 + ox] = sc[cz + oz - 1][cy + oy - 1][cx + ox - 1];
        double m[3];
        myc_normal(s, m);
        double al = plane_alpha(m[0], m[1], m[2], ct);
        double mn2 = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        sft = mn2 * ddv;
        sm[0][q] = m[0]; sm[1][q] = m[1]; sm[2][q] = m[2]; sm[3][q] = al;
      }
    }
    ss[q] = sft;
  }
  __syncthreads();

  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // sum dc, unplaced, sum de, sum c, sum e
  if (gx < nx && gy < ny && gz < nz) {
    const size_t id = ((size_t)gz * ny + gy) * nx + gx;
    const double ct = sc[lz + H][ly + H][lx + H];
    const int qs = ((lz + 1) * PY + (ly + 1)) * PX + (lx + 1);
    double cn = ct;
    if (is_mixed(ct, g.eps)) {
      double sft = ss[qs];
      if (sft != 0.0) {
        double m0 = sm[0][qs], m1 = sm[1][qs], m2 = sm[2][qs], al = sm[3][qs];
        double lo = 0.0, hi = 0.0;
        if (m0 < 0.0) lo += m0; else hi += m0;
        if (m1 < 0.0) lo += m1; else hi += m1;
        if (m2 < 0.0) lo += m2; else hi += m2;
        double ast = al + sft;
        if (ast < lo) ast = lo;
        if (ast > hi) ast = hi;
        cn = volume(m0, m1, m2, ast);
      }
    } else {
      const bool full = ct >= 1.0 - g.eps;
      double best = 0.0;
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            if (!ox && !oy && !oz) continue;
            if (g.bc[0] != 0 && (gx + ox < 0 || gx + ox >= nx)) continue;
            if (g.bc[1] != 0 && (gy + oy < 0 || gy + oy >= ny)) continue;
            if (g.bc[2] != 0 && (gz + oz < 0 || gz + oz >= nz)) continue;
            const int qn = qs + (oz * PY + oy) * PX + ox;
            const double sft = ss[qn];
            if (sft == 0.0) continue;
            if ((sft < 0.0) != full) continue;
            const double m0 = sm[0][qn], m1 = sm[1][qn], m2 = sm[2][qn], al = sm[3][qn];
            const double shiftv = -((m0 * (double)(-ox) + m1 * (double)(-oy)) + m2 * (double)(-oz));
            const double a_old = al + shiftv;
            const double a_new = (al + sft) + shiftv;
            const double sw = volume(m0, m1, m2, a_new) - volume(m0, m1, m2, a_old);
            if (fabs(sw) > fabs(best)) best = sw;
          }
      if (best != 0.0) {
        double v = ct + best;
        double vc = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        acc[1] = v - vc;
        cn = vc;
      }
    }
    const double dc = cn - ct;
    const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
    const double en = e_in[id] + de;
    c_out[id] = cn;
    e_out[id] = en;
    acc[0] = dc;
    acc[2] = de;
    acc[3] = cn;
    acc[4] = en;
  }
  const int block_lin = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_sums_sh<5>(acc, sums, block_lin);
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

int shift_blocks(const GridDev& g) {
  dim3 gr = sh_grid(g);
  return (int)(gr.x * gr.y * gr.z);
}

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, SumOut sums, cudaStream_t st) {
  k_shift<<<sh_grid(g), dim3(kShBX, kShBY, kShBZ), 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sums);
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
