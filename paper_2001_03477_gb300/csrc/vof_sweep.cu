// vof_sweep.cu -- direction-split geometric VOF sweep with the thermal
// energy fluxed in tandem (Malan et al., arXiv:2001.03477, Sec. 3.3.1 Step 1
// with the Weymouth-Yue split scheme, and Sec. 3.4.1 Eq. disc_et_adv), plus
// the unfused energy update from exported VOF fluxes.
//
// One CTA owns a tile of cells.  c is staged in shared memory with a halo of
// 3 cells along the sweep axis and 1 across (MYC stencils of the donor
// cells), T = e / C_p(c) with a halo of 3 along the sweep axis (WENO5).
// Each face of the tile is evaluated once (geometry only when its donor is
// mixed), then every cell applies
//   c <- c + (F_l - cc a_l) - (F_r - cc a_r)
//   e <- e + (G_l - Theta a_l) - (G_r - Theta a_r),
//   G = (T_f C_pl) F + (T_f C_pg) (a - F),
// with cc = [c^n > 1/2] and Theta = C_p(cc) T^n frozen at the start of the
// step (see the `state` convention in include/vofgb.h).
#include "vof_launch.h"

namespace vofgb {

template <int AX>
struct SweepTile;
template <>
struct SweepTile<0> { static constexpr int BX = 32, BY = 4, BZ = 2; };
template <>
struct SweepTile<1> { static constexpr int BX = 32, BY = 8, BZ = 1; };
template <>
struct SweepTile<2> { static constexpr int BX = 32, BY = 1, BZ = 8; };

constexpr int kThreads = 256;

// block sum of up to 4 values into partials/diag
template <int K>
__device__ __forceinline__ void block_sums(double (&v)[K], SumOut out, int block_lin) {
  __shared__ double red[K][kThreads / 32];
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
      for (int w = 0; w < kThreads / 32; ++w) s += red[k][w];
      if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = s;
      else if (out.diag) atomicAdd(out.diag + k, s);
    }
  }
}

__device__ __forceinline__ size_t face_index(int ax, int f, int i, int j, int k, int nx, int ny) {
  // f along ax; (i,j,k) cell coordinates for the other two axes
  if (ax == 0) return ((size_t)k * ny + j) * (nx + 1) + f;
  if (ax == 1) return ((size_t)k * (ny + 1) + f) * nx + i;
  return ((size_t)f * ny + j) * nx + i;
}

template <int AX, bool ENERGY>
__global__ void __launch_bounds__(kThreads)
k_sweep(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
        double* __restrict__ e_out, const double* __restrict__ uf, uint8_t* __restrict__ state,
        double* __restrict__ theta, double* __restrict__ flux_out, SumOut sums, int* __restrict__ status) {
  constexpr int BX = SweepTile<AX>::BX, BY = SweepTile<AX>::BY, BZ = SweepTile<AX>::BZ;
  constexpr int HX = AX == 0 ? 3 : 1, HY = AX == 1 ? 3 : 1, HZ = AX == 2 ? 3 : 1;
  constexpr int CX = BX + 2 * HX, CY = BY + 2 * HY, CZ = BZ + 2 * HZ;
  constexpr int OX = AX == 0 ? 3 : 0, OY = AX == 1 ? 3 : 0, OZ = AX == 2 ? 3 : 0;  // T-tile halo
  constexpr int TX = BX + 2 * OX, TY = BY + 2 * OY, TZ = BZ + 2 * OZ;
  constexpr int FX = BX + (AX == 0), FY = BY + (AX == 1), FZ = BZ + (AX == 2);  // faces of the tile
  constexpr int NF = FX * FY * FZ;
  constexpr int NT = ENERGY ? TX * TY * TZ : 1;
  constexpr int NG = ENERGY ? NF : 1;

  __shared__ double sc[CZ][CY][CX];
  __shared__ double sT[NT];
  __shared__ double sE[NT];
  __shared__ double sF[NF];
  __shared__ double sA[NF];
  __shared__ double sG[NG];

  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);

  for (int q = tid; q < CX * CY * CZ; q += kThreads) {
    int lx = q % CX, ly = (q / CX) % CY, lz = q / (CX * CY);
    int gx = map_idx(x0 + lx - HX, nx, g.bc[0]);
    int gy = map_idx(y0 + ly - HY, ny, g.bc[1]);
    int gz = map_idx(z0 + lz - HZ, nz, g.bc[2]);
    sc[lz][ly][lx] = c_in[((size_t)gz * ny + gy) * nx + gx];
  }
  __syncthreads();
  if (ENERGY) {
    for (int q = tid; q < NT; q += kThreads) {
      int lx = q % TX, ly = (q / TX) % TY, lz = q / (TX * TY);
      int gx = map_idx(x0 + lx - OX, nx, g.bc[0]);
      int gy = map_idx(y0 + ly - OY, ny, g.bc[1]);
      int gz = map_idx(z0 + lz - OZ, nz, g.bc[2]);
      double ev = e_in[((size_t)gz * ny + gy) * nx + gx];
      double cv = sc[lz - OZ + HZ][ly - OY + HY][lx - OX + HX];
      sE[q] = ev;
      sT[q] = ev / heat_cap(g.Cp_l, g.Cp_g, cv);
    }
  }
  __syncthreads();

  const int nax = g.n[AX];
  for (int q = tid; q < NF; q += kThreads) {
    int fx = q % FX, fy = (q / FX) % FY, fz = q / (FX * FY);
    int cx = x0 + fx, cy = y0 + fy, cz = z0 + fz;  // cell on the + side of the face
    int f = AX == 0 ? cx : (AX == 1 ? cy : cz);
    bool ok = (AX == 0 ? (cy < ny && cz < nz && cx <= nx)
                       : AX == 1 ? (cx < nx && cz < nz && cy <= ny) : (cx < nx && cy < ny && cz <= nz));
    double Fv = 0.0, Gv = 0.0, a = 0.0;
    if (ok) {
      int fr = (g.bc[AX] == 0 && f == nax) ? 0 : f;
      a = uf[face_index(AX, fr, cx, cy, cz, nx, ny)] * g.lam;
      if (a != 0.0) {
        // donor cell in c-tile coordinates
        int dx = fx + HX, dy = fy + HY, dz = fz + HZ;
        if (a > 0.0) {
          if (AX == 0) dx -= 1;
          else if (AX == 1) dy -= 1;
          else dz -= 1;
        }
        double cd = sc[dz][dy][dx];
        if (is_mixed(cd, g.eps)) {
          double s[27];
#pragma unroll
          for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
              for (int ox = 0; ox < 3; ++ox) s[(oz * 3 + oy) * 3 + ox] = sc[dz + oz - 1][dy + oy - 1][dx + ox - 1];
          double m[3];
          myc_normal(s, m);
          double al = plane_alpha(m[0], m[1], m[2], cd);
          double da = fabs(a);
          if (da > 1.0 && status) atomicOr(status, DEV_CFL);
          double xs = a > 0.0 ? 1.0 - da : 0.0;
          double vol = slab_volume(m, al, AX, xs, da);
          Fv = a > 0.0 ? vol : -vol;
        } else {
          Fv = cd * a;
        }
        if (ENERGY) {
          // WENO5 stencil centred on the donor in T-tile coordinates
          int tx = dx - HX + OX, ty = dy - HY + OY, tz = dz - HZ + OZ;
          double v[5];
#pragma unroll
          for (int r = -2; r <= 2; ++r) {
            int rr = a > 0.0 ? r : -r;
            int px = tx + (AX == 0 ? rr : 0), py = ty + (AX == 1 ? rr : 0), pz = tz + (AX == 2 ? rr : 0);
            v[r + 2] = sT[(pz * TY + py) * TX + px];
          }
          double Tf = weno5(v[0], v[1], v[2], v[3], v[4]);
          Gv = (Tf * g.Cp_l) * Fv + (Tf * g.Cp_g) * (a - Fv);
        }
      }
      if (flux_out) {
        int fl = AX == 0 ? fx : (AX == 1 ? fy : fz);
        int bl = AX == 0 ? BX : (AX == 1 ? BY : BZ);
        if (fl < bl || f == nax) flux_out[face_index(AX, f, cx, cy, cz, nx, ny)] = Fv;
      }
    }
    sF[q] = Fv;
    sA[q] = a;
    if (ENERGY) sG[q] = Gv;
  }
  __syncthreads();

  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  double clip[1] = {0.0};
  if (gx < nx && gy < ny && gz < nz) {
    const size_t id = ((size_t)gz * ny + gy) * nx + gx;
    const double c = sc[lz + HZ][ly + HY][lx + HX];
    const int qa = (lz * FY + ly) * FX + lx;
    const int qb = qa + (AX == 0 ? 1 : (AX == 1 ? FX : FX * FY));
    const double Fl = sF[qa], Fr = sF[qb], al = sA[qa], ar = sA[qb];
    const uint8_t stv = state ? state[id] : (uint8_t)0;
    const bool dirty = stv & 1;
    const double ccv = dirty ? (double)((stv >> 1) & 1) : (c > 0.5 ? 1.0 : 0.0);
    const double lf = Fl - ccv * al, rf = Fr - ccv * ar;
    const double cn = (c + lf) - rf;
    const double cc2 = cn < 0.0 ? 0.0 : (cn > 1.0 ? 1.0 : cn);
    clip[0] = cn - cc2;
    c_out[id] = cc2;
    if (ENERGY) {
      const int qt = ((lz + OZ) * TY + (ly + OY)) * TX + (lx + OX);
      const double e = sE[qt];
      const double th = dirty ? theta[id] : heat_cap(g.Cp_l, g.Cp_g, ccv) * sT[qt];
      const double le = sG[qa] - th * al, re = sG[qb] - th * ar;
      const double en = (e + le) - re;
      e_out[id] = en;
      if (state && !dirty && (cc2 != c || en != e)) {
        state[id] = (uint8_t)(1 | (ccv > 0.5 ? 2 : 0));
        theta[id] = th;
      }
    }
  }
  const int block_lin = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_sums<1>(clip, sums, block_lin);
}

// Energy update from given face VOF fluxes (the unfused form).
template <int AX>
__global__ void __launch_bounds__(kThreads)
k_energy(GridDev g, const double* __restrict__ c_before, const double* __restrict__ c_after,
         const double* __restrict__ e_in, double* __restrict__ e_out, const double* __restrict__ Fface,
         const double* __restrict__ uf, uint8_t* __restrict__ state, double* __restrict__ theta) {
  constexpr int BX = SweepTile<AX>::BX, BY = SweepTile<AX>::BY, BZ = SweepTile<AX>::BZ;
  constexpr int OX = AX == 0 ? 3 : 0, OY = AX == 1 ? 3 : 0, OZ = AX == 2 ? 3 : 0;
  constexpr int TX = BX + 2 * OX, TY = BY + 2 * OY, TZ = BZ + 2 * OZ;
  constexpr int FX = BX + (AX == 0), FY = BY + (AX == 1), FZ = BZ + (AX == 2);
  constexpr int NF = FX * FY * FZ;
  __shared__ double sT[TX * TY * TZ];
  __shared__ double sE[TX * TY * TZ];
  __shared__ double sC[TX * TY * TZ];
  __shared__ double sG[NF];
  __shared__ double sA[NF];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
  const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
  for (int q = tid; q < TX * TY * TZ; q += kThreads) {
    int lx = q % TX, ly = (q / TX) % TY, lz = q / (TX * TY);
    int gx = map_idx(x0 + lx - OX, nx, g.bc[0]);
    int gy = map_idx(y0 + ly - OY, ny, g.bc[1]);
    int gz = map_idx(z0 + lz - OZ, nz, g.bc[2]);
    size_t id = ((size_t)gz * ny + gy) * nx + gx;
    double ev = e_in[id], cv = c_before[id];
    sE[q] = ev;
    sC[q] = cv;
    sT[q] = ev / heat_cap(g.Cp_l, g.Cp_g, cv);
  }
  __syncthreads();
  const int nax = g.n[AX];
  for (int q = tid; q < NF; q += kThreads) {
    int fx = q % FX, fy = (q / FX) % FY, fz = q / (FX * FY);
    int cx = x0 + fx, cy = y0 + fy, cz = z0 + fz;
    int f = AX == 0 ? cx : (AX == 1 ? cy : cz);
    bool ok = (AX == 0 ? (cy < ny && cz < nz && cx <= nx)
                       : AX == 1 ? (cx < nx && cz < nz && cy <= ny) : (cx < nx && cy < ny && cz <= nz));
    double Gv = 0.0, a = 0.0;
    if (ok) {
      int fr = (g.bc[AX] == 0 && f == nax) ? 0 : f;
      a = uf[face_index(AX, fr, cx, cy, cz, nx, ny)] * g.lam;
      if (a != 0.0) {
        double Fv = Fface[face_index(AX, f, cx, cy, cz, nx, ny)];
        int tx = fx + OX, ty = fy + OY, tz = fz + OZ;
        if (a > 0.0) {
          if (AX == 0) tx -= 1;
          else if (AX == 1) ty -= 1;
          else tz -= 1;
        }
        double v[5];
#pragma unroll
        for (int r = -2; r <= 2; ++r) {
          int rr = a > 0.0 ? r : -r;
          int px = tx + (AX == 0 ? rr : 0), py = ty + (AX == 1 ? rr : 0), pz = tz + (AX == 2 ? rr : 0);
          v[r + 2] = sT[(pz * TY + py) * TX + px];
        }
        double Tf = weno5(v[0], v[1], v[2], v[3], v[4]);
        Gv = (Tf * g.Cp_l) * Fv + (Tf * g.Cp_g) * (a - Fv);
      }
    }
    sG[q] = Gv;
    sA[q] = a;
  }
  __syncthreads();
  const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
  const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
  if (gx < nx && gy < ny && gz < nz) {
    const size_t id = ((size_t)gz * ny + gy) * nx + gx;
    const int qt = ((lz + OZ) * TY + (ly + OY)) * TX + (lx + OX);
    const int qa = (lz * FY + ly) * FX + lx;
    const int qb = qa + (AX == 0 ? 1 : (AX == 1 ? FX : FX * FY));
    const double c = sC[qt], e = sE[qt];
    const uint8_t stv = state ? state[id] : (uint8_t)0;
    const bool dirty = stv & 1;
    const double ccv = dirty ? (double)((stv >> 1) & 1) : (c > 0.5 ? 1.0 : 0.0);
    const double th = dirty ? theta[id] : heat_cap(g.Cp_l, g.Cp_g, ccv) * sT[qt];
    const double le = sG[qa] - th * sA[qa], re = sG[qb] - th * sA[qb];
    const double en = (e + le) - re;
    e_out[id] = en;
    if (state && !dirty && (c_after[id] != c || en != e)) {
      state[id] = (uint8_t)(1 | (ccv > 0.5 ? 2 : 0));
      theta[id] = th;
    }
  }
}

template <int AX>
static dim3 sweep_grid(const GridDev& g) {
  return dim3((g.n[0] + SweepTile<AX>::BX - 1) / SweepTile<AX>::BX, (g.n[1] + SweepTile<AX>::BY - 1) / SweepTile<AX>::BY,
              (g.n[2] + SweepTile<AX>::BZ - 1) / SweepTile<AX>::BZ);
}

template <int AX>
static dim3 sweep_block() {
  return dim3(SweepTile<AX>::BX, SweepTile<AX>::BY, SweepTile<AX>::BZ);
}

int sweep_blocks(int axis, const GridDev& g) {
  dim3 gr = axis == 0 ? sweep_grid<0>(g) : (axis == 1 ? sweep_grid<1>(g) : sweep_grid<2>(g));
  return (int)(gr.x * gr.y * gr.z);
}

template <int AX>
static cudaError_t launch_sweep_ax(const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                                   double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                                   SumOut sums, cudaStream_t st) {
  int* status = device_status_ptr();
  if (e_in)
    k_sweep<AX, true><<<sweep_grid<AX>(g), sweep_block<AX>(), 0, st>>>(g, c_in, e_in, c_out, e_out, uf, state, theta,
                                                                       flux_out, sums, status);
  else
    k_sweep<AX, false><<<sweep_grid<AX>(g), sweep_block<AX>(), 0, st>>>(g, c_in, nullptr, c_out, nullptr, uf, state,
                                                                        theta, flux_out, sums, status);
  return cudaGetLastError();
}

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SumOut sums, cudaStream_t st) {
  if (axis == 0) return launch_sweep_ax<0>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, st);
  if (axis == 1) return launch_sweep_ax<1>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, st);
  return launch_sweep_ax<2>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, st);
}

cudaError_t launch_energy(int axis, const GridDev& g, const double* c_before, const double* c_after,
                          const double* e_in, double* e_out, const double* F, const double* uf, uint8_t* state,
                          double* theta, cudaStream_t st) {
  if (axis == 0)
    k_energy<0><<<sweep_grid<0>(g), sweep_block<0>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  else if (axis == 1)
    k_energy<1><<<sweep_grid<1>(g), sweep_block<1>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  else
    k_energy<2><<<sweep_grid<2>(g), sweep_block<2>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  return cudaGetLastError();
}

}  // namespace vofgb
