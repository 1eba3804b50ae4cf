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

__device__ __forceinline__ size_t face_index(int ax, int f, int i, int j, int k, int nx, int ny) {
  // f along ax; (i,j,k) cell coordinates for the other two axes
  if (ax == 0) return ((size_t)k * ny + j) * (nx + 1) + f;
  if (ax == 1) return ((size_t)k * (ny + 1) + f) * nx + i;
  return ((size_t)f * ny + j) * nx + i;
}

// ---------------------------------------------------------------------------
// No-op cells.  A cell's c and e come out bit-identical when the 7 cells
// around it along the sweep axis have the same (c, e) bits, c is exactly 0 or
// 1 and the cell has not changed earlier in the step: both donors are then
// pure with the same c, F = c a, both face temperatures equal T, and
// (G - Theta a) vanishes exactly on both faces.  No-op cells cost no FP64
// work; face fluxes are evaluated only next to non-no-op cells and
// T = e / C_p(c) only where such a face needs it.
// ---------------------------------------------------------------------------

constexpr unsigned kFull = 0xffffffffu;
constexpr long long kOneBits = 0x3FF0000000000000LL;

__device__ __forceinline__ bool same_bits(double a, double b) { return dbits(a) == dbits(b); }
__device__ __forceinline__ bool is01(double c) { long long b = dbits(c); return b == 0 || b == kOneBits; }

__device__ __forceinline__ size_t cell_at(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

// Face VOF flux of a mixed donor (rare path): MYC on the donor's 27-cell
// stencil (read through the read-only cache), plane constant, slab volume.
__device__ __noinline__ double mixed_donor_flux(GridDev g, const double* __restrict__ c_in, int ax, int dx, int dy,
                                                int dz, double cd, double a, int* status) {
  double s[27];
#pragma unroll
  for (int oz = 0; oz < 3; ++oz) {
    int zz = map_idx(dz + oz - 1, g.n[2], g.bc[2]);
#pragma unroll
    for (int oy = 0; oy < 3; ++oy) {
      int yy = map_idx(dy + oy - 1, g.n[1], g.bc[1]);
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        int xx = map_idx(dx + ox - 1, g.n[0], g.bc[0]);
        s[(oz * 3 + oy) * 3 + ox] = __ldg(c_in + cell_at(g, xx, yy, zz));
      }
    }
  }
  double m[3];
  myc_normal(s, m);
  double al = plane_alpha(m[0], m[1], m[2], cd);
  double da = fabs(a);
  if (da > 1.0 && status) atomicOr(status, DEV_CFL);
  double xs = dgt0(a) ? 1.0 - da : 0.0;
  double vol = slab_volume(m, al, ax, xs, da);
  return dgt0(a) ? vol : -vol;
}

// energy flux G = T_f (C_pl F + C_pg (a - F)) with T_f = WENO5 of the
// upwind-ordered stencil (out of line: only faces next to non-no-op cells)
__device__ __noinline__ double face_energy_flux(double Cp_l, double Cp_g, double Fv, double a, double t0, double t1,
                                                double t2, double t3, double t4) {
  const double Tf = weno5(t0, t1, t2, t3, t4);
  return (Tf * Cp_l) * Fv + (Tf * Cp_g) * (a - Fv);
}

// energy flux of a face from its upwind-ordered temperature stencil
__device__ __forceinline__ double energy_flux(const GridDev& g, double Fv, double a, double t0, double t1, double t2,
                                              double t3, double t4) {
  double Tf = weno5(t0, t1, t2, t3, t4);
  return (Tf * g.Cp_l) * Fv + (Tf * g.Cp_g) * (a - Fv);
}

// WY update of one cell from its two faces; returns the clipped volume
template <bool ENERGY>
__device__ __forceinline__ double update_cell(const GridDev& g, size_t id, double c, double e, double T, uint8_t stv,
                                              double Fl, double Gl, double al, double Fr, double Gr, double ar,
                                              double* __restrict__ c_out, double* __restrict__ e_out,
                                              uint8_t* __restrict__ state, double* __restrict__ theta) {
  const bool dirty = stv & 1;
  const double ccv = dirty ? (double)((stv >> 1) & 1) : (dgthalf(c) ? 1.0 : 0.0);
  const double lf = Fl - ccv * al, rf = Fr - ccv * ar;
  const double cn = (c + lf) - rf;
  double cc2 = cn, clip = 0.0;
  if (dlt0(cn)) { cc2 = 0.0; clip = cn; }
  else if (dgt1(cn)) { cc2 = 1.0; clip = cn - 1.0; }
  c_out[id] = cc2;
  if (ENERGY) {
    const double th = dirty ? theta[id] : heat_cap(g.Cp_l, g.Cp_g, ccv) * T;
    const double le = Gl - th * al, re = Gr - th * ar;
    const double en = (e + le) - re;
    e_out[id] = en;
    if (state && !dirty && (!deq(cc2, c) || !deq(en, e))) {
      state[id] = (uint8_t)(1 | (ccv > 0.5 ? 2 : 0));
      theta[id] = th;
    }
  }
  return clip;
}

template <int NV>
__device__ __forceinline__ void block_reduce_out(double (&v)[NV], SumOut out) {
  __shared__ double red[NV][8];  // up to 8 warps per CTA (256 threads)
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nwarps = (int)(blockDim.x * blockDim.y * blockDim.z) >> 5;
  const int lane = tid & 31, warp = tid >> 5;
  const int block_lin = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    // whole warps of zeros (the common case) skip the FP64 shuffle tree
    if (__any_sync(kFull, dnz(x))) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    } else {
      x = 0.0;
    }
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[k][w];
      if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = s;
      else if (out.diag && dnz(s)) atomicAdd(out.diag + k, s);
    }
  }
}

// Tile sweep: one thread per cell.  A CTA stages c and e of its tile plus a
// halo of 4 cells along the sweep axis (no transverse halo: the 27-cell MYC
// stencil of a mixed donor is read from global memory, which only the few
// interface faces need).  Phases, separated by barriers:
//   1. no-op flags of the tile cells and of the first halo cell on each side
//      (7-cell window along the axis has equal (c, e) bits, c is 0 or 1, the
//      cell has not changed earlier in the step);
//   2. T = e / C_p(c) only for cells within 3 of a non-no-op cell;
//   3. face fluxes only for faces next to a non-no-op cell;
//   4. cell updates; no-op cells are copied.
template <int AX>
struct TileShape;
template <>
struct TileShape<0> { static constexpr int X = 64, Y = 4, Z = 1; };
template <>
struct TileShape<1> { static constexpr int X = 16, Y = 16, Z = 1; };
template <>
struct TileShape<2> { static constexpr int X = 16, Y = 1, Z = 16; };

constexpr int kHalo = 4;
static_assert(TileShape<0>::X * TileShape<0>::Y * TileShape<0>::Z == 256, "256 threads per sweep CTA");
static_assert(TileShape<1>::X * TileShape<1>::Y * TileShape<1>::Z == 256, "256 threads per sweep CTA");
static_assert(TileShape<2>::X * TileShape<2>::Y * TileShape<2>::Z == 256, "256 threads per sweep CTA");

template <int AX, bool ENERGY>
__global__ void __launch_bounds__(256, 3)
k_sweep_tile(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
             double* __restrict__ e_out, const double* __restrict__ uf, uint8_t* __restrict__ state,
             double* __restrict__ theta, double* __restrict__ flux_out, SumOut sums, int* __restrict__ status) {
  constexpr int TX = TileShape<AX>::X, TY = TileShape<AX>::Y, TZ = TileShape<AX>::Z;
  constexpr int TA = AX == 0 ? TX : (AX == 1 ? TY : TZ);  // tile length along the axis
  constexpr int TT = (TX * TY * TZ) / TA;                  // transverse cells of the tile
  constexpr int HL = TA + 2 * kHalo;                       // staged length along the axis
  constexpr int NH = HL * TT;
  constexpr int NFL = TA + 1;                              // faces per line
  constexpr int NF = NFL * TT;
  constexpr int FL = TA + 2;                               // flagged positions per line: -1 .. TA
  __shared__ double sc[NH];
  __shared__ double se[ENERGY ? NH : 1];
  __shared__ double sT[ENERGY ? NH : 1];
  __shared__ uint8_t snoop[FL * TT];
  __shared__ double sF[NF];
  __shared__ double sG[ENERGY ? NF : 1];
  __shared__ double sA[NF];

  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int n_ax = g.n[AX];
  const int bca = g.bc[AX];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int a0 = AX == 0 ? x0 : (AX == 1 ? y0 : z0);
  const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
  // transverse line index t in [0, TT) <-> (tile coords of the two other axes)
  auto line_coords = [&](int t, int pos, int& gx, int& gy, int& gz) {
    if (AX == 0) { gx = x0 + pos; gy = y0 + t % TY; gz = z0 + t / TY; }
    else if (AX == 1) { gx = x0 + t % TX; gy = y0 + pos; gz = z0 + t / TX; }
    else { gx = x0 + t % TX; gy = y0 + t / TX; gz = z0 + pos; }
  };
  auto line_ok = [&](int t) {
    int gx, gy, gz;
    line_coords(t, 0, gx, gy, gz);
    return (AX == 0 || gx < nx) && (AX == 1 || gy < ny) && (AX == 2 || gz < nz);
  };
  // staged index of (line t, position p in [-kHalo, TA + kHalo)) -- lines are
  // contiguous along the axis for AX = 0 and interleaved otherwise so that a
  // warp's loads stay coalesced along x
  auto hidx = [&](int t, int p) { return AX == 0 ? t * HL + (p + kHalo) : (p + kHalo) * TT + t; };

  // 1. stage c, e
  for (int q = tid; q < NH; q += 256) {
    int t, p;
    if (AX == 0) { t = q / HL; p = q % HL - kHalo; }
    else { p = q / TT - kHalo; t = q % TT; }
    int gx, gy, gz;
    line_coords(t, p, gx, gy, gz);
    const int xx = map_idx(gx, nx, g.bc[0]), yy = map_idx(gy, ny, g.bc[1]), zz = map_idx(gz, nz, g.bc[2]);
    const size_t id = ((size_t)zz * ny + yy) * nx + xx;
    sc[q] = __ldg(c_in + id);
    if (ENERGY) se[q] = __ldg(e_in + id);
  }
  __syncthreads();
  // 2. no-op flags of positions -1 .. TA
  for (int q = tid; q < FL * TT; q += 256) {
    const int t = q / FL, p = q % FL - 1;
    int gx, gy, gz;
    line_coords(t, p, gx, gy, gz);
    const int ga = a0 + p;
    bool noop;
    if (!line_ok(t) || (bca != 0 && (ga < 0 || ga >= n_ax))) {
      noop = true;  // not a cell of the grid: needs no face
    } else {
      const int h0 = hidx(t, p);
      const double c0 = sc[h0];
      noop = is01(c0);
      if (noop) {
#pragma unroll
        for (int d = -3; d <= 3; ++d) {
          const int hd = hidx(t, p + d);
          noop = noop && same_bits(sc[hd], c0) && (!ENERGY || same_bits(se[hd], se[h0]));
        }
      }
      if (noop && state) {
        const int xx = map_idx(gx, nx, g.bc[0]), yy = map_idx(gy, ny, g.bc[1]), zz = map_idx(gz, nz, g.bc[2]);
        noop = !(state[((size_t)zz * ny + yy) * nx + xx] & 1);
      }
    }
    snoop[q] = noop ? 1 : 0;
  }
  __syncthreads();
  // 3. T where some cell within 3 positions is not a no-op
  if (ENERGY) {
    for (int q = tid; q < NH; q += 256) {
      int t, p;
      if (AX == 0) { t = q / HL; p = q % HL - kHalo; }
      else { p = q / TT - kHalo; t = q % TT; }
      bool need = false;
#pragma unroll
      for (int d = -3; d <= 3; ++d) {
        const int pp = p + d;
        if (pp >= -1 && pp <= TA) need = need || !snoop[t * FL + pp + 1];
      }
      if (need) sT[q] = se[q] / heat_cap(g.Cp_l, g.Cp_g, sc[q]);
    }
  }
  __syncthreads();
  // 4. faces f = 0..TA of each line (face f between positions f-1 and f)
  for (int q = tid; q < NF; q += 256) {
    const int t = q / NFL, f = q % NFL;
    double Fv = 0.0, Gv = 0.0, a = 0.0;
    const int gfa = a0 + f;
    const bool need = line_ok(t) && gfa <= n_ax && (flux_out || !snoop[t * FL + f] || !snoop[t * FL + f + 1]);
    if (need) {
      int gx, gy, gz;
      line_coords(t, f, gx, gy, gz);
      const int fr = (bca == 0 && gfa == n_ax) ? 0 : gfa;
      size_t fid;
      if (AX == 0) fid = ((size_t)gz * ny + gy) * (nx + 1) + fr;
      else if (AX == 1) fid = ((size_t)gz * (ny + 1) + fr) * nx + gx;
      else fid = ((size_t)fr * ny + gy) * nx + gx;
      a = __ldg(uf + fid) * g.lam;
      if (dnz(a)) {
        const bool pos = dgt0(a);
        const int pd = pos ? f - 1 : f;  // donor position
        const double cd = sc[hidx(t, pd)];
        if (is_mixed_b(cd, g)) {
          int dx, dy, dz;
          line_coords(t, pd, dx, dy, dz);
          Fv = mixed_donor_flux(g, c_in, AX, map_idx(dx, nx, g.bc[0]), map_idx(dy, ny, g.bc[1]),
                                map_idx(dz, nz, g.bc[2]), cd, a, status);
        } else {
          Fv = cd * a;
        }
        if (ENERGY) {
          double v[5];
#pragma unroll
          for (int r = -2; r <= 2; ++r) v[r + 2] = sT[hidx(t, pd + (pos ? r : -r))];
          Gv = face_energy_flux(g.Cp_l, g.Cp_g, Fv, a, v[0], v[1], v[2], v[3], v[4]);
        }
      }
      if (flux_out && (f < TA || gfa == n_ax)) {
        size_t fo;
        if (AX == 0) fo = ((size_t)gz * ny + gy) * (nx + 1) + gfa;
        else if (AX == 1) fo = ((size_t)gz * (ny + 1) + gfa) * nx + gx;
        else fo = ((size_t)gfa * ny + gy) * nx + gx;
        flux_out[fo] = Fv;
      }
    }
    sF[q] = Fv;
    sA[q] = a;
    if (ENERGY) sG[q] = Gv;
  }
  __syncthreads();
  // 5. cells
  double clip = 0.0;
  {
    const int lx = threadIdx.x, ly = threadIdx.y, lz = threadIdx.z;
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx < nx && gy < ny && gz < nz) {
      const int p = AX == 0 ? lx : (AX == 1 ? ly : lz);
      const int t = AX == 0 ? ly + TY * lz : (AX == 1 ? lx + TX * lz : lx + TX * ly);
      const size_t id = ((size_t)gz * ny + gy) * nx + gx;
      const int h = hidx(t, p);
      const double c = sc[h];
      const double e = ENERGY ? se[h] : 0.0;
      if (snoop[t * FL + p + 1]) {
        c_out[id] = c;
        if (ENERGY) e_out[id] = e;
      } else {
        const int qa = t * NFL + p, qb = qa + 1;
        const uint8_t stv = state ? state[id] : (uint8_t)0;
        clip = update_cell<ENERGY>(g, id, c, e, ENERGY ? sT[h] : 0.0, stv, sF[qa], ENERGY ? sG[qa] : 0.0, sA[qa],
                                   sF[qb], ENERGY ? sG[qb] : 0.0, sA[qb], c_out, e_out, state, theta);
      }
    }
  }
  double v[1] = {clip};
  block_reduce_out<1>(v, sums);
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

template <int AX>
static dim3 tile_grid(const GridDev& g) {
  using S = TileShape<AX>;
  return dim3((g.n[0] + S::X - 1) / S::X, (g.n[1] + S::Y - 1) / S::Y, (g.n[2] + S::Z - 1) / S::Z);
}

template <int AX>
static dim3 tile_block() {
  return dim3(TileShape<AX>::X, TileShape<AX>::Y, TileShape<AX>::Z);
}

int sweep_blocks(int axis, const GridDev& g) {
  dim3 gr = axis == 0 ? tile_grid<0>(g) : (axis == 1 ? tile_grid<1>(g) : tile_grid<2>(g));
  return (int)(gr.x * gr.y * gr.z);
}

template <int AX>
static void launch_tile(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                        const double* uf, uint8_t* state, double* theta, double* flux_out, SumOut sums,
                        int* status, cudaStream_t st) {
  if (e_in)
    k_sweep_tile<AX, true><<<tile_grid<AX>(g), tile_block<AX>(), 0, st>>>(g, c_in, e_in, c_out, e_out, uf, state,
                                                                           theta, flux_out, sums, status);
  else
    k_sweep_tile<AX, false><<<tile_grid<AX>(g), tile_block<AX>(), 0, st>>>(g, c_in, nullptr, c_out, nullptr, uf,
                                                                            state, theta, flux_out, sums, status);
}

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SumOut sums, cudaStream_t st) {
  int* status = device_status_ptr();
  if (axis == 0) launch_tile<0>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, status, st);
  else if (axis == 1) launch_tile<1>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, status, st);
  else launch_tile<2>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums, status, st);
  return cudaGetLastError();
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
