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

// ---------------------------------------------------------------------------
// Marching sweeps.  A thread (sweeps along y and z) or a warp (sweep along x)
// walks along the sweep axis through a segment of one grid line, holding a
// window of 8 cells (c, e, T) in registers.  A cell is a no-op -- its c and e
// come out bit-identical -- when the 7 cells around it along the axis have
// the same (c, e) bits, c is exactly 0 or 1 and the cell has not changed
// earlier in the step (then both donors are pure with the same c, F = c a,
// both face temperatures are T, and (G - Theta a) vanishes exactly on both
// faces).  No-op cells cost no FP64 work; face fluxes are evaluated only
// where an adjacent cell is not a no-op; T = e / C_p(c) is divided only where
// (c, e) differs from the previous cell of the line.
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

// energy flux of a face from its upwind-ordered temperature stencil (kept
// out of line: it runs only on faces next to non-trivial cells)
__device__ __noinline__ double energy_flux(const GridDev& g, double Fv, double a, double t0, double t1, double t2,
                                              double t3, double t4) {
  double Tf = weno5(t0, t1, t2, t3, t4);
  return (Tf * g.Cp_l) * Fv + (Tf * g.Cp_g) * (a - Fv);
}

// WY update of one cell from its two faces; returns the clipped volume
template <bool ENERGY>
__device__ __noinline__ double update_cell(const GridDev& g, size_t id, double c, double e, double T, uint8_t stv,
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
  __shared__ double red[NV][8];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
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
      for (int w = 0; w < 8; ++w) s += red[k][w];
      if (out.partials) out.partials[(size_t)block_lin * out.stride + k] = s;
      else if (out.diag && dnz(s)) atomicAdd(out.diag + k, s);
    }
  }
}

constexpr int kSegCol = 32;   // cells per thread along y / z
constexpr int kSegRow = 256;  // cells per warp along x (multiple of 32)

// Sweep along y (AX = 1) or z (AX = 2): block = 32 lanes along x x 8 warps
// along the remaining axis; each thread walks kSegCol cells of its line.
// While face k is processed the window holds c, e of cells k-1..k+3
// (wc[0..4]) and T of cells k-3..k+3 (wT[0..6]).
template <int AX, bool ENERGY>
__global__ void __launch_bounds__(256, 2)
k_sweep_col(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
            double* __restrict__ e_out, const double* __restrict__ uf, uint8_t* __restrict__ state,
            double* __restrict__ theta, double* __restrict__ flux_out, SumOut sums, int* __restrict__ status) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int n_ax = AX == 1 ? ny : nz;
  const int n_t = AX == 1 ? nz : ny;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int t = blockIdx.y * 8 + threadIdx.y;
  const int s0 = blockIdx.z * kSegCol;
  const int s1 = min(s0 + kSegCol, n_ax);
  const bool act = (x < nx) && (t < n_t);
  const int bca = g.bc[AX];
  double clip = 0.0;
  if (act) {
    const size_t stride = AX == 1 ? (size_t)nx : (size_t)nx * ny;
    const size_t cbase = AX == 1 ? (size_t)t * ny * nx + x : (size_t)t * nx + x;
    const size_t fstride = stride;
    const size_t fbase = AX == 1 ? (size_t)t * (ny + 1) * nx + x : (size_t)t * nx + x;
    double wc[5], we[5], wT[7];
    int run = 0;
    double pc = 0.0, pe = 0.0, pT = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const size_t id = cbase + stride * map_idx(s0 - 4 + i, n_ax, bca);
      const double cv = __ldg(c_in + id);
      const double ev = ENERGY ? __ldg(e_in + id) : 0.0;
      const bool same = i > 0 && same_bits(cv, pc) && (!ENERGY || same_bits(ev, pe));
      const double Tv = ENERGY ? (same ? pT : ev / heat_cap(g.Cp_l, g.Cp_g, cv)) : 0.0;
      if (i >= 3) { wc[i - 3] = cv; we[i - 3] = ev; }
      if (i >= 1) wT[i - 1] = Tv;
      run = same ? run + 1 : 1;
      pc = cv; pe = ev; pT = Tv;
    }
    double Fp = 0.0, Gp = 0.0, ap = 0.0;
    bool noop_prev = true;
    uint8_t st_prev = 0;
    double nc, ne = 0.0;
    {
      const size_t id = cbase + stride * map_idx(s0 + 4, n_ax, bca);
      nc = __ldg(c_in + id);
      if (ENERGY) ne = __ldg(e_in + id);
    }
    double nu = __ldg(uf + fbase + fstride * ((bca == 0 && s0 == n_ax) ? 0 : s0));
    uint8_t nst = (state && s0 < s1) ? state[cbase + stride * s0] : (uint8_t)0;
    for (int k = s0; k <= s1; ++k) {
      const bool inner = k < s1;
      const double a = nu * g.lam;
      const uint8_t st_cur = nst;
      const double tc = nc, te = ne;
      if (inner) {
        const size_t id = cbase + stride * map_idx(k + 5, n_ax, bca);
        nc = __ldg(c_in + id);
        if (ENERGY) ne = __ldg(e_in + id);
        const int f1 = k + 1;
        nu = __ldg(uf + fbase + fstride * ((bca == 0 && f1 == n_ax) ? 0 : f1));
        nst = (state && k + 1 < s1) ? state[cbase + stride * (k + 1)] : (uint8_t)0;
      }
      // cell k is a no-op when cells k-3..k+3 agree, c_k is 0 or 1 and the
      // cell is still clean
      const bool noop_cur = inner && run >= 7 && is01(wc[1]) && !(st_cur & 1);
      const bool need = flux_out || (k > s0 && !noop_prev) || (inner && !noop_cur);
      double F = 0.0, G = 0.0;
      if (need && dnz(a)) {
        const bool pos = dgt0(a);
        const double cd = pos ? wc[0] : wc[1];
        if (is_mixed_b(cd, g)) {
          const int ds = map_idx(pos ? k - 1 : k, n_ax, bca);
          F = mixed_donor_flux(g, c_in, AX, x, AX == 1 ? ds : t, AX == 2 ? ds : t, cd, a, status);
        } else {
          F = cd * a;
        }
        if (ENERGY) {
          G = pos ? energy_flux(g, F, a, wT[0], wT[1], wT[2], wT[3], wT[4])
                  : energy_flux(g, F, a, wT[5], wT[4], wT[3], wT[2], wT[1]);
        }
      }
      if (flux_out && (inner || k == n_ax)) flux_out[fbase + fstride * k] = F;
      if (k > s0) {
        const size_t id = cbase + stride * (k - 1);
        if (noop_prev) {
          c_out[id] = wc[0];
          if (ENERGY) e_out[id] = we[0];
        } else {
          clip += update_cell<ENERGY>(g, id, wc[0], we[0], wT[2], st_prev, Fp, Gp, ap, F, G, a, c_out, e_out, state,
                                      theta);
        }
      }
      Fp = F; Gp = G; ap = a;
      noop_prev = noop_cur;
      st_prev = st_cur;
      if (inner) {
        // shift the window and append cell k + 4
        const bool same = same_bits(tc, wc[4]) && (!ENERGY || same_bits(te, we[4]));
        const double tT = ENERGY ? (same ? wT[6] : te / heat_cap(g.Cp_l, g.Cp_g, tc)) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) { wc[i] = wc[i + 1]; we[i] = we[i + 1]; }
#pragma unroll
        for (int i = 0; i < 6; ++i) wT[i] = wT[i + 1];
        wc[4] = tc; we[4] = te; wT[6] = tT;
        run = same ? run + 1 : 1;
      }
    }
  }
  double v[1] = {clip};
  block_reduce_out<1>(v, sums);
}

// value at lane + d (d in [-4, 4]) of the concatenated chunks P | C | N
__device__ __forceinline__ double lane_get(double vP, double vC, double vN, int lane, int d) {
  const int idx = lane + d;
  const int src = idx & 31;
  const double a = __shfl_sync(kFull, vP, src);
  const double b = __shfl_sync(kFull, vC, src);
  const double c = __shfl_sync(kFull, vN, src);
  return idx < 0 ? a : (idx < 32 ? b : c);
}

// Sweep along x: each warp walks a row segment of kSegRow cells in chunks of
// 32 (lane = cell), neighbours across lanes by shuffles and ballot masks.
template <bool ENERGY>
__global__ void __launch_bounds__(256, 2)
k_sweep_row(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
            double* __restrict__ e_out, const double* __restrict__ uf, uint8_t* __restrict__ state,
            double* __restrict__ theta, double* __restrict__ flux_out, SumOut sums, int* __restrict__ status) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int lane = threadIdx.x;
  const int row = blockIdx.y * 8 + threadIdx.y;  // row = z * ny + y
  const int x0 = blockIdx.x * kSegRow;
  const int x1 = min(x0 + kSegRow, nx);
  const bool rowok = row < ny * nz;
  const int ry = rowok ? row % ny : 0, rz = rowok ? row / ny : 0;
  const size_t rbase = ((size_t)rz * ny + ry) * nx;
  const size_t fbase = ((size_t)rz * ny + ry) * (nx + 1);
  const int bcx = g.bc[0];
  double clip = 0.0;
  if (rowok) {
    auto ldc = [&](int X) { return __ldg(c_in + rbase + map_idx(X, nx, bcx)); };
    auto lde = [&](int X) { return ENERGY ? __ldg(e_in + rbase + map_idx(X, nx, bcx)) : 0.0; };
    auto ldst = [&](int X) -> uint8_t { return (state && X >= x0 && X < x1) ? state[rbase + X] : (uint8_t)0; };
    // chunks: P = cells base-32.., C = base.., N = base+32..; start with C = chunk -1
    int base = x0 - 32;
    double cP = ldc(base - 32 + lane), eP = lde(base - 32 + lane);
    double cC = ldc(base + lane), eC = lde(base + lane);
    double cN = ldc(base + 32 + lane), eN = lde(base + 32 + lane);
    uint8_t sC = ldst(base + lane), sN = ldst(base + 32 + lane);
    auto eqmask = [&](double cprev_last, double eprev_last, double cc, double ee) -> unsigned {
      double cl = __shfl_up_sync(kFull, cc, 1), el = __shfl_up_sync(kFull, ee, 1);
      if (lane == 0) { cl = cprev_last; el = eprev_last; }
      return __ballot_sync(kFull, same_bits(cc, cl) && (!ENERGY || same_bits(ee, el)));
    };
    unsigned eqP = eqmask(cP, eP, cP, eP);  // lane-0 bit of the first chunk is never used
    unsigned eqC = eqmask(__shfl_sync(kFull, cP, 31), __shfl_sync(kFull, eP, 31), cC, eC);
    unsigned eqN = eqmask(__shfl_sync(kFull, cC, 31), __shfl_sync(kFull, eC, 31), cN, eN);
    // carried right face of the previous chunk's lane 31
    double Fc = 0.0, Gc = 0.0, ac = 0.0;
    for (; base < x1; base += 32) {
      // prefetch chunk N+1
      const int bn = base + 64;
      const double cNN = ldc(bn + lane), eNN = lde(bn + lane);
      const uint8_t sNN = ldst(bn + lane);
      const int f = base + lane + 1;  // right face of this lane's cell
      const bool fok = f >= x0 && f <= x1;
      const double u = fok ? __ldg(uf + fbase + ((bcx == 0 && f == nx) ? 0 : f)) : 0.0;
      const double a = u * g.lam;
      const bool cell_ok = base + lane >= x0 && base + lane < x1;
      // no-op masks: uniform over [l-3, l+3] needs eq bits at l-2..l+3
      const unsigned long long M1 = ((unsigned long long)eqC << 32) | eqP;
      const unsigned long long M2 = ((unsigned long long)eqN << 32) | eqC;
      const bool uni = lane >= 2 ? (((M2 >> (lane - 2)) & 0x3Full) == 0x3Full)
                                 : (((M1 >> (32 + lane - 2)) & 0x3Full) == 0x3Full);
      const bool noopC = uni && is01(cC) && !(sC & 1);
      const bool uniN0 = ((M2 >> 30) & 0x3Full) == 0x3Full;
      const double cN0 = __shfl_sync(kFull, cN, 0);
      const uint8_t sN0 = (uint8_t)__shfl_sync(kFull, (int)sN, 0);
      const bool noopN0 = uniN0 && is01(cN0) && !(sN0 & 1);
      const int noop_next = __shfl_down_sync(kFull, (int)noopC, 1);  // every lane takes part
      const bool noopR = lane < 31 ? (bool)noop_next : noopN0;
      // right face needed by this cell (inside the segment) or the next one
      const bool next_ok = f < x1;
      const bool need = fok && (flux_out || (cell_ok && !noopC) || (next_ok && !noopR));
      double F = 0.0, G = 0.0;
      const unsigned needm = __ballot_sync(kFull, need && dnz(a));
      if (needm) {
        double TP = 0.0, TC = 0.0, TN = 0.0;
        if (ENERGY) {
          TP = eP / heat_cap(g.Cp_l, g.Cp_g, cP);
          TC = eC / heat_cap(g.Cp_l, g.Cp_g, cC);
          TN = eN / heat_cap(g.Cp_l, g.Cp_g, cN);
        }
        const double cR = lane_get(cP, cC, cN, lane, 1);
        double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0;
        const bool pos = dgt0(a);
        if (ENERGY) {
          const double Tm2 = lane_get(TP, TC, TN, lane, -2), Tm1 = lane_get(TP, TC, TN, lane, -1);
          const double T1 = lane_get(TP, TC, TN, lane, 1), T2 = lane_get(TP, TC, TN, lane, 2);
          const double T3 = lane_get(TP, TC, TN, lane, 3);
          if (pos) { t0 = Tm2; t1 = Tm1; t2 = TC; t3 = T1; t4 = T2; }
          else { t0 = T3; t1 = T2; t2 = T1; t3 = TC; t4 = Tm1; }
        }
        if ((needm >> lane) & 1u) {
          const double cd = pos ? cC : cR;
          if (is_mixed_b(cd, g)) {
            const int dx = pos ? base + lane : base + lane + 1;
            F = mixed_donor_flux(g, c_in, 0, map_idx(dx, nx, bcx), ry, rz, cd, a, status);
          } else {
            F = cd * a;
          }
          if (ENERGY) G = energy_flux(g, F, a, t0, t1, t2, t3, t4);
        }
      }
      if (flux_out && fok && (f < x1 || f == nx)) flux_out[fbase + f] = F;
      // left face = right face of the lane to the left (lane 0: carried)
      double Fl = __shfl_up_sync(kFull, F, 1), Gl = __shfl_up_sync(kFull, G, 1), al = __shfl_up_sync(kFull, a, 1);
      if (lane == 0) { Fl = Fc; Gl = Gc; al = ac; }
      Fc = __shfl_sync(kFull, F, 31); Gc = __shfl_sync(kFull, G, 31); ac = __shfl_sync(kFull, a, 31);
      if (cell_ok) {
        const size_t id = rbase + base + lane;
        if (noopC) {
          c_out[id] = cC;
          if (ENERGY) e_out[id] = eC;
        } else {
          const double TC = ENERGY ? eC / heat_cap(g.Cp_l, g.Cp_g, cC) : 0.0;
          clip += update_cell<ENERGY>(g, id, cC, eC, TC, sC, Fl, Gl, al, F, G, a, c_out, e_out, state, theta);
        }
      }
      // rotate chunks
      const double c31 = __shfl_sync(kFull, cN, 31), e31 = __shfl_sync(kFull, eN, 31);
      const unsigned eqNN = eqmask(c31, e31, cNN, eNN);
      cP = cC; eP = eC;
      cC = cN; eC = eN; sC = sN;
      cN = cNN; eN = eNN; sN = sNN;
      eqP = eqC; eqC = eqN; eqN = eqNN;
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

static dim3 col_grid(int axis, const GridDev& g) {
  const int n_ax = g.n[axis], n_t = axis == 1 ? g.n[2] : g.n[1];
  return dim3((g.n[0] + 31) / 32, (n_t + 7) / 8, (n_ax + kSegCol - 1) / kSegCol);
}

static dim3 row_grid(const GridDev& g) {
  return dim3((g.n[0] + kSegRow - 1) / kSegRow, (g.n[1] * g.n[2] + 7) / 8, 1);
}

int sweep_blocks(int axis, const GridDev& g) {
  dim3 gr = axis == 0 ? row_grid(g) : col_grid(axis, g);
  return (int)(gr.x * gr.y * gr.z);
}

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SumOut sums, cudaStream_t st) {
  int* status = device_status_ptr();
  const dim3 blk(32, 8);
  if (axis == 0) {
    if (e_in)
      k_sweep_row<true><<<row_grid(g), blk, 0, st>>>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sums,
                                                      status);
    else
      k_sweep_row<false><<<row_grid(g), blk, 0, st>>>(g, c_in, nullptr, c_out, nullptr, uf, state, theta, flux_out,
                                                       sums, status);
  } else if (axis == 1) {
    if (e_in)
      k_sweep_col<1, true><<<col_grid(1, g), blk, 0, st>>>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out,
                                                            sums, status);
    else
      k_sweep_col<1, false><<<col_grid(1, g), blk, 0, st>>>(g, c_in, nullptr, c_out, nullptr, uf, state, theta,
                                                             flux_out, sums, status);
  } else {
    if (e_in)
      k_sweep_col<2, true><<<col_grid(2, g), blk, 0, st>>>(g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out,
                                                            sums, status);
    else
      k_sweep_col<2, false><<<col_grid(2, g), blk, 0, st>>>(g, c_in, nullptr, c_out, nullptr, uf, state, theta,
                                                             flux_out, sums, status);
  }
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
