// vof_sweep.cu -- direction-split geometric VOF sweep with the thermal
// energy fluxed in tandem (Malan et al., arXiv:2001.03477, Sec. 3.3.1 Step 1
// with the Weymouth-Yue split scheme, and Sec. 3.4.1 Eq. disc_et_adv), plus
// the unfused energy update from exported VOF fluxes.
//
// Every cell applies
//   c <- c + (F_l - cc a_l) - (F_r - cc a_r)
//   e <- e + (G_l - Theta a_l) - (G_r - Theta a_r),
//   G = (T_f C_pl) F + (T_f C_pg) (a - F),  T_f = WENO5 of T = e / C_p(c),
// with cc = [c^n > 1/2] and Theta = C_p(cc) T^n frozen at the start of the
// step (see the `state` convention in include/vofgb.h).  With Li's
// Lagrangian-explicit scheme (vof_grid.scheme = VOF_SCHEME_LE, the other
// Step 1 Sec. 3.3.1 names) cc and Theta are the cell's own c and
// (T C_pl) c + (T C_pg)(1 - c) before the sweep, and a mixed donor fluxes
// J times the liquid in the preimage of width |a| / J next to the face,
// J = 1 + (a_r - a_l) its stretch.
//
// Four kernels per sweep:
//   A (stream): walks the grid lines (skipping quiet tiles in an in-place
//     step), copies the cells that provably do not change (no-op cells,
//     below) to the output when out of place, and lists the other cells per
//     warp in a fixed order, plus grid-wide lists of the mixed cells and of
//     the faces to evaluate (left face of every listed cell, right face of
//     every run end);
//   M (prep): the PLIC plane of every mixed cell and T of every listed cell;
//   F (faces): each listed face once: VOF flux (PLIC slab of a mixed donor)
//     and energy flux (WENO5 face temperature);
//   U (update): one warp per kernel-A list, one listed cell per lane: c, e
//     and the frozen state from the two face fluxes.
// The bulk of the grid costs kernel A's streaming pass, and the FP64 work
// (the scarce unit on this part) runs lane-dense over compact lists.
#include "vof_launch.h"
#include "vof_sums.cuh"

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
// (G - Theta a) vanishes exactly on both faces.
// ---------------------------------------------------------------------------

constexpr unsigned kFull = 0xffffffffu;
constexpr long long kOneBits = 0x3FF0000000000000LL;

__device__ __forceinline__ bool same_bits(double a, double b) { return dbits(a) == dbits(b); }
__device__ __forceinline__ bool is01(double c) { long long b = dbits(c); return b == 0 || b == kOneBits; }

__device__ __forceinline__ size_t cell_at(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

// energy flux G = T_f (C_pl F + C_pg (a - F)) with T_f = WENO5 of the
// upwind-ordered stencil
__device__ __forceinline__ double face_energy_flux(double Cp_l, double Cp_g, double Fv, double a, double t0, double t1,
                                                double t2, double t3, double t4, bool f32) {
  const double Tf = f32 ? weno5_f(t0, t1, t2, t3, t4) : weno5_df(t0, t1, t2, t3, t4);
  // one rounding of (T_f C_pl) F, as in the separate product: a pure cell
  // (F = a or 0) still gives (T_f C_pl) a or (T_f C_pg) a exactly
  return fma(Tf * Cp_l, Fv, (Tf * Cp_g) * (a - Fv));
}

// WY update of one cell from its two faces; returns the clipped volume
// LAG: the Lagrangian-explicit form (a compile-time choice, so that the
// Weymouth-Yue kernel carries none of its FP64 arithmetic)
template <bool ENERGY, bool LAG>
__device__ __forceinline__ double update_cell(const GridDev& g, size_t id, double c, double e, double T, uint8_t stv,
                                              double Fl, double Gl, double al, double Fr, double Gr, double ar,
                                              double* __restrict__ c_out, double* __restrict__ e_out,
                                              uint8_t* __restrict__ state, double* __restrict__ theta, double& dc,
                                              double& de) {
  // Lagrangian-explicit sweeps: the dilatation terms use the cell's own
  // c and Theta; no frozen state
  constexpr bool lag = LAG;
  const bool dirty = !lag && (stv & 1);
  const bool ccb = dirty ? ((stv >> 1) & 1) != 0 : dgthalf(c);
  // Weymouth-Yue: cc is 0 or 1, so cc a is a or 0 exactly (no multiply);
  // Lagrangian explicit: the cell's own c
  const double lf = lag ? Fl - c * al : (ccb ? Fl - al : Fl);
  const double rf = lag ? Fr - c * ar : (ccb ? Fr - ar : Fr);
  const double cn = (c + lf) - rf;
  double cc2 = cn, clip = 0.0;
  if (dlt0(cn)) { cc2 = 0.0; clip = cn; }
  else if (dgt1(cn)) { cc2 = 1.0; clip = cn - 1.0; }
  c_out[id] = cc2;
  dc = cc2 - c;
  de = 0.0;
  if (ENERGY) {
    // C_p(cc) with cc in {0, 1} is C_pl or C_pg exactly
    const double th = lag ? (T * g.Cp_l) * c + (T * g.Cp_g) * (1.0 - c)
                         : (dirty ? theta[id] : (ccb ? g.Cp_l : g.Cp_g) * T);
    const double le = Gl - th * al, re = Gr - th * ar;
    const double en = (e + le) - re;
    e_out[id] = en;
    de = en - e;
    if (!lag && state && !dirty && (!deq(cc2, c) || !deq(en, e))) {
      state[id] = (uint8_t)(1 | (ccb ? 2 : 0));
      theta[id] = th;
    }
  }
  return clip;
}

// ---------------------------------------------------------------------------
// Kernel A for the sweeps along y (AX = 1) and z (AX = 2): a warp owns 32
// consecutive x at one position of the remaining axis and walks kSegA cells
// along the sweep axis; each lane keeps a run length of equal (c, e) cells.
// ---------------------------------------------------------------------------
constexpr int kSegA = 32;     // cells per lane along y / z
constexpr int kWarpsA = 8;    // warps per CTA of kernel A
constexpr int kSegRow = 256;  // cells per warp along x (multiple of 32)
constexpr int kPlaneThreads = 128;  // kernel M: CTA size; grid kPlaneCTAs
constexpr int kPlaneCTAs = 152 * 8;

// Staged face entries carry this flag when a cell next to the face is mixed
// (its donor may need the PLIC geometry); kernel A's per-warp cell list
// keeps it too (kernel U masks it off).
constexpr uint32_t kMixedAdj = 0x80000000u;

// Copies n staged entries to the grid-wide face list, flagged ones to the
// back and the others to the front, as face items (cell << 1 | side).
__device__ __forceinline__ void copy_faces(const SweepScratch& sc, const uint32_t* src, int n, uint32_t side, int bf,
                                           int bb, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  for (int j0 = 0; j0 < n; j0 += 32) {  // n is warp-uniform
    const int j = j0 + lane;
    const uint32_t v = j < n ? src[j] : 0u;
    const bool ok = j < n, fl = ok && (v & kMixedAdj);
    const unsigned mf = __ballot_sync(kFull, fl), mo = __ballot_sync(kFull, ok && !fl);
    const uint32_t item = ((v & ~kMixedAdj) << 1) | side;
    if (fl) sc.gface[sc.gface_cap - 1 - (uint32_t)(bb + __popc(mf & lt))] = item;
    else if (ok) sc.gface[bf + __popc(mo & lt)] = item;
    bf += __popc(mo);
    bb += __popc(mf);
  }
}

// Appends a warp's lists (staged in its own slots) to the grid-wide lists:
// its mixed cells to the list of kernel M, and one face item per listed cell
// (its left face) and per run end (the right face of a listed cell whose
// next cell along the axis is not listed) to the list of kernel F -- faces
// next to a mixed cell at its back, so that the warps of kernel F that
// evaluate PLIC slab volumes are few and the others never diverge.  One
// atomic per list and warp reserves the slots; the order of the grid-wide
// lists varies from run to run, and nothing that reads them depends on it.
__device__ __forceinline__ void append_lists(const SweepScratch& sc, const uint32_t* list, int nlist, int nlist_m,
                                             const uint32_t* mlist, int nmixed, const uint32_t* rlist, int nrun,
                                             int nrun_m, int lane) {
  int bm = 0, bf = 0, bb = 0;
  const int nfront = (nlist - nlist_m) + (nrun - nrun_m), nback = nlist_m + nrun_m;
  if (lane == 0) {
    if (nmixed) bm = atomicAdd(sc.counters + 0, nmixed);
    if (nfront) bf = atomicAdd(sc.counters + 1, nfront);
    if (nback) bb = atomicAdd(sc.counters + 2, nback);
  }
  bm = __shfl_sync(kFull, bm, 0);
  bf = __shfl_sync(kFull, bf, 0);
  bb = __shfl_sync(kFull, bb, 0);
  __syncwarp();
  for (int i = lane; i < nmixed; i += 32) sc.gmix[bm + i] = mlist[i];
  copy_faces(sc, list, nlist, 0u, bf, bb, lane);
  copy_faces(sc, rlist, nrun, 1u, bf + (nlist - nlist_m), bb + nlist_m, lane);
}

// i-th face item of the grid-wide list (front part, then the back part)
__device__ __forceinline__ uint32_t face_item(const SweepScratch& sc, int i, int nfront) {
  return i < nfront ? sc.gface[i] : sc.gface[sc.gface_cap - 1 - (uint32_t)(i - nfront)];
}

template <int AX, bool ENERGY>
__device__ __forceinline__ void k_stream_col_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out, double* __restrict__ e_out, const uint8_t* __restrict__ state, const SweepScratch& sc, int force_all, int cap, int copy, const VB vb) {
  const int nx = g.n[0], ny = g.n[1];
  const int n_ax = g.n[AX];
  const int n_t = AX == 1 ? g.n[2] : g.n[1];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = vb.bx * 32 + lane;
  const int t = vb.by * kWarpsA + warp;
  const int s0 = vb.bz * kSegA, s1 = min(s0 + kSegA, n_ax);
  const bool act = x < nx && t < n_t;
  const int xs = act ? x : 0, ts = act ? t : 0;
  const int bca = g.bc[AX];
  const size_t stride = AX == 1 ? (size_t)nx : (size_t)nx * ny;
  const size_t cbase = AX == 1 ? (size_t)ts * ny * nx + xs : (size_t)ts * nx + xs;
  const size_t sub = ((size_t)vb.bz * vb.gy + vb.by) * kWarpsA * vb.gx + (size_t)warp * vb.gx +
                     vb.bx;
  uint32_t* list = sc.list + sub * (size_t)cap;
  uint32_t* mlist = sc.mlist + sub * (size_t)cap;
  uint32_t* rlist = sc.rlist + sub * (size_t)cap;
  const unsigned lt = (1u << lane) - 1u;
  if (sc.tiles.quiet && !force_all) {
    // in place: a warp whose 32 x 32 cells lie in quiet tiles has no work
    // (lanes 0..15 check its 4 x 4 tiles; t is the same for the warp)
    bool q = true;
    const int txi = vb.bx * 4 + (lane & 3), tai = (s0 >> 3) + (lane >> 2);
    if (lane < 16 && txi * kTile < nx && tai * kTile < s1 && t < n_t) {
      const int tt = t >> 3;
      const int ty_ = AX == 1 ? tai : tt, tz_ = AX == 1 ? tt : tai;
      q = sc.tiles.quiet[((size_t)tz_ * sc.tiles.nt[1] + ty_) * sc.tiles.nt[0] + txi] != 0;
    }
    if (__all_sync(kFull, q)) {
      if (lane == 0) sc.count[sub] = 0;
      return;
    }
  }
  int nlist = 0, nmixed = 0, nrun = 0, nlist_m = 0, nrun_m = 0;
  bool prev_listed = false;  // cell k-1 of this segment listed
  double cm1 = 0.0;          // c of cell s0 - 1
  // window: cells k .. k+3 (c, e) and run = equal cells ending at k+3;
  // cells k+4 .. k+7 are in flight (prefetch queue pc/pe)
  double wc[4], we[4], qc[4], qe[4];
  int run = 0;
  double pc = 0.0, pe = 0.0;
#pragma unroll
  for (int i = -4; i < 4; ++i) {
    const size_t id = cbase + stride * map_idx(s0 + i, n_ax, bca);
    const double cv = __ldg(c_in + id);
    const double ev = ENERGY ? __ldg(e_in + id) : 0.0;
    const bool same = i > -4 && same_bits(cv, pc) && (!ENERGY || same_bits(ev, pe));
    run = same ? run + 1 : 1;
    if (i >= 0) { wc[i] = cv; we[i] = ev; }
    if (i == -1) cm1 = cv;
    pc = cv; pe = ev;
  }
  bool prev_mixed = act && is_mixed_b(cm1, g);  // cell k-1 mixed
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const size_t id = cbase + stride * map_idx(s0 + 4 + i, n_ax, bca);
    qc[i] = __ldg(c_in + id);
    qe[i] = ENERGY ? __ldg(e_in + id) : 0.0;
  }
  // frozen-state flags of cells k .. k+3, loaded ahead like c and e (a
  // flag read in the iteration that needs it would put one memory round
  // trip into every step of the walk)
  uint8_t sq[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) sq[i] = (act && state && s0 + i < s1) ? state[cbase + stride * (s0 + i)] : (uint8_t)0;
  for (int k = s0; k < s1; ++k) {
    // cell k + 4 from the queue; cell k + 8 joins it
    const double cn = qc[0], en = qe[0];
    {
      const size_t idq = cbase + stride * map_idx(k + 8, n_ax, bca);
#pragma unroll
      for (int i = 0; i < 3; ++i) { qc[i] = qc[i + 1]; qe[i] = qe[i + 1]; }
      qc[3] = __ldg(c_in + idq);
      qe[3] = ENERGY ? __ldg(e_in + idq) : 0.0;
    }
    const size_t id = cbase + stride * k;
    const uint8_t stv = sq[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) sq[i] = sq[i + 1];
    sq[3] = (act && state && k + 4 < s1) ? state[id + stride * 4] : (uint8_t)0;
    // cells k-3..k+3 equal <=> run (ending at k+3) >= 7
    const bool noop = act && !force_all && run >= 7 && is01(wc[0]) && !(stv & 1);
    if (act && noop && copy) {  // out of place: no-op cells are copied
      c_out[id] = wc[0];
      if (ENERGY) e_out[id] = we[0];
    }
    const bool listed = act && !noop;
    const bool mixed = act && is_mixed_b(wc[0], g);
    const uint32_t madj = (mixed || prev_mixed) ? kMixedAdj : 0u;  // face k
    const unsigned m = __ballot_sync(kFull, listed);
    if (listed) list[nlist + __popc(m & lt)] = (uint32_t)id | madj;
    nlist += __popc(m);
    nlist_m += __popc(__ballot_sync(kFull, listed && madj));
    const unsigned mm = __ballot_sync(kFull, mixed);
    if (mixed) mlist[nmixed + __popc(mm & lt)] = (uint32_t)id;
    nmixed += __popc(mm);
    const bool rend = prev_listed && !listed;  // cell k-1 ends a run (face k)
    const unsigned mr = __ballot_sync(kFull, rend);
    if (rend) rlist[nrun + __popc(mr & lt)] = (uint32_t)(id - stride) | madj;
    nrun += __popc(mr);
    nrun_m += __popc(__ballot_sync(kFull, rend && madj));
    prev_listed = listed;
    prev_mixed = mixed;
    // shift the window
    const bool same = same_bits(cn, wc[3]) && (!ENERGY || same_bits(en, we[3]));
#pragma unroll
    for (int i = 0; i < 3; ++i) { wc[i] = wc[i + 1]; we[i] = we[i + 1]; }
    wc[3] = cn; we[3] = en;
    run = same ? run + 1 : 1;
  }
  // the segment's last cell ends a run unless the next cell along the axis
  // (next segment, or cell 0 across a periodic boundary) is listed; the
  // window now holds cells s1 .. s1+3
  bool next_listed = false;
  if (s1 < n_ax || bca == 0) {
    const size_t idn = cbase + stride * map_idx(s1, n_ax, bca);
    const uint8_t stn = (act && state) ? state[idn] : (uint8_t)0;
    next_listed = act && !(!force_all && run >= 7 && is01(wc[0]) && !(stn & 1));
  }
  const bool rend = prev_listed && !next_listed;
  const uint32_t madj = (prev_mixed || (act && is_mixed_b(wc[0], g))) ? kMixedAdj : 0u;  // face s1
  const unsigned mr = __ballot_sync(kFull, rend);
  if (rend) rlist[nrun + __popc(mr & lt)] = (uint32_t)(cbase + stride * (s1 - 1)) | madj;
  nrun += __popc(mr);
  nrun_m += __popc(__ballot_sync(kFull, rend && madj));
  if (lane == 0) sc.count[sub] = nlist;
  append_lists(sc, list, nlist, nlist_m, mlist, nmixed, rlist, nrun, nrun_m, lane);
}

template <int AX, bool ENERGY>
__global__ void __launch_bounds__(32 * kWarpsA)
k_stream_col(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
             double* __restrict__ e_out, const uint8_t* __restrict__ state, SweepScratch sc, int force_all,
             int cap, int copy) {
  pdl_wait();
  k_stream_col_body<AX, ENERGY>(g, c_in, e_in, c_out, e_out, state, sc, force_all, cap, copy, vb_self());
}

// ---------------------------------------------------------------------------
// Kernel A for the sweep along x: a warp owns kSegRow cells of one row and
// walks them in chunks of 32 (lane = cell); equality with the previous cell
// is a ballot mask, so "cells l-3..l+3 equal" is a 6-bit window test.
// ---------------------------------------------------------------------------
template <bool ENERGY>
__device__ __forceinline__ void k_stream_row_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out, double* __restrict__ e_out, const uint8_t* __restrict__ state, const SweepScratch& sc, int force_all, int cap, int copy, const VB vb) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int row = vb.bx * 8 + warp;  // row = z * ny + y (grid x: rows, grid y: segments)
  const int x0 = vb.by * kSegRow, x1 = min(x0 + kSegRow, nx);
  const bool rowok = row < ny * nz;
  const size_t rbase = (size_t)(rowok ? row : 0) * nx;
  const int bcx = g.bc[0];
  const size_t sub = (size_t)row * vb.gy + vb.by;
  if (!rowok) {  // whole warp: empty list
    if (lane == 0) sc.count[sub] = 0;
    return;
  }
  uint32_t* list = sc.list + sub * (size_t)cap;
  uint32_t* mlist = sc.mlist + sub * (size_t)cap;
  uint32_t* rlist = sc.rlist + sub * (size_t)cap;
  const unsigned lt = (1u << lane) - 1u;
  // quiet tiles of the segment (bit l: its l-th tile)
  unsigned qmask = 0u;
  if (sc.tiles.quiet && !force_all) {
    // in place: a warp whose row segment lies in quiet tiles has no work
    // (lane l checks the l-th tile of the segment)
    bool q = true;
    const int txi = (x0 >> 3) + lane;
    if (txi * kTile < x1) {
      const int y = row % ny, z = row / ny;
      q = sc.tiles.quiet[((size_t)(z >> 3) * sc.tiles.nt[1] + (y >> 3)) * sc.tiles.nt[0] + txi] != 0;
    }
    if (__all_sync(kFull, q)) {
      if (lane == 0) sc.count[sub] = 0;
      return;
    }
    qmask = __ballot_sync(kFull, q);
  }
  int nlist = 0, nmixed = 0, nrun = 0, nlist_m = 0, nrun_m = 0;
  auto ldc = [&](int X) { return __ldg(c_in + rbase + map_idx(X, nx, bcx)); };
  auto lde = [&](int X) { return ENERGY ? __ldg(e_in + rbase + map_idx(X, nx, bcx)) : 0.0; };
  auto eqmask = [&](double cprev, double eprev, double cc, double ee) -> unsigned {
    double cl = __shfl_up_sync(kFull, cc, 1), el = __shfl_up_sync(kFull, ee, 1);
    if (lane == 0) { cl = cprev; el = eprev; }
    return __ballot_sync(kFull, same_bits(cc, cl) && (!ENERGY || same_bits(ee, el)));
  };
  // chunks P (base-32), C (base), N (base+32)
  int base = x0;
  double cP = ldc(base - 32 + lane), eP = lde(base - 32 + lane);
  double cC = ldc(base + lane), eC = lde(base + lane);
  double cN = ldc(base + 32 + lane), eN = lde(base + 32 + lane);
  const double cPP = ldc(base - 33), ePP = lde(base - 33);
  unsigned eqP = eqmask(cPP, ePP, cP, eP);
  unsigned eqC = eqmask(__shfl_sync(kFull, cP, 31), __shfl_sync(kFull, eP, 31), cC, eC);
  unsigned eqN = eqmask(__shfl_sync(kFull, cC, 31), __shfl_sync(kFull, eC, 31), cN, eN);
  bool mixed_carry = is_mixed_b(__shfl_sync(kFull, cP, 31), g);  // cell base - 1 mixed
  // frozen-state flags of the current chunk and of the next, loaded one
  // chunk ahead with c and e (cell X + 1 past the row end wraps on a
  // periodic axis; past a zero-gradient end its flag is not used)
  auto lds_ = [&](int X) { return state ? state[rbase + map_idx(X, nx, bcx)] : (uint8_t)0; };
  uint8_t stC = lds_(base + lane);
  for (; base < x1; base += 32) {
    const double cNN = ldc(base + 64 + lane), eNN = lde(base + 64 + lane);
    const uint8_t stN = lds_(base + 32 + lane);
    if (((qmask >> ((base - x0) >> 3)) & 0xFu) == 0xFu) {
      // a chunk of quiet tiles: no-op cells only, none listed or mixed (the
      // previous chunk's run ends were found looking into this one); the
      // pipeline moves on
      const double c31 = __shfl_sync(kFull, cN, 31), e31 = __shfl_sync(kFull, eN, 31);
      const unsigned eqNN = eqmask(c31, e31, cNN, eNN);
      mixed_carry = false;
      cP = cC; eP = eC;
      cC = cN; eC = eN;
      cN = cNN; eN = eNN;
      eqP = eqC; eqC = eqN; eqN = eqNN;
      stC = stN;
      continue;
    }
    const int X = base + lane;
    const bool cell_ok = X < x1;
    const uint8_t stv = cell_ok ? stC : (uint8_t)0;
    const unsigned long long M1 = ((unsigned long long)eqC << 32) | eqP;
    const unsigned long long M2 = ((unsigned long long)eqN << 32) | eqC;
    // cells X-3..X+3 equal <=> eq bits of X-2..X+3
    const bool uni = lane >= 2 ? (((M2 >> (lane - 2)) & 0x3Full) == 0x3Full)
                               : (((M1 >> (32 + lane - 2)) & 0x3Full) == 0x3Full);
    const bool noop = cell_ok && !force_all && uni && is01(cC) && !(stv & 1);
    if (cell_ok) {
      if (noop && copy) {  // out of place: no-op cells are copied
        c_out[rbase + X] = cC;
        if (ENERGY) e_out[rbase + X] = eC;
      }
    }
    const bool listed = cell_ok && !noop;
    const bool mx_raw = is_mixed_b(cC, g);
    const bool mx_up = __shfl_up_sync(kFull, mx_raw, 1);
    const bool mx_prev = lane == 0 ? mixed_carry : mx_up;  // cell X - 1 mixed
    mixed_carry = __shfl_sync(kFull, mx_raw, 31);
    const uint32_t madj = (mx_raw || mx_prev) ? kMixedAdj : 0u;  // face X
    const unsigned m = __ballot_sync(kFull, listed);
    if (listed) list[nlist + __popc(m & lt)] = (uint32_t)(rbase + X) | madj;
    nlist += __popc(m);
    nlist_m += __popc(__ballot_sync(kFull, listed && madj));
    const bool mixed = cell_ok && mx_raw;
    const unsigned mm = __ballot_sync(kFull, mixed);
    if (mixed) mlist[nmixed + __popc(mm & lt)] = (uint32_t)(rbase + X);
    nmixed += __popc(mm);
    // is cell X+1 listed?  (lane 31: the next chunk's first cell; past the
    // segment end the next segment's first cell, or cell 0 across a
    // periodic boundary; none past a zero-gradient boundary)
    const bool uni_n = lane >= 1 ? (((M2 >> (lane - 1)) & 0x3Full) == 0x3Full) : (((M1 >> 31) & 0x3Full) == 0x3Full);
    const double c_dn = __shfl_down_sync(kFull, cC, 1), c_n0 = __shfl_sync(kFull, cN, 0);
    const double c_next = lane == 31 ? c_n0 : c_dn;
    const int Xn = X + 1;
    const bool in_line = Xn < nx || bcx == 0;
    const uint8_t st_dn = (uint8_t)__shfl_down_sync(kFull, (unsigned)stC, 1);
    const uint8_t st_n0 = (uint8_t)__shfl_sync(kFull, (unsigned)stN, 0);
    const uint8_t stn = (listed && in_line) ? (lane == 31 ? st_n0 : st_dn) : (uint8_t)0;
    const bool next_listed = in_line && !(!force_all && uni_n && is01(c_next) && !(stn & 1));
    const bool rend = listed && !next_listed;
    const uint32_t madj_r = (mx_raw || is_mixed_b(c_next, g)) ? kMixedAdj : 0u;  // face X + 1
    const unsigned mr = __ballot_sync(kFull, rend);
    if (rend) rlist[nrun + __popc(mr & lt)] = (uint32_t)(rbase + X) | madj_r;
    nrun += __popc(mr);
    nrun_m += __popc(__ballot_sync(kFull, rend && madj_r));
    const double c31 = __shfl_sync(kFull, cN, 31), e31 = __shfl_sync(kFull, eN, 31);
    const unsigned eqNN = eqmask(c31, e31, cNN, eNN);
    cP = cC; eP = eC;
    cC = cN; eC = eN;
    cN = cNN; eN = eNN;
    eqP = eqC; eqC = eqN; eqN = eqNN;
    stC = stN;
  }
  if (lane == 0) sc.count[sub] = nlist;
  append_lists(sc, list, nlist, nlist_m, mlist, nmixed, rlist, nrun, nrun_m, lane);
}

template <bool ENERGY>
__global__ void __launch_bounds__(256)
k_stream_row(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
             double* __restrict__ e_out, const uint8_t* __restrict__ state, SweepScratch sc, int force_all,
             int cap, int copy) {
  pdl_wait();
  k_stream_row_body<ENERGY>(g, c_in, e_in, c_out, e_out, state, sc, force_all, cap, copy, vb_self());
}

// ---------------------------------------------------------------------------
// Kernel M: per-cell preparation over the grid-wide lists, one item per
// thread (every lane busy): first the PLIC plane (MYC normal + plane
// constant) of every mixed cell, then T = e / C_p(c) of every listed cell
// (the left-face items of the face list).  The plane items take long and
// are few; the T items fill the machine around them.  Every cell that
// differs from its predecessor along the axis is listed (its 7-cell window
// is not uniform), so after this kernel T is stored for all of those --
// the only T values kernel F reads back -- and for every listed cell, which
// kernel U reads.
// ---------------------------------------------------------------------------
// PLIC plane (MYC normal, plane constant) of the 3x3x3 stencil centred on
// position (qx, qy, qz), each index mapped by the boundary conditions.
// F32: the precision form's FP32 MYC normal (its own instance, so that the
// FP64 form keeps its register budget); YOUNGS: Youngs' normal instead
template <bool F32, bool YOUNGS = false>
__device__ __forceinline__ double4 stencil_plane(const GridDev& g, const double* __restrict__ c_in, int qx, int qy,
                                                 int qz) {
  double s[27];
#pragma unroll
  for (int oz = 0; oz < 3; ++oz) {
    const int zz = map_idx(qz + oz - 1, g.n[2], g.bc[2]);
#pragma unroll
    for (int oy = 0; oy < 3; ++oy) {
      const int yy = map_idx(qy + oy - 1, g.n[1], g.bc[1]);
#pragma unroll
      for (int ox = 0; ox < 3; ++ox) {
        const int xx = map_idx(qx + ox - 1, g.n[0], g.bc[0]);
        s[(oz * 3 + oy) * 3 + ox] = __ldg(c_in + cell_at(g, xx, yy, zz));
      }
    }
  }
  double m[3];
  if (YOUNGS) youngs_normal(s, m);
  else if (F32) myc_normal_f(s, m);
  else myc_normal(s, m);
  double4 pl;
  pl.x = m[0]; pl.y = m[1]; pl.z = m[2];
  pl.w = plane_alpha(m[0], m[1], m[2], s[13]);
  return pl;
}

// Items: the mixed cells (their planes), then with e_in the T items, then,
// on a zero-gradient sweep axis `ax`, the two ends of every line: where the
// end cell is mixed, the plane of the ghost donor beyond it (position -1 or
// n) from the ghost's own 3x3x3 stencil of the boundary-filled field, whose
// cells beyond the boundary are copies of the boundary layer (dc/dn = 0);
// stored in sc.gplane[side][line].
// NRM 1: the mixed cells' normals are already in sc.plane (the learned
// normal with its MYC fallback, vof_mlp.cu); only their plane constants are
// formed here.  NRM 2: Youngs' normal.  Ghost donors keep MYC.
template <bool F32, int NRM>
__device__ __forceinline__ void k_prep_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ e_in, const SweepScratch& sc, int ax, const VB vb) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int nm = sc.counters[0], nf = sc.counters[1];
  const int cnt = nm + (e_in ? nf + sc.counters[2] : 0);
  const int n_ax = g.n[ax];
  const int lines = g.bc[ax] != 0 ? (int)((size_t)nx * ny * nz / (size_t)n_ax) : 0;
  const int total = cnt + 2 * lines;
  for (int i = vb.bx * blockDim.x + threadIdx.x; i < total; i += vb.gx * blockDim.x) {
    if (i >= cnt) {
      const int j = i - cnt;
      const int side = j >= lines ? 1 : 0;
      const int li = j - side * lines;
      // the line's two other coordinates (x fastest)
      int x = 0, y = 0, z = 0;
      if (ax == 0) { y = li % ny; z = li / ny; }
      else if (ax == 1) { x = li % nx; z = li / nx; }
      else { x = li % nx; y = li / nx; }
      const int kend = side ? n_ax - 1 : 0;
      const int ex = ax == 0 ? kend : x, ey = ax == 1 ? kend : y, ez = ax == 2 ? kend : z;
      if (!is_mixed_b(__ldg(c_in + cell_at(g, ex, ey, ez)), g)) continue;
      const int qk = side ? n_ax : -1;
      const double4 pl = stencil_plane<F32>(g, c_in, ax == 0 ? qk : x, ax == 1 ? qk : y, ax == 2 ? qk : z);
      reinterpret_cast<double4*>(sc.gplane)[j] = pl;
      continue;
    }
    if (i >= nm) {
      const uint32_t item = face_item(sc, i - nm, nf);
      if (item & 1u) continue;  // right-face item: its cell has a left item too
      const size_t id = item >> 1;
      sc.T[id] = temp_of(g, __ldg(e_in + id), __ldg(c_in + id));
      continue;
    }
    const size_t id = sc.gmix[i];
    if (NRM == 1) {
      double4* pl = reinterpret_cast<double4*>(sc.plane) + id;
      const double4 m = *pl;
      pl->w = plane_alpha(m.x, m.y, m.z, __ldg(c_in + id));
      continue;
    }
    int x, y, z;
    cell_xyz(g, id, x, y, z);
    reinterpret_cast<double4*>(sc.plane)[id] = stencil_plane<F32, NRM == 2>(g, c_in, x, y, z);
  }
}

template <bool F32, int NRM>
__global__ void __launch_bounds__(kPlaneThreads)
k_prep(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, SweepScratch sc, int ax) {
  pdl_wait();
  k_prep_body<F32, NRM>(g, c_in, e_in, sc, ax, vb_self());
}

// ---------------------------------------------------------------------------
// Kernel F: one face per thread over the grid-wide face list -- the left face
// of every listed cell and the right face of every run end, so each face is
// evaluated once.  VOF flux F (PLIC slab of a mixed donor, c a of a pure
// one) and energy flux G (WENO5 face temperature) go to per-face scratch.
// T comes from kernel M for window cells that differ from their
// predecessor; a cell equal to its predecessor has its predecessor's T.
// ---------------------------------------------------------------------------
constexpr int kFaceThreads = 128;
constexpr int kFaceCTAs = 152 * 8;

template <int AX>
__device__ __forceinline__ size_t face_of(const GridDev& g, int f, int x, int y, int z) {
  if (AX == 0) return ((size_t)z * g.n[1] + y) * (g.n[0] + 1) + f;
  if (AX == 1) return ((size_t)z * (g.n[1] + 1) + f) * g.n[0] + x;
  return ((size_t)f * g.n[1] + y) * g.n[0] + x;
}

template <int AX, bool ENERGY>
__device__ __forceinline__ void k_faces_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ e_in, const double* __restrict__ uf, double* __restrict__ flux_out, const SweepScratch& sc, int* __restrict__ status, const VB vb) {
  const int nx = g.n[0], ny = g.n[1];
  const int n_ax = g.n[AX];
  const int bca = g.bc[AX];
  const int nf = sc.counters[1];
  const int cnt = nf + sc.counters[2];
  const size_t stride = AX == 0 ? 1 : (AX == 1 ? (size_t)nx : (size_t)nx * ny);
  for (int i = vb.bx * blockDim.x + threadIdx.x; i < cnt; i += vb.gx * blockDim.x) {
    const uint32_t item = face_item(sc, i, nf);
    const size_t id = item >> 1;
    const int side = (int)(item & 1u);
    int x, y, z;
    cell_xyz(g, id, x, y, z);
    const int k = AX == 0 ? x : (AX == 1 ? y : z);
    const size_t lbase = id - stride * k;  // cell index of position 0 of this line
    const int f = k + side;                // face between cells f-1 and f
    // (c, e) of cells f-4..f+2 and T of f-3..f+2 (cells that differ from
    // their predecessor read back, others equal to it; the first divided)
    double cw[7], ew[7], Tw[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const size_t jd = lbase + stride * map_idx(f - 4 + j, n_ax, bca);
      cw[j] = __ldg(c_in + jd);
      ew[j] = ENERGY ? __ldg(e_in + jd) : 0.0;
      if (ENERGY && j >= 1) {
        const bool dif = !(same_bits(cw[j], cw[j - 1]) && same_bits(ew[j], ew[j - 1]));
        Tw[j] = dif ? sc.T[jd] : (j == 1 ? temp_of(g, ew[j], cw[j]) : Tw[j - 1]);
      }
    }
    const int fr = (bca == 0 && f == n_ax) ? 0 : f;
    const size_t fid = face_of<AX>(g, fr, x, y, z);
    const double a = __ldg(uf + fid) * g.lam;
    double Fv = 0.0, Gv = 0.0;
    if (dnz(a)) {
      const bool pos = dgt0(a);
      const double cd = pos ? cw[3] : cw[4];  // donor f-1 (a > 0) or f (a < 0)
      if (is_mixed_b(cd, g)) {
        const int dq = pos ? f - 1 : f;  // donor position along the axis
        double4 pl;
        if (bca != 0 && (dq < 0 || dq >= n_ax)) {
          // ghost donor behind a zero-gradient boundary: its own plane (k_prep)
          const size_t lines = (size_t)nx * ny * g.n[2] / (size_t)n_ax;
          const size_t li = AX == 0 ? (size_t)z * ny + y : (AX == 1 ? (size_t)z * nx + x : (size_t)y * nx + x);
          pl = reinterpret_cast<const double4*>(sc.gplane)[(dq < 0 ? 0 : lines) + li];
        } else {
          pl = reinterpret_cast<const double4*>(sc.plane)[lbase + stride * map_idx(dq, n_ax, bca)];
        }
        const double mv[3] = {pl.x, pl.y, pl.z};
        const double da = fabs(a);
        if (da > 1.0 && status) atomicOr(status, DEV_CFL);
        // Weymouth-Yue: the donor slab of width |a|; Lagrangian explicit:
        // the preimage of width |a| / J, J = 1 + (a_r - a_l) of the donor,
        // its liquid stretched by J (the width capped at 1)
        double w = da, J = 1.0;
        if (g.le) {
          const int dk = map_idx(pos ? f - 1 : f, n_ax, bca);
          const int dk1 = (bca == 0 && dk + 1 == n_ax) ? 0 : dk + 1;
          const double adl = __ldg(uf + face_of<AX>(g, dk, x, y, z)) * g.lam;
          const double adr = __ldg(uf + face_of<AX>(g, dk1, x, y, z)) * g.lam;
          J = 1.0 + (adr - adl);
          if (J > da) {
            w = da / J;
          } else {
            w = 1.0;
            if (status) atomicOr(status, DEV_CFL);
          }
        }
        double vol = g.f32 ? slab_volume_f(mv, pl.w, AX, pos ? 1.0 - w : 0.0, w, cd)
                           : slab_volume_nn(mv, pl.w, AX, pos ? 1.0 - w : 0.0, w);
        if (g.le) vol = J * vol;
        Fv = pos ? vol : -vol;
      } else {
        Fv = cd * a;
      }
      if (ENERGY) {
        // upwind-ordered stencil around the donor
        const double t0 = pos ? Tw[1] : Tw[6];
        const double t1 = pos ? Tw[2] : Tw[5];
        const double t2 = pos ? Tw[3] : Tw[4];
        const double t3 = pos ? Tw[4] : Tw[3];
        const double t4 = pos ? Tw[5] : Tw[2];
        Gv = face_energy_flux(g.Cp_l, g.Cp_g, Fv, a, t0, t1, t2, t3, t4, g.f32 != 0);
      }
    }
    sc.F[fid] = Fv;
    if (ENERGY) sc.G[fid] = Gv;
    if (flux_out) {
      // every face of the line, the periodic face n_ax (= face 0) included
      flux_out[face_of<AX>(g, f, x, y, z)] = Fv;
      if (bca == 0 && f == 0) flux_out[face_of<AX>(g, n_ax, x, y, z)] = Fv;
      if (bca == 0 && f == n_ax) flux_out[face_of<AX>(g, 0, x, y, z)] = Fv;
    }
  }
}

template <int AX, bool ENERGY>
__global__ void __launch_bounds__(kFaceThreads)
k_faces(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, const double* __restrict__ uf,
        double* __restrict__ flux_out, SweepScratch sc, int* __restrict__ status) {
  pdl_wait();
  k_faces_body<AX, ENERGY>(g, c_in, e_in, uf, flux_out, sc, status, vb_self());
}

// ---------------------------------------------------------------------------
// Kernel U: each CTA takes `ngrp` groups of kUpdLists consecutive kernel-A lists,
// dealt in turn (a fixed assignment and order, so the sums are
// reproducible), one listed cell per thread:
// the WY update from the two face fluxes.  It reads no cell but its own, so
// it may update in place (c_out == c_in, e_out == e_in); kernel A then
// copies nothing.
// ---------------------------------------------------------------------------
// The groups of lists this CTA takes, cell by cell; v accumulates the
// CTA's contributions to the sums in a fixed order.
template <int AX, bool ENERGY, bool LAG>
__device__ __forceinline__ void update_groups(const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                                              double* e_out, const double* __restrict__ uf,
                                              uint8_t* __restrict__ state, double* __restrict__ theta,
                                              const SweepScratch& sc, int nsub, int cap, int ngrp, const VB vb,
                                              int (&pre)[33], int (&lst)[32], double (&v)[kNSums]) {
  const int n_ax = g.n[AX];
  const int bca = g.bc[AX];
  static_assert(kUpdLists * kUpdBatch == 32, "one list per lane of warp 0");
  for (int grp = 0; grp < ngrp; grp += kUpdBatch) {
    // Groups of kUpdLists consecutive lists are dealt to the CTAs in turn
    // (CTA b takes groups b, b + gx, ...), so the lists of one region of the
    // grid spread over all CTAs whatever the interface's position; the CTA
    // walks kUpdBatch of its groups at a time, their lists in order as one
    // sequence of cells (fixed order): short lists still fill whole warps,
    // and one scan and one barrier serve the batch.
    if ((grp * (int)vb.gx + (int)vb.bx) * kUpdLists >= nsub) break;  // uniform over the CTA
    if (threadIdx.x < 32) {
      // the lists' starts: an inclusive scan of their counts over warp 0
      const int l = threadIdx.x;
      const int gi = grp + l / kUpdLists;
      const int sub = (gi * (int)vb.gx + (int)vb.bx) * kUpdLists + (l % kUpdLists);
      int incl = (gi < ngrp && sub < nsub) ? sc.count[sub] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += t;
      }
      pre[l + 1] = incl;
      lst[l] = sub;
      if (l == 0) pre[0] = 0;
    }
    __syncthreads();
    const int total = pre[32];
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
      // the list of entry j: the last w with pre[w] <= j (pre[0] = 0)
      int w = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (pre[w + step] <= j) w += step;
      const size_t id = sc.list[(size_t)lst[w] * cap + (j - pre[w])] & ~kMixedAdj;
      int x, y, z;
      cell_xyz(g, id, x, y, z);
      const int k = AX == 0 ? x : (AX == 1 ? y : z);
      const int f1 = (bca == 0 && k + 1 == n_ax) ? 0 : k + 1;
      const size_t fl = face_of<AX>(g, k, x, y, z), fr = face_of<AX>(g, f1, x, y, z);
      const double al = __ldg(uf + fl) * g.lam, ar = __ldg(uf + fr) * g.lam;
      const double Fl = sc.F[fl], Fr = sc.F[fr];
      const double Gl = ENERGY ? sc.G[fl] : 0.0, Gr = ENERGY ? sc.G[fr] : 0.0;
      // plain loads: in place, this thread writes the cell afterwards
      const double c = c_in[id];
      const double e = ENERGY ? e_in[id] : 0.0;
      const double T = ENERGY ? sc.T[id] : 0.0;
      const uint8_t stv = state ? state[id] : (uint8_t)0;
      double dc, de;
      v[kSumClip] += update_cell<ENERGY, LAG>(g, id, c, e, T, stv, Fl, Gl, al, Fr, Gr, ar, c_out, e_out, state,
                                              theta, dc, de);
      v[kSumC] += dc;
      v[kSumE] += de;
    }
    __syncthreads();  // pre[] and lst[] are rewritten by the next batch
  }
}

template <int AX, bool ENERGY>
__device__ __forceinline__ void k_update_body(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out, const double* __restrict__ uf, uint8_t* __restrict__ state, double* __restrict__ theta, const SweepScratch& sc, int nsub, int cap, int ngrp, const VB vb) {
  __shared__ int pre[33];
  __shared__ int lst[32];
  double v[kNSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (g.le)  // uniform: one loop or the other, never both forms' arithmetic
    update_groups<AX, ENERGY, true>(g, c_in, e_in, c_out, e_out, uf, state, theta, sc, nsub, cap, ngrp, vb, pre, lst,
                                    v);
  else
    update_groups<AX, ENERGY, false>(g, c_in, e_in, c_out, e_out, uf, state, theta, sc, nsub, cap, ngrp, vb, pre,
                                     lst, v);
  // work counts of this sweep (kernel A's counters are final by now)
  if (sc.stats && vb.bx == 0 && threadIdx.x == 0) {
    sc.stats[0] = sc.counters[0];
    sc.stats[1] = sc.counters[1] + sc.counters[2];
  }
  if (sc.mlp_stat && vb.bx == 0 && threadIdx.x == 0) {
    sc.mlp_stat[0] = sc.counters[3];
  }
  block_sums(v, sc.sums, vb.bx);
}

template <int AX, bool ENERGY>
__global__ void __launch_bounds__(256)
k_update(GridDev g, const double* c_in, const double* e_in, double* c_out, double* e_out,
         const double* __restrict__ uf, uint8_t* __restrict__ state,
         double* __restrict__ theta, SweepScratch sc, int nsub, int cap, int ngrp) {
  pdl_wait();
  k_update_body<AX, ENERGY>(g, c_in, e_in, c_out, e_out, uf, state, theta, sc, nsub, cap, ngrp, vb_self());
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
    sT[q] = temp_of(g, ev, cv);
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
        // the fused sweep's face energy flux, bit for bit
        Gv = face_energy_flux(g.Cp_l, g.Cp_g, Fv, a, v[0], v[1], v[2], v[3], v[4], g.f32 != 0);
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
    const bool lag = g.le != 0;  // Lagrangian explicit: the cell's own Theta, no frozen state
    const bool dirty = !lag && (stv & 1);
    const double ccv = dirty ? (double)((stv >> 1) & 1) : (c > 0.5 ? 1.0 : 0.0);
    const double Tc = sT[qt];
    const double th = lag ? (Tc * g.Cp_l) * c + (Tc * g.Cp_g) * (1.0 - c)
                          : (dirty ? theta[id] : heat_cap(g.Cp_l, g.Cp_g, ccv) * Tc);
    const double le = sG[qa] - th * sA[qa], re = sG[qb] - th * sA[qb];
    const double en = (e + le) - re;
    e_out[id] = en;
    if (!lag && state && !dirty && (c_after[id] != c || en != e)) {
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


// ---------------------------------------------------------------------------
// Launch plans
// ---------------------------------------------------------------------------
SweepPlan sweep_plan(int axis, const GridDev& g) {
  SweepPlan p;
  if (axis == 0) {
    // rows on grid x (no 65535 limit), segments of a row on grid y
    p.gridA = dim3((g.n[1] * g.n[2] + 7) / 8, (g.n[0] + kSegRow - 1) / kSegRow, 1);
    p.blockA = dim3(32, 8, 1);
    p.cap = g.n[0] < kSegRow ? g.n[0] : kSegRow;  // cells a warp covers
    p.nsub = (long long)p.gridA.x * p.gridA.y * 8;
  } else {
    const int n_t = axis == 1 ? g.n[2] : g.n[1];
    p.gridA = dim3((g.n[0] + 31) / 32, (n_t + kWarpsA - 1) / kWarpsA, (g.n[axis] + kSegA - 1) / kSegA);
    p.blockA = dim3(32, kWarpsA, 1);
    p.cap = (g.n[0] < 32 ? g.n[0] : 32) * (g.n[axis] < kSegA ? g.n[axis] : kSegA);
    p.nsub = (long long)p.gridA.x * p.gridA.y * p.gridA.z * kWarpsA;
  }
  // kernel U: groups of kUpdLists consecutive lists, dealt to the CTAs in
  // turn; about one CTA per 4096 cells, at most one wave (4 per SM): each
  // CTA's FP64 sum tree then serves many listed cells
  const long long cells = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long groups = (p.nsub + kUpdLists - 1) / kUpdLists;
  long long target = (cells + 4095) / 4096;
  if (target > 152 * 4) target = 152 * 4;
  if (target < 1) target = 1;
  const long long ngrp = (groups + target - 1) / target;
  p.lpc = (int)(kUpdLists * ngrp);
  p.gridB = (unsigned)((groups + ngrp - 1) / ngrp);
  return p;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// faces of the axis with the most: N + lines
static size_t max_faces(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  size_t lines = 0;
  for (int a = 0; a < 3; ++a) {
    const size_t l = N / (size_t)g.n[a];
    lines = l > lines ? l : lines;
  }
  return N + lines;
}

size_t sweep_scratch_bytes(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  size_t best = 0;
  for (int a = 0; a < 3; ++a) {
    SweepPlan p = sweep_plan(a, g);
    size_t b = 0;
    b += al256(N * 8);                          // T
    b += al256((size_t)p.nsub * p.cap * 4);     // lists
    b += al256((size_t)p.nsub * 4);             // counts
    b += al256((size_t)p.nsub * p.cap * 4);     // mixed lists (staging)
    b += al256((size_t)p.nsub * p.cap * 4);     // run ends (staging)
    b += 256;                                   // counters
    b += al256(N * 4);                          // grid-wide mixed list
    b += al256(2 * N * 4);                      // grid-wide face list
    b += al256(N * 32);                         // planes
    b += al256(2 * (N / (size_t)g.n[a]) * 32);  // ghost donors' planes
    b += 2 * al256(max_faces(g) * 8);           // face fluxes F, G
    best = b > best ? b : best;
  }
  return best;
}

SweepScratch carve_sweep_scratch(int axis, const GridDev& g, void* ws, SumOut sums) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  SweepPlan p = sweep_plan(axis, g);
  char* b = static_cast<char*>(ws);
  SweepScratch s;
  s.T = reinterpret_cast<double*>(b);           b += al256(N * 8);
  s.list = reinterpret_cast<uint32_t*>(b);      b += al256((size_t)p.nsub * p.cap * 4);
  s.count = reinterpret_cast<int*>(b);          b += al256((size_t)p.nsub * 4);
  s.sums = sums;
  s.tiles = TileMap{nullptr, {0, 0, 0}};
  s.stats = nullptr;
  s.mlp_stat = nullptr;
  s.mlist = reinterpret_cast<uint32_t*>(b);     b += al256((size_t)p.nsub * p.cap * 4);
  s.rlist = reinterpret_cast<uint32_t*>(b);     b += al256((size_t)p.nsub * p.cap * 4);
  s.counters = reinterpret_cast<int*>(b);       b += 256;
  s.gmix = reinterpret_cast<uint32_t*>(b);      b += al256(N * 4);
  s.gface = reinterpret_cast<uint32_t*>(b);     b += al256(2 * N * 4);
  s.gface_cap = (uint32_t)(2 * N);
  s.plane = reinterpret_cast<double*>(b);       b += al256(N * 32);
  s.gplane = reinterpret_cast<double*>(b);      b += al256(2 * (N / (size_t)g.n[axis]) * 32);
  s.F = reinterpret_cast<double*>(b);           b += al256(max_faces(g) * 8);
  s.G = reinterpret_cast<double*>(b);
  return s;
}

int sweep_blocks(int axis, const GridDev& g) { return (int)sweep_plan(axis, g).gridB; }

template <int AX, bool ENERGY>
static void launch_ab(const SweepPlan& p, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                      double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                      SweepScratch sc, int* status, cudaStream_t st) {
  if (AX == 0)
    launch_pdl(k_stream_row<ENERGY>, p.gridA, p.blockA, st, g, c_in, e_in, c_out, e_out, state, sc,
               flux_out != nullptr, p.cap, c_out != c_in);
  else
    launch_pdl(k_stream_col<AX == 0 ? 1 : AX, ENERGY>, p.gridA, p.blockA, st, g, c_in, e_in, c_out, e_out,
               state, sc, flux_out != nullptr, p.cap, c_out != c_in);
  prof_mark(AX == 0 ? "sweep_x.stream" : (AX == 1 ? "sweep_y.stream" : "sweep_z.stream"), st);
  if (g.mlp == 1) {
    // learned normals of the mixed cells (tensor cores), then their planes
    launch_mlp_sweep_normals(g, c_in, sc, st);
    if (g.f32) launch_pdl(k_prep<true, 1>, kPlaneCTAs, kPlaneThreads, st, g, c_in, e_in, sc, AX);
    else launch_pdl(k_prep<false, 1>, kPlaneCTAs, kPlaneThreads, st, g, c_in, e_in, sc, AX);
  } else if (g.mlp == 2) {
    launch_pdl(k_prep<false, 2>, kPlaneCTAs, kPlaneThreads, st, g, c_in, e_in, sc, AX);
  } else if (g.f32) {
    launch_pdl(k_prep<true, 0>, kPlaneCTAs, kPlaneThreads, st, g, c_in, e_in, sc, AX);
  } else {
    launch_pdl(k_prep<false, 0>, kPlaneCTAs, kPlaneThreads, st, g, c_in, e_in, sc, AX);
  }
  prof_mark(AX == 0 ? "sweep_x.prep" : (AX == 1 ? "sweep_y.prep" : "sweep_z.prep"), st);
  launch_pdl(k_faces<AX, ENERGY>, kFaceCTAs, kFaceThreads, st, g, c_in, e_in, uf, flux_out, sc, status);
  prof_mark(AX == 0 ? "sweep_x.faces" : (AX == 1 ? "sweep_y.faces" : "sweep_z.faces"), st);
  launch_pdl(k_update<AX, ENERGY>, p.gridB, 256, st, g, c_in, e_in, c_out, e_out, uf, state, theta, sc,
             (int)p.nsub, p.cap, p.lpc / kUpdLists);
  prof_mark(AX == 0 ? "sweep_x.update" : (AX == 1 ? "sweep_y.update" : "sweep_z.update"), st);
}

cudaError_t launch_sweep(int axis, const GridDev& g, const double* c_in, const double* e_in, double* c_out,
                         double* e_out, const double* uf, uint8_t* state, double* theta, double* flux_out,
                         SweepScratch sc, bool zero_counters, cudaStream_t st) {
  int* status = device_status_ptr();
  const SweepPlan p = sweep_plan(axis, g);
  if (zero_counters) {  // else the caller's tile pass cleared them
    const cudaError_t err = cudaMemsetAsync(sc.counters, 0, 4 * sizeof(int), st);
    if (err != cudaSuccess) return err;
    prof_mark("sweep.memset", st);
  }
  if (e_in) {
    if (axis == 0) launch_ab<0, true>(p, g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sc, status, st);
    else if (axis == 1) launch_ab<1, true>(p, g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sc, status, st);
    else launch_ab<2, true>(p, g, c_in, e_in, c_out, e_out, uf, state, theta, flux_out, sc, status, st);
  } else {
    if (axis == 0) launch_ab<0, false>(p, g, c_in, nullptr, c_out, nullptr, uf, state, theta, flux_out, sc, status, st);
    else if (axis == 1)
      launch_ab<1, false>(p, g, c_in, nullptr, c_out, nullptr, uf, state, theta, flux_out, sc, status, st);
    else launch_ab<2, false>(p, g, c_in, nullptr, c_out, nullptr, uf, state, theta, flux_out, sc, status, st);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Grouped sweep kernels: every box of a batch in one launch (in place, with
// energy, no exported fluxes); each CTA takes its box's arguments.
// ---------------------------------------------------------------------------
template <int AX>
__global__ void __launch_bounds__(256) k_stream_grp(GroupMap m, const SweepArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ SweepArgs sA;
  const SweepArgs& A = cta_args(args, b, sA);
  if (AX == 0)
    k_stream_row_body<true>(A.g, A.c, A.e, A.c, A.e, A.state, A.sc, 0, A.cap, 0, vb);
  else
    k_stream_col_body<AX == 0 ? 1 : AX, true>(A.g, A.c, A.e, A.c, A.e, A.state, A.sc, 0, A.cap, 0, vb);
}
template <bool F32, int NRM>
__global__ void __launch_bounds__(kPlaneThreads) k_prep_grp(GroupMap m, const SweepArgs* __restrict__ args, int ax) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ SweepArgs sA;
  const SweepArgs& A = cta_args(args, b, sA);
  k_prep_body<F32, NRM>(A.g, A.c, A.e, A.sc, ax, vb);
}
template <int AX>
__global__ void __launch_bounds__(kFaceThreads) k_faces_grp(GroupMap m, const SweepArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ SweepArgs sA;
  const SweepArgs& A = cta_args(args, b, sA);
  k_faces_body<AX, true>(A.g, A.c, A.e, A.uf, nullptr, A.sc, A.status, vb);
}
template <int AX>
__global__ void __launch_bounds__(256) k_update_grp(GroupMap m, const SweepArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ SweepArgs sA;
  const SweepArgs& A = cta_args(args, b, sA);
  k_update_body<AX, true>(A.g, A.c, A.e, A.c, A.e, A.uf, A.state, A.theta, A.sc, A.nsub, A.cap, A.ngrp, vb);
}

template <int AX>
static void launch_sweep_grp_t(int f32, int youngs, const GroupMap* m, const SweepArgs* a, const unsigned* n,
                               cudaStream_t st) {
  if (n[0]) k_stream_grp<AX><<<n[0], dim3(32, 8), 0, st>>>(m[0], a);
  prof_mark("group.stream", st);
  if (n[1]) {
    if (youngs) k_prep_grp<false, 2><<<n[1], kPlaneThreads, 0, st>>>(m[1], a, AX);
    else if (f32) k_prep_grp<true, 0><<<n[1], kPlaneThreads, 0, st>>>(m[1], a, AX);
    else k_prep_grp<false, 0><<<n[1], kPlaneThreads, 0, st>>>(m[1], a, AX);
  }
  prof_mark("group.prep", st);
  if (n[2]) k_faces_grp<AX><<<n[2], kFaceThreads, 0, st>>>(m[2], a);
  prof_mark("group.faces", st);
  if (n[3]) k_update_grp<AX><<<n[3], 256, 0, st>>>(m[3], a);
  prof_mark("group.update", st);
}

cudaError_t launch_sweep_grp(int axis, int f32, int youngs, const GroupMap* maps, const SweepArgs* a,
                             const unsigned* ctas, cudaStream_t st) {
  if (axis == 0) launch_sweep_grp_t<0>(f32, youngs, maps, a, ctas, st);
  else if (axis == 1) launch_sweep_grp_t<1>(f32, youngs, maps, a, ctas, st);
  else launch_sweep_grp_t<2>(f32, youngs, maps, a, ctas, st);
  return cudaGetLastError();
}

int prep_ctas() { return kPlaneCTAs; }

cudaError_t launch_energy(int axis, const GridDev& g, const double* c_before, const double* c_after,
                          const double* e_in, double* e_out, const double* F, const double* uf, uint8_t* state,
                          double* theta, cudaStream_t st) {
  if (axis == 0)
    k_energy<0><<<sweep_grid<0>(g), sweep_block<0>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  else if (axis == 1)
    k_energy<1><<<sweep_grid<1>(g), sweep_block<1>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  else
    k_energy<2><<<sweep_grid<2>(g), sweep_block<2>(), 0, st>>>(g, c_before, c_after, e_in, e_out, F, uf, state, theta);
  prof_mark("energy", st);
  return cudaGetLastError();
}

}  // namespace vofgb
