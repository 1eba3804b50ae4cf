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
#include "vof_sums.cuh"

namespace vofgb {

constexpr int kShBX = 32, kShBY = 4, kShBZ = 2, kShThreads = kShBX * kShBY * kShBZ;

__device__ __forceinline__ bool same_bits_dev(double a, double b) { return dbits(a) == dbits(b); }

// ---------------------------------------------------------------------------
// Shift in four kernels.
//   stream:    (out of place: copies c, e to the output; stand-alone: sums
//              c, e) lists the moving mixed cells per warp (up to 256 cells
//              of one x row per warp, fixed order) and appends them to a
//              grid-wide list, cells with c
//              within 1e-3 of 0 or 1 ("edge" cells, whose plane constant
//              takes the bisection) at its back, the others at its front;
//   planes:    one moving mixed cell per thread over the grid-wide list:
//              plane (MYC normal + plane constant), shift |m|_2 dd, the
//              cell's own shifted volume, and the receivers it settles --
//              pure neighbours of the receding phase whose first reaching
//              neighbour (scan order z outer, x inner) it is;
//   receivers: one receiver per thread: the largest volume swept in it by
//              the extended planes of its reaching neighbours;
//   sums:      per warp list in fixed order, applies and sums the changes
//              of every moving cell and of the receivers it settled, so the
//              sums do not depend on the order of the grid-wide lists.
// Only the last kernel writes c and e, and each cell it writes is touched by
// one thread, so the shift may run in place (c_out == c_in, e_out == e_in).
// ---------------------------------------------------------------------------
constexpr int kWarpCells = 256;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kListThreads = 128;     // planes / receivers kernels: CTA size
constexpr int kListCTAs = 152 * 4;    // and grid (grid-stride loops)

__device__ __forceinline__ void decode(const GridDev& g, size_t id, int& x, int& y, int& z) { cell_xyz(g, id, x, y, z); }

__device__ __forceinline__ size_t cell_id(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

// c within 1e-3 of 0 or 1: alpha(c) is ill-conditioned and the plane is
// extrapolated into neighbours, so its constant takes the bisection
__device__ __forceinline__ bool edge_cell(double c) {
  return dbits(c) < 0x3F50624DD2F1A9FCLL /* 1e-3 */ || dbits(c) > 0x3FEFF7CED916872BLL /* 0.999 */;
}

// neighbour of (x, y, z) at offset (ox, oy, oz); false beyond a
// zero-gradient boundary
__device__ __forceinline__ bool neighbour(const GridDev& g, int x, int y, int z, int ox, int oy, int oz, size_t& id) {
  int px = x + ox, py = y + oy, pz = z + oz;
  if (g.bc[0] != 0 && (px < 0 || px >= g.n[0])) return false;
  if (g.bc[1] != 0 && (py < 0 || py >= g.n[1])) return false;
  if (g.bc[2] != 0 && (pz < 0 || pz >= g.n[2])) return false;
  id = cell_id(g, map_idx(px, g.n[0], g.bc[0]), map_idx(py, g.n[1], g.bc[1]), map_idx(pz, g.n[2], g.bc[2]));
  return true;
}

// offsets as bit indices: ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1), 0..26
__device__ __forceinline__ int offset_bit(int ox, int oy, int oz) { return ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1); }

__device__ __forceinline__ void k_shift_stream_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out, double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, const ShiftScratch& sc, const SumOut& sums, int copy, const VB vb) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int nx = g.n[0], ny = g.n[1];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const unsigned lt = (1u << lane) - 1u;
  const int row = vb.bx * 8 + warp;  // row = z * ny + y (grid x: rows, grid y: segments)
  const bool rowok = row < ny * g.n[2];
  const int x0 = vb.by * kWarpCells, x1 = min(x0 + kWarpCells, nx);
  const size_t rbase = (size_t)(rowok ? row : 0) * nx;
  const size_t w = (size_t)row * vb.gy + vb.by;  // list of this warp
  const int cap = nx < kWarpCells ? nx : kWarpCells;
  uint32_t* list = sc.list + w * cap;
  const bool do_sums = sums.partials || sums.diag;
  // quiet tiles of the row segment (in place only): bit l = tile l quiet
  unsigned qmask = 0u;
  if (sc.tiles.quiet && !copy && !do_sums && rowok) {
    const int txi = (x0 >> 3) + lane;
    const int y = row % ny, z = row / ny;
    const bool q = txi * kTile < x1 &&
                   sc.tiles.quiet[((size_t)(z >> 3) * sc.tiles.nt[1] + (y >> 3)) * sc.tiles.nt[0] + txi] != 0;
    qmask = __ballot_sync(kFullMask, q);
  }
  int n = 0, ne = 0;
  double v[kNSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const bool uni_moving = dnz(dd_uniform);
  if (rowok) {
    for (int it = 0; it < kWarpCells / 32 && x0 + 32 * it < x1; ++it) {
      if (((qmask >> (4 * it)) & 0xFu) == 0xFu) continue;  // four quiet tiles: no mixed cell
      const int X = x0 + 32 * it + lane;
      const bool ok = X < x1;
      const size_t id = rbase + X;
      double c = 0.0;
      if (ok) {
        c = __ldg(c_in + id);
        if (copy || do_sums) {
          const double e = __ldg(e_in + id);
          if (copy) {  // out of place: every cell starts as a copy
            c_out[id] = c;
            e_out[id] = e;
          }
          v[kSumC] += c;
          v[kSumE] += e;
        }
      }
      bool moving = ok && is_mixed_b(c, g);
      double ddv = dd_uniform;
      if (moving) {
        if (dd) ddv = __ldg(dd + id);
        moving = dd ? dnz(ddv) : uni_moving;
      }
      // every visited cell's reach byte and claim word are written here, so
      // the later kernels (which read them only next to moving cells, never
      // in a skipped quiet tile) need no cleared arrays
      if (ok) {
        sc.reach[id] = moving ? (dlt0(ddv) ? 1 : 2) : 0;
        sc.claim[id] = 0u;
      }
      const unsigned m = __ballot_sync(kFullMask, moving);
      if (moving) list[n + __popc(m & lt)] = (uint32_t)id;
      n += __popc(m);
      ne += __popc(__ballot_sync(kFullMask, moving && edge_cell(c)));
    }
    if (lane == 0) sc.count[w] = n;
  }
  if (n > 0) {  // warp-uniform: append to the grid-wide list
    int bn = 0, be = 0;
    if (lane == 0) {
      if (n - ne) bn = atomicAdd(sc.counters + 0, n - ne);
      if (ne) be = atomicAdd(sc.counters + 1, ne);
    }
    bn = __shfl_sync(kFullMask, bn, 0);
    be = __shfl_sync(kFullMask, be, 0);
    __syncwarp();
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const bool vv = j < n;
      const uint32_t id = vv ? list[j] : 0u;
      const bool edge = vv && edge_cell(__ldg(c_in + id));
      const unsigned me = __ballot_sync(kFullMask, edge), mn = __ballot_sync(kFullMask, vv && !edge);
      if (edge) sc.gmix[N - 1 - (size_t)(be + __popc(me & lt))] = id;
      else if (vv) sc.gmix[bn + __popc(mn & lt)] = id;
      be += __popc(me);
      bn += __popc(mn);
    }
  }
  block_sums(v, sums, vb.bx + vb.gx * vb.by);
}

__global__ void __launch_bounds__(256)
k_shift_stream(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
               double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, ShiftScratch sc,
               SumOut sums, int copy) {
  pdl_wait();
  k_shift_stream_body(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc, sums, copy, vb_self());
}

// One moving mixed cell: plane (MYC normal + plane constant), shift
// |m|_2 dd, its own shifted volume, and the claims on the receivers it
// reaches.  LANES = 3: the three lanes leader .. leader + 2 (mask gmask) of
// one cell share its bisection (edge cells); every lane computes the same
// values, and the stores and the claims' atomic ORs repeat them harmlessly.
template <int LANES>
__device__ __forceinline__ void shift_plane_cell(const GridDev& g, const double* __restrict__ c_in,
                                                 const double* __restrict__ dd, double dd_uniform,
                                                 const ShiftScratch& sc, size_t id, unsigned gmask, int leader,
                                                 int sub) {
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
  double al;
  if (LANES == 3) al = plane_alpha_bisect_t<3>(m[0], m[1], m[2], ct, gmask, leader, sub);
  else al = edge_cell(ct) ? plane_alpha_bisect(m[0], m[1], m[2], ct) : plane_alpha(m[0], m[1], m[2], ct);
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
  sc.cnew[id] = volume_nn(m[0], m[1], m[2], ast);  // applied by the sums kernel
  // claim the receivers this shift reaches: bit 31 - b of a pure
  // neighbour's claim word, b = this cell's offset index seen from it
  // (scan order); the first reaching neighbour in the scan order -- the
  // one that settles the receiver -- holds the highest set bit whatever
  // the order of the atomics
  const bool full = dlt0(ddv);  // the kind of pure cell this shift reaches
  for (int oz = -1; oz <= 1; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        if (!ox && !oy && !oz) continue;
        size_t pid;
        if (!neighbour(g, x, y, z, ox, oy, oz, pid)) continue;
        const double cp = __ldg(c_in + pid);
        if (is_mixed_b(cp, g) || is_full_b(cp, g) != full) continue;
        atomicOr(sc.claim + pid, 0x80000000u >> offset_bit(-ox, -oy, -oz));
      }
}

// The list's front (cells whose plane constant is inverted directly): one
// per thread.  Its back (edge cells, whose constant takes the bisection): ten
// per warp, three lanes each, the warps' chunks taken from the grid's last
// warp down -- warps the front leaves idle, on SMs of their own -- so the
// bisections' long FP64 chains run side by side.
__device__ __forceinline__ void k_shift_planes_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform, const ShiftScratch& sc, const VB vb) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int nn = sc.counters[0], ne = sc.counters[1];
  const int lane = threadIdx.x & 31;
  const int stride = vb.gx * blockDim.x;
  for (int i = vb.bx * blockDim.x + threadIdx.x; i < nn; i += stride)
    shift_plane_cell<1>(g, c_in, dd, dd_uniform, sc, sc.gmix[i], 0u, 0, 0);
  const int nw = (int)(vb.gx * (blockDim.x >> 5)), gw = (int)((vb.bx * blockDim.x + threadIdx.x) >> 5);
  const int nchunk = (ne + 9) / 10;
  for (int wc = nw - 1 - gw; wc < nchunk; wc += nw) {
    const int j = wc * 10 + lane / 3;
    if (lane >= 30 || j >= ne) continue;
    const int leader = (lane / 3) * 3;
    shift_plane_cell<3>(g, c_in, dd, dd_uniform, sc, sc.gmix[N - 1 - (size_t)j], 7u << leader, leader,
                        lane - leader);
  }
}

__global__ void __launch_bounds__(kListThreads)
k_shift_planes(GridDev g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform,
               ShiftScratch sc) {
  pdl_wait();
  k_shift_planes_body(g, c_in, dd, dd_uniform, sc, vb_self());
}

// Per moving mixed cell (same list, after all claims are in): the receivers
// it settles are the pure neighbours whose highest claim bit is its own
// (on periodic axes of 1 or 2 cells several offsets lead to the same cell;
// only the first of them in the scan order settles it); they are appended to
// the receiver list, one atomic per warp.
__device__ __forceinline__ void k_shift_own_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform, const ShiftScratch& sc, const VB vb) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int nn = sc.counters[0], ne = sc.counters[1];
  const int lane = threadIdx.x & 31;
  const int total = nn + ne;
  // whole warps iterate together (the receiver append below is warp-wide)
  const int stride = vb.gx * blockDim.x;
  for (int i0 = vb.bx * blockDim.x + (threadIdx.x & ~31); i0 < total; i0 += stride) {
    const int i = i0 + lane;
    const bool v = i < total;
    unsigned own = 0u;
    int x = 0, y = 0, z = 0;
    if (v) {
      const size_t id = i < nn ? sc.gmix[i] : sc.gmix[N - 1 - (size_t)(i - nn)];
      decode(g, id, x, y, z);
      const double ddv = dd ? __ldg(dd + id) : dd_uniform;
      const bool full = dlt0(ddv);
#pragma unroll
      for (int b = 0; b < 27; ++b) {
        if (b == 13) continue;
        const int ox = b % 3 - 1, oy = (b / 3) % 3 - 1, oz = b / 9 - 1;
        size_t pid;
        if (!neighbour(g, x, y, z, ox, oy, oz, pid)) continue;
        const double cp = __ldg(c_in + pid);
        const unsigned cl = __ldg(sc.claim + pid);
        if (is_mixed_b(cp, g) || is_full_b(cp, g) != full) continue;
        if (__clz(cl) == offset_bit(-ox, -oy, -oz)) own |= 1u << b;
      }
      sc.own[id] = own;
    }
    // append the settled receivers: one atomic per warp
    const int k = __popc(own);
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += t;
    }
    const int wtot = __shfl_sync(kFullMask, incl, 31);
    int base = 0;
    if (lane == 31 && wtot) base = atomicAdd(sc.counters + 2, wtot);
    base = __shfl_sync(kFullMask, base, 31) + incl - k;
    while (own) {
      const int b = __ffs(own) - 1;
      own &= own - 1u;
      const int oz = b / 9 - 1, oy = (b / 3) % 3 - 1, ox = b % 3 - 1;
      size_t pid = 0;
      neighbour(g, x, y, z, ox, oy, oz, pid);
      sc.recv[base++] = (uint32_t)pid;
    }
  }
}

__global__ void __launch_bounds__(kListThreads)
k_shift_own(GridDev g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform,
            ShiftScratch sc) {
  pdl_wait();
  k_shift_own_body(g, c_in, dd, dd_uniform, sc, vb_self());
}

// Per receiver (a pure cell some moving neighbour settles): the largest
// change |V(alpha* + s) - V(alpha + s)| among the planes of its reaching
// neighbours, extended into it (s: the plane's offset seen from the
// receiver), the first such maximum in the scan order of the offsets.  Four
// lanes share a receiver, lane j taking the offsets b = j mod 4; the lanes'
// results are combined by the same rule (larger change, then smaller b), so
// the result is the one-lane scan's.
constexpr int kRecvLanes = 4;
__device__ __forceinline__ void k_shift_receivers_body(const GridDev& g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform, const ShiftScratch& sc, const VB vb) {
  const int nr = sc.counters[2];
  const int lane = threadIdx.x & 31, sub = lane & (kRecvLanes - 1);
  constexpr int kPerWarp = 32 / kRecvLanes;
  const int gw = (int)((vb.bx * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((vb.gx * blockDim.x) >> 5);
  // whole warps iterate together (the combination below is a shuffle)
  for (int r0 = gw * kPerWarp; r0 < nr; r0 += nwarps * kPerWarp) {
    const int i = r0 + lane / kRecvLanes;
    const bool valid = i < nr;
    double best = 0.0;
    int bestb = 27;
    size_t pid = 0;
    if (valid) {
      pid = sc.recv[i];
      const double cp = __ldg(c_in + pid);
      const unsigned want = is_full_b(cp, g) ? 1u : 2u;
      const bool full = want == 1u;
      int px, py, pz;
      decode(g, pid, px, py, pz);
      for (int b = sub; b < 27; b += kRecvLanes) {  // this lane's offsets in scan order
        if (b == 13) continue;
        const int rx = b % 3 - 1, ry = (b / 3) % 3 - 1, rz = b / 9 - 1;
        size_t sid;
        if (!neighbour(g, px, py, pz, rx, ry, rz, sid)) continue;
        if (!(__ldg(sc.reach + sid) & want)) continue;  // not a reaching neighbour
        const double sft = sc.shift[sid];
        if (!dnz(sft)) continue;  // a zero normal does not move
        const double4 pl = reinterpret_cast<const double4*>(sc.plane)[sid];
        const double m0 = pl.x, m1 = pl.y, m2 = pl.z, al = pl.w;
        // the receiver sits at offset -(rx, ry, rz) from the source
        const double shiftv = -((m0 * (double)(-rx) + m1 * (double)(-ry)) + m2 * (double)(-rz));
        const double a_old = al + shiftv;
        const double a_new = (al + sft) + shiftv;
        double lo = 0.0, hi = 0.0;
        if (dlt0(m0)) lo += m0; else hi += m0;
        if (dlt0(m1)) lo += m1; else hi += m1;
        if (dlt0(m2)) lo += m2; else hi += m2;
        // the extended plane stays outside the receiver: both volumes are
        // exactly 1 (or 0); the margin clears the rounding of that test
        if (full ? (a_new >= hi + 1e-9) : (a_new <= lo - 1e-9)) continue;
        const VolNormal vn = volume_normal_nn(m0, m1, m2);
        const double sw = volume_at_nn(vn, a_new) - volume_at_nn(vn, a_old);
        if (nn_lt(fabs(best), fabs(sw))) {
          best = sw;
          bestb = b;
        }
      }
    }
    // combine the receiver's lanes: larger |change|, then the earlier offset
#pragma unroll
    for (int o = 1; o < kRecvLanes; o <<= 1) {
      const double ob = __shfl_xor_sync(kFullMask, best, o);
      const int obb = __shfl_xor_sync(kFullMask, bestb, o);
      const long long mine = dbits(fabs(best)), other = dbits(fabs(ob));
      if (other > mine || (other == mine && obb < bestb)) {
        best = ob;
        bestb = obb;
      }
    }
    if (valid && sub == 0) sc.sweep[pid] = best;  // applied by the sums kernel
  }
}

__global__ void __launch_bounds__(kListThreads)
k_shift_receivers(GridDev g, const double* __restrict__ c_in, const double* __restrict__ dd, double dd_uniform,
                  ShiftScratch sc) {
  pdl_wait();
  k_shift_receivers_body(g, c_in, dd, dd_uniform, sc, vb_self());
}

// Applies the new values (moving cells and the receivers they settle) and
// sums the changes, per warp list in fixed order.  Every cell it writes is
// read and written by one thread only, so it may work in place.
__device__ __forceinline__ void k_shift_sums_body(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out, const ShiftScratch& sc, long long nwarps, const SumOut& sums, const VB vb) {
  const int lane = threadIdx.x & 31;
  const size_t w = (size_t)vb.bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int cap = g.n[0] < kWarpCells ? g.n[0] : kWarpCells;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // dc, clamped, de
  if ((long long)w < nwarps) {
    const int cnt = sc.count[w];
    const uint32_t* list = sc.list + w * cap;
    for (int i = lane; i < cnt; i += 32) {
      const size_t qid = list[i];
      const double ct = c_in[qid], cn = sc.cnew[qid];
      if (!same_bits_dev(cn, ct)) {
        const double dc = cn - ct;
        const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
        const double eq = e_in[qid];
        c_out[qid] = cn;
        e_out[qid] = eq + de;
        acc[0] += dc;
        acc[2] += de;
      }
      unsigned own = sc.own[qid];
      if (!own) continue;
      int x, y, z;
      decode(g, qid, x, y, z);
      while (own) {
        const int b = __ffs(own) - 1;
        own &= own - 1u;
        size_t pid = 0;
        neighbour(g, x, y, z, b % 3 - 1, (b / 3) % 3 - 1, b / 9 - 1, pid);
        const double best = sc.sweep[pid];
        if (!dnz(best)) continue;
        const double cp = c_in[pid];
        const double v = cp + best;
        const double vc = dlt0(v) ? 0.0 : (dgt1(v) ? 1.0 : v);
        if (!deq(v, vc)) acc[1] += v - vc;
        if (!same_bits_dev(vc, cp)) {
          const double dc = vc - cp;
          const double de = dc * (g.Cp_l - g.Cp_g) * g.T_sat;
          const double ep = e_in[pid];
          c_out[pid] = vc;
          e_out[pid] = ep + de;
          acc[0] += dc;
          acc[2] += de;
        }
      }
    }
  }
  double v[kNSums];
  v[kSumC] = acc[0];  // sum c_out = sum c_in + sum dc
  v[kSumE] = acc[2];
  v[kSumClip] = 0.0;
  v[kSumShDc] = acc[0];
  v[kSumUnpl] = acc[1];
  v[kSumShDe] = acc[2];
  if (sc.stats && vb.bx == 0 && threadIdx.x == 0) {
    sc.stats[0] = sc.counters[0];
    sc.stats[1] = sc.counters[1];
    sc.stats[2] = sc.counters[2];
  }
  block_sums(v, sums, vb.bx);
}

__global__ void __launch_bounds__(256)
k_shift_sums(GridDev g, const double* c_in, const double* e_in, double* c_out, double* e_out, ShiftScratch sc,
             long long nwarps, SumOut sums) {
  pdl_wait();
  k_shift_sums_body(g, c_in, e_in, c_out, e_out, sc, nwarps, sums, vb_self());
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

// one list per x-row segment of up to kWarpCells cells
static long long shift_warps(const GridDev& g) {
  return (long long)((g.n[0] + kWarpCells - 1) / kWarpCells) * g.n[1] * g.n[2];
}

int shift_sum_blocks(const GridDev& g) { return (int)((shift_warps(g) + 7) / 8); }

static dim3 shift_stream_grid(const GridDev& g) {
  return dim3((unsigned)((g.n[1] * g.n[2] + 7) / 8), (unsigned)((g.n[0] + kWarpCells - 1) / kWarpCells), 1);
}

int shift_stream_blocks(const GridDev& g) {
  const dim3 d = shift_stream_grid(g);
  return (int)(d.x * d.y);
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t shift_scratch_bytes(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_warps(g);
  const size_t cap = g.n[0] < kWarpCells ? g.n[0] : kWarpCells;
  return al256(nw * cap * 4)  // per-warp lists
         + al256(nw * 4)      // counts
         + 256                // counters
         + al256(N * 4)       // grid-wide list of moving cells
         + al256(N * 4)       // receivers
         + al256(N * 32)      // planes
         + al256(N * 8)       // shifts
         + al256(N * 8)       // sweeps
         + al256(N * 8)       // new c of moving cells
         + al256(N * 4)       // settled-receiver masks
         + al256(N)           // reach bytes
         + al256(N * 4);      // receiver claims
}

ShiftScratch carve_shift_scratch(const GridDev& g, void* ws) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_warps(g);
  const size_t cap = g.n[0] < kWarpCells ? g.n[0] : kWarpCells;
  char* b = static_cast<char*>(ws);
  ShiftScratch s;
  s.list = reinterpret_cast<uint32_t*>(b);   b += al256(nw * cap * 4);
  s.count = reinterpret_cast<int*>(b);       b += al256(nw * 4);
  s.counters = reinterpret_cast<int*>(b);    b += 256;
  s.gmix = reinterpret_cast<uint32_t*>(b);   b += al256(N * 4);
  s.recv = reinterpret_cast<uint32_t*>(b);   b += al256(N * 4);
  s.plane = reinterpret_cast<double*>(b);    b += al256(N * 32);
  s.shift = reinterpret_cast<double*>(b);    b += al256(N * 8);
  s.sweep = reinterpret_cast<double*>(b);    b += al256(N * 8);
  s.cnew = reinterpret_cast<double*>(b);     b += al256(N * 8);
  s.own = reinterpret_cast<uint32_t*>(b);    b += al256(N * 4);
  s.reach = reinterpret_cast<uint8_t*>(b);   b += al256(N);
  s.claim = reinterpret_cast<uint32_t*>(b);
  s.tiles = TileMap{nullptr, {0, 0, 0}};
  s.stats = nullptr;
  return s;
}

__global__ void __launch_bounds__(256) k_shift_stream_grp(GroupMap m, const ShiftArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ ShiftArgs sA;
  const ShiftArgs& A = cta_args(args, b, sA);
  const SumOut none = sums_to_partials(nullptr, kNSums);
  k_shift_stream_body(A.g, A.c, A.e, A.c, A.e, A.dd, A.dd_uniform, A.sc, none, 0, vb);
}
__global__ void __launch_bounds__(kListThreads) k_shift_planes_grp(GroupMap m, const ShiftArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ ShiftArgs sA;
  const ShiftArgs& A = cta_args(args, b, sA);
  k_shift_planes_body(A.g, A.c, A.dd, A.dd_uniform, A.sc, vb);
}
__global__ void __launch_bounds__(kListThreads) k_shift_own_grp(GroupMap m, const ShiftArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ ShiftArgs sA;
  const ShiftArgs& A = cta_args(args, b, sA);
  k_shift_own_body(A.g, A.c, A.dd, A.dd_uniform, A.sc, vb);
}
__global__ void __launch_bounds__(kListThreads) k_shift_receivers_grp(GroupMap m, const ShiftArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ ShiftArgs sA;
  const ShiftArgs& A = cta_args(args, b, sA);
  k_shift_receivers_body(A.g, A.c, A.dd, A.dd_uniform, A.sc, vb);
}
__global__ void __launch_bounds__(256) k_shift_sums_grp(GroupMap m, const ShiftArgs* __restrict__ args) {
  unsigned b;
  const VB vb = vb_group(m, b);
  __shared__ ShiftArgs sA;
  const ShiftArgs& A = cta_args(args, b, sA);
  k_shift_sums_body(A.g, A.c, A.e, A.c, A.e, A.sc, A.nw, A.sums, vb);
}

cudaError_t launch_shift_grp(const GroupMap* m, const ShiftArgs* a, const unsigned* n, cudaStream_t st) {
  if (n[0]) k_shift_stream_grp<<<n[0], dim3(32, 8), 0, st>>>(m[0], a);
  prof_mark("group.shift_stream", st);
  if (n[1]) k_shift_planes_grp<<<n[1], kListThreads, 0, st>>>(m[1], a);
  prof_mark("group.shift_planes", st);
  if (n[2]) k_shift_own_grp<<<n[2], kListThreads, 0, st>>>(m[2], a);
  prof_mark("group.shift_own", st);
  if (n[3]) k_shift_receivers_grp<<<n[3], kListThreads, 0, st>>>(m[3], a);
  prof_mark("group.shift_receivers", st);
  if (n[4]) k_shift_sums_grp<<<n[4], 256, 0, st>>>(m[4], a);
  prof_mark("group.shift_sums", st);
  return cudaGetLastError();
}

int shift_list_ctas() { return kListCTAs; }
long long shift_warps_of(const GridDev& g) { return shift_warps(g); }
dim3 shift_stream_grid_of(const GridDev& g) { return shift_stream_grid(g); }

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, ShiftScratch sc, SumOut stream_sums,
                         SumOut sums, bool zero_counters, cudaStream_t st) {
  const long long nw = shift_warps(g);
  cudaError_t err = cudaSuccess;
  if (zero_counters) {  // else the caller's tile pass cleared them
    err = cudaMemsetAsync(sc.counters, 0, 3 * sizeof(int), st);
    if (err != cudaSuccess) return err;
    prof_mark("shift.memset", st);
  }
  launch_pdl(k_shift_stream, shift_stream_grid(g), dim3(32, 8), st, g, c_in, e_in, c_out, e_out, dd, dd_uniform,
             sc, stream_sums, c_out != c_in);
  prof_mark("shift.stream", st);
  launch_pdl(k_shift_planes, kListCTAs, kListThreads, st, g, c_in, dd, dd_uniform, sc);
  prof_mark("shift.planes", st);
  launch_pdl(k_shift_own, kListCTAs, kListThreads, st, g, c_in, dd, dd_uniform, sc);
  prof_mark("shift.own", st);
  launch_pdl(k_shift_receivers, kListCTAs, kListThreads, st, g, c_in, dd, dd_uniform, sc);
  prof_mark("shift.receivers", st);
  launch_pdl(k_shift_sums, shift_sum_blocks(g), 256, st, g, c_in, e_in, c_out, e_out, sc, nw, sums);
  prof_mark("shift.sums", st);
  err = cudaGetLastError();
  if (err == cudaSuccess && state) {
    err = cudaMemsetAsync(state, 0, (size_t)g.n[0] * g.n[1] * g.n[2], st);
    prof_mark("shift.memset_state", st);
  }
  return err;
}

cudaError_t launch_reconstruct(const GridDev& g, const double* c, double* m, double* alpha, uint8_t* mixed,
                               cudaStream_t st) {
  k_reconstruct<<<sh_grid(g), dim3(kShBX, kShBY, kShBZ), 0, st>>>(g, c, m, alpha, mixed);
  prof_mark("reconstruct", st);
  return cudaGetLastError();
}

// Deterministic reduction of per-block partials: one CTA, fixed order.
// Fixed-order reduction of per-CTA partial sums in two levels: kReduceCTAs
// CTAs each sum a fixed contiguous range of rows (one row per thread, then a
// shared-memory tree) into scratch, then one CTA per job sums those partials
// the same way.  The order depends only on the sizes, so the sums are
// identical run to run.
constexpr int kReduceThreads = 256;


// The CTA's per-thread values v[k] (k < nk) summed in a fixed order: staged
// in shared memory, warp k sums entry lane, lane + 32, ... then a shuffle
// tree; lane 0 of warp k writes out[k].  One barrier for all nk values.
__device__ __forceinline__ void cta_sums(const double (&v)[kMaxReduceK], int nk, double* out,
                                         double (*red)[kReduceThreads]) {
#pragma unroll
  for (int k = 0; k < kMaxReduceK; ++k)
    if (k < nk) red[k][threadIdx.x] = v[k];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < nk) {
    double x = 0.0;
#pragma unroll
    for (int j = 0; j < kReduceThreads / 32; ++j) x += red[w][lane + 32 * j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) out[w] = x;
  }
  __syncthreads();  // red is reused
}
static_assert(kMaxReduceK <= kReduceThreads / 32, "a warp per output");

// part `part` of `nparts` of a job's rows into out[k] (k < nk)
__device__ __forceinline__ void reduce1_body(const ReduceJob& J, unsigned part, unsigned nparts, double* out,
                                             double (*red)[kReduceThreads]) {
  const int chunk = (J.nblocks + (int)nparts - 1) / (int)nparts;
  const int b0 = (int)part * chunk, b1 = min(b0 + chunk, J.nblocks);
  double s[kMaxReduceK];
#pragma unroll
  for (int k = 0; k < kMaxReduceK; ++k) s[k] = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += kReduceThreads) {
    const double* row = J.partials + (size_t)b * J.stride + J.k0;
#pragma unroll
    for (int k = 0; k < kMaxReduceK; ++k)
      if (k < J.nk) s[k] += row[k];
  }
  cta_sums(s, J.nk, out, red);
}
// a job's nparts partials (kMaxReduceK apart) into J.out (read from L2: in
// the fused reduction other CTAs of the same launch wrote them)
__device__ __forceinline__ void reduce2_body(const ReduceJob& J, const double* part, int nparts,
                                             double (*red)[kReduceThreads]) {
  double s[kMaxReduceK];
#pragma unroll
  for (int k = 0; k < kMaxReduceK; ++k) s[k] = 0.0;
  for (int b = threadIdx.x; b < nparts; b += kReduceThreads) {
#pragma unroll
    for (int k = 0; k < kMaxReduceK; ++k)
      if (k < J.nk) s[k] += __ldcg(part + (size_t)b * kMaxReduceK + k);
  }
  cta_sums(s, J.nk, J.out, red);
}

// Both levels in one launch (one job): every CTA its part, and the CTA that
// finishes last (a ticket, zero at the start and left zero) the second
// level -- the same arithmetic and order as the grouped pair k_reduce1_grp
// and k_reduce2_grp below, so a box sums to the same bits either way.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_fused(ReduceJobs jobs, double* __restrict__ scratch,
                                                                 int* __restrict__ ticket) {
  __shared__ double red[kMaxReduceK][kReduceThreads];
  __shared__ int last;
  pdl_wait();
  const ReduceJob J = jobs.job[0];
  reduce1_body(J, blockIdx.x, gridDim.x, scratch + (size_t)blockIdx.x * kMaxReduceK, red);
  __threadfence();  // this CTA's partials before its ticket
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (last) {
    __threadfence();  // the other CTAs' partials before they are read
    reduce2_body(J, scratch, (int)gridDim.x, red);
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// grouped: the first level over (box, part) CTAs, the second one CTA per box,
// in the same order as a box's own reduction (job 0, kReduceCTAs parts)
__global__ void __launch_bounds__(kReduceThreads) k_reduce1_grp(GroupMap m, const ReduceBox* __restrict__ rb) {
  __shared__ double red[kMaxReduceK][kReduceThreads];
  unsigned b;
  const VB vb = vb_group(m, b);
  const ReduceBox R = rb[b];
  const ReduceJob J{R.rows, R.nblocks, kNSums, 0, kNSums, R.out};
  reduce1_body(J, vb.bx, kReduceCTAs, R.scratch + (size_t)vb.bx * kMaxReduceK, red);
}
__global__ void __launch_bounds__(kReduceThreads) k_reduce2_grp(const ReduceBox* __restrict__ rb) {
  __shared__ double red[kMaxReduceK][kReduceThreads];
  const ReduceBox R = rb[blockIdx.x];
  const ReduceJob J{R.rows, R.nblocks, kNSums, 0, kNSums, R.out};
  reduce2_body(J, R.scratch, kReduceCTAs, red);
}

cudaError_t launch_reduce_grp(const GroupMap& m1, const ReduceBox* rb, unsigned ctas1, unsigned nbox,
                              cudaStream_t st) {
  if (ctas1) k_reduce1_grp<<<ctas1, kReduceThreads, 0, st>>>(m1, rb);
  prof_mark("group.reduce1", st);
  if (nbox) k_reduce2_grp<<<nbox, kReduceThreads, 0, st>>>(rb);
  prof_mark("group.reduce2", st);
  return cudaGetLastError();
}

size_t reduce_scratch_bytes() { return (size_t)kMaxReduceJobs * kReduceCTAs * kMaxReduceK * sizeof(double); }

cudaError_t launch_reduce_fused(const ReduceJob& job, double* scratch, int* ticket, cudaStream_t st) {
  if (job.nk > kMaxReduceK) return cudaErrorInvalidValue;
  ReduceJobs jobs{};
  jobs.job[0] = job;
  launch_pdl(k_reduce_fused, kReduceCTAs, kReduceThreads, st, jobs, scratch, ticket);
  prof_mark("reduce", st);
  return cudaGetLastError();
}

}  // namespace vofgb
