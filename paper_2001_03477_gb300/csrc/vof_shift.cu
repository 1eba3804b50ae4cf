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
// Shift in four kernels.
//   stream:    copies c, e to the output and sums them; lists the moving
//              mixed cells per warp (256 consecutive cells per warp, fixed
//              order) and appends them to a grid-wide list, cells with c
//              within 1e-3 of 0 or 1 ("edge" cells, whose plane constant
//              takes the bisection) at its back, the others at its front;
//   planes:    one moving mixed cell per thread over the grid-wide list:
//              plane (MYC normal + plane constant), shift |m|_2 dd, the
//              cell's own shifted volume, and the receivers it settles --
//              pure neighbours of the receding phase whose first reaching
//              neighbour (scan order z outer, x inner) it is;
//   receivers: one receiver per thread: the largest volume swept in it by
//              the extended planes of its reaching neighbours;
//   sums:      per warp list in fixed order, the changes of every moving
//              cell and of the receivers it settled, so the sums do not
//              depend on the order of the grid-wide lists.
// ---------------------------------------------------------------------------
constexpr int kWarpCells = 256;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kListThreads = 128;     // planes / receivers kernels: CTA size
constexpr int kListCTAs = 152 * 4;    // and grid (grid-stride loops)

__device__ __forceinline__ void decode(const GridDev& g, size_t id, int& x, int& y, int& z) {
  x = (int)(id % (size_t)g.n[0]);
  const size_t r = id / (size_t)g.n[0];
  y = (int)(r % (size_t)g.n[1]);
  z = (int)(r / (size_t)g.n[1]);
}

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

// moving mixed cell whose shift has the sign that reaches a receiver of this kind
__device__ __forceinline__ bool reaches(const GridDev& g, const double* __restrict__ c_in,
                                        const double* __restrict__ dd, double dd_uniform, size_t q, bool full) {
  if (!is_mixed_b(__ldg(c_in + q), g)) return false;
  const double ddv = dd ? __ldg(dd + q) : dd_uniform;
  return dnz(ddv) && (dlt0(ddv) == full);
}

// offsets as bit indices: ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1), 0..26
__device__ __forceinline__ int offset_bit(int ox, int oy, int oz) { return ((oz + 1) * 3 + (oy + 1)) * 3 + (ox + 1); }

__global__ void __launch_bounds__(256)
k_shift_stream(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
               double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, ShiftScratch sc,
               SumOut sums) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const size_t w = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  uint32_t* list = sc.list + w * kWarpCells;
  int n = 0, ne = 0;
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
    const unsigned m = __ballot_sync(kFullMask, moving);
    if (moving) list[n + __popc(m & lt)] = (uint32_t)id;
    n += __popc(m);
    ne += __popc(__ballot_sync(kFullMask, moving && edge_cell(c)));
  }
  if (lane == 0 && (long long)w * kWarpCells < (long long)N) sc.count[w] = n;
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
      const bool v = j < n;
      const uint32_t id = v ? list[j] : 0u;
      const bool edge = v && edge_cell(__ldg(c_in + id));
      const unsigned me = __ballot_sync(kFullMask, edge), mn = __ballot_sync(kFullMask, v && !edge);
      if (edge) sc.gmix[N - 1 - (size_t)(be + __popc(me & lt))] = id;
      else if (v) sc.gmix[bn + __popc(mn & lt)] = id;
      be += __popc(me);
      bn += __popc(mn);
    }
  }
  block_sums_sh<5>(acc, sums, blockIdx.x);
}

__global__ void __launch_bounds__(kListThreads)
k_shift_planes(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in, double* __restrict__ c_out,
               double* __restrict__ e_out, const double* __restrict__ dd, double dd_uniform, ShiftScratch sc) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const int nn = sc.counters[0], ne = sc.counters[1];
  const int lane = threadIdx.x & 31;
  const int total = nn + ne;
  // whole warps iterate together (the receiver append below is warp-wide)
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < total; i0 += stride) {
    const int i = i0 + lane;
    const bool v = i < total;
    unsigned own = 0u;
    int x = 0, y = 0, z = 0;
    if (v) {
      const size_t id = i < nn ? sc.gmix[i] : sc.gmix[N - 1 - (size_t)(i - nn)];
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
      const double al = edge_cell(ct) ? plane_alpha_bisect(m[0], m[1], m[2], ct) : plane_alpha(m[0], m[1], m[2], ct);
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
        c_out[id] = cn;
        e_out[id] = __ldg(e_in + id) + (cn - ct) * (g.Cp_l - g.Cp_g) * g.T_sat;
      }
      // receivers this cell settles
      const bool full = dlt0(ddv);  // the kind of pure cell this shift reaches
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            if (!ox && !oy && !oz) continue;
            size_t pid;
            if (!neighbour(g, x, y, z, ox, oy, oz, pid)) continue;
            const double cp = __ldg(c_in + pid);
            if (is_mixed_b(cp, g) || is_full_b(cp, g) != full) continue;
            int px, py, pz;
            decode(g, pid, px, py, pz);
            int first = -1;
            for (int rz = -1; rz <= 1 && first < 0; ++rz)
              for (int ry = -1; ry <= 1 && first < 0; ++ry)
                for (int rx = -1; rx <= 1 && first < 0; ++rx) {
                  if (!rx && !ry && !rz) continue;
                  size_t sid;
                  if (!neighbour(g, px, py, pz, rx, ry, rz, sid)) continue;
                  if (reaches(g, c_in, dd, dd_uniform, sid, full)) first = offset_bit(rx, ry, rz);
                }
            // on periodic axes of 1 or 2 cells several offsets lead to the
            // same cell; only the offset back to this cell settles it
            if (first == offset_bit(-ox, -oy, -oz)) own |= 1u << offset_bit(ox, oy, oz);
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
k_shift_receivers(GridDev g, const double* __restrict__ c_in, const double* __restrict__ e_in,
                  double* __restrict__ c_out, double* __restrict__ e_out, const double* __restrict__ dd,
                  double dd_uniform, ShiftScratch sc) {
  const int nr = sc.counters[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
    const size_t pid = sc.recv[i];
    const double cp = __ldg(c_in + pid);
    const bool full = is_full_b(cp, g);
    int px, py, pz;
    decode(g, pid, px, py, pz);
    double best = 0.0;
    for (int rz = -1; rz <= 1; ++rz)
      for (int ry = -1; ry <= 1; ++ry)
        for (int rx = -1; rx <= 1; ++rx) {
          if (!rx && !ry && !rz) continue;
          size_t sid;
          if (!neighbour(g, px, py, pz, rx, ry, rz, sid)) continue;
          if (!reaches(g, c_in, dd, dd_uniform, sid, full)) continue;
          const double sft = sc.shift[sid];
          if (!dnz(sft)) continue;  // a zero normal does not move
          const double4 pl = reinterpret_cast<const double4*>(sc.plane)[sid];
          const double m0 = pl.x, m1 = pl.y, m2 = pl.z, al = pl.w;
          // the receiver sits at offset -(rx, ry, rz) from the source
          const double shiftv = -((m0 * (double)(-rx) + m1 * (double)(-ry)) + m2 * (double)(-rz));
          const double a_old = al + shiftv;
          const double a_new = (al + sft) + shiftv;
          double lo = 0.0, hi = 0.0;
          if (m0 < 0.0) lo += m0; else hi += m0;
          if (m1 < 0.0) lo += m1; else hi += m1;
          if (m2 < 0.0) lo += m2; else hi += m2;
          // the extended plane stays outside the receiver: both volumes are
          // exactly 1 (or 0); the margin clears the rounding of that test
          if (full ? (a_new >= hi + 1e-9) : (a_new <= lo - 1e-9)) continue;
          const double sw = volume(m0, m1, m2, a_new) - volume(m0, m1, m2, a_old);
          if (fabs(sw) > fabs(best)) best = sw;
        }
    sc.sweep[pid] = best;
    if (dnz(best)) {
      const double v = cp + best;
      const double vc = dlt0(v) ? 0.0 : (dgt1(v) ? 1.0 : v);
      if (!same_bits_dev(vc, cp)) {
        c_out[pid] = vc;
        e_out[pid] = __ldg(e_in + pid) + (vc - cp) * (g.Cp_l - g.Cp_g) * g.T_sat;
      }
    }
  }
}

__global__ void __launch_bounds__(256)
k_shift_sums(GridDev g, const double* __restrict__ c_in, const double* __restrict__ c_out, ShiftScratch sc,
             long long nwarps, SumOut sums) {
  const int lane = threadIdx.x & 31;
  const size_t w = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if ((long long)w < nwarps) {
    const int cnt = sc.count[w];
    const uint32_t* list = sc.list + w * kWarpCells;
    for (int i = lane; i < cnt; i += 32) {
      const size_t qid = list[i];
      const double dq = c_out[qid] - __ldg(c_in + qid);
      acc[0] += dq;
      acc[2] += dq * (g.Cp_l - g.Cp_g) * g.T_sat;
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
        const double cp = __ldg(c_in + pid);
        const double v = cp + best;
        const double vc = dlt0(v) ? 0.0 : (dgt1(v) ? 1.0 : v);
        if (!deq(v, vc)) acc[1] += v - vc;
        const double dc = vc - cp;
        acc[0] += dc;
        acc[2] += dc * (g.Cp_l - g.Cp_g) * g.T_sat;
      }
    }
  }
  acc[3] = acc[0];  // sum c_out = sum c_in + sum dc
  acc[4] = acc[2];
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

// CTAs of the stream and sums kernels (8 warps of 256 cells)
int shift_blocks(const GridDev& g) { return (int)((shift_warps(g) + 7) / 8); }

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t shift_scratch_bytes(const GridDev& g) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_blocks(g) * 8;
  return al256(nw * kWarpCells * 4)  // per-warp lists
         + al256(nw * 4)             // counts
         + 256                       // counters
         + al256(N * 4)              // grid-wide list of moving cells
         + al256(N * 4)              // receivers
         + al256(N * 32)             // planes
         + al256(N * 8)              // shifts
         + al256(N * 8)              // sweeps
         + al256(N * 4);             // settled-receiver masks
}

ShiftScratch carve_shift_scratch(const GridDev& g, void* ws) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const size_t nw = (size_t)shift_blocks(g) * 8;
  char* b = static_cast<char*>(ws);
  ShiftScratch s;
  s.list = reinterpret_cast<uint32_t*>(b);   b += al256(nw * kWarpCells * 4);
  s.count = reinterpret_cast<int*>(b);       b += al256(nw * 4);
  s.counters = reinterpret_cast<int*>(b);    b += 256;
  s.gmix = reinterpret_cast<uint32_t*>(b);   b += al256(N * 4);
  s.recv = reinterpret_cast<uint32_t*>(b);   b += al256(N * 4);
  s.plane = reinterpret_cast<double*>(b);    b += al256(N * 32);
  s.shift = reinterpret_cast<double*>(b);    b += al256(N * 8);
  s.sweep = reinterpret_cast<double*>(b);    b += al256(N * 8);
  s.own = reinterpret_cast<uint32_t*>(b);
  return s;
}

cudaError_t launch_shift(const GridDev& g, const double* c_in, const double* e_in, double* c_out, double* e_out,
                         const double* dd, double dd_uniform, uint8_t* state, ShiftScratch sc, SumOut sums,
                         cudaStream_t st) {
  const long long nw = shift_warps(g);
  const unsigned nb = (unsigned)shift_blocks(g);
  // the stream and sums kernels write partials to consecutive sets of nb CTAs
  SumOut s0 = sums, s1 = sums;
  if (sums.partials) s1.partials = sums.partials + (size_t)nb * sums.stride;
  cudaError_t err = cudaMemsetAsync(sc.counters, 0, 3 * sizeof(int), st);
  if (err != cudaSuccess) return err;
  k_shift_stream<<<nb, 256, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc, s0);
  k_shift_planes<<<kListCTAs, kListThreads, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc);
  k_shift_receivers<<<kListCTAs, kListThreads, 0, st>>>(g, c_in, e_in, c_out, e_out, dd, dd_uniform, sc);
  k_shift_sums<<<nb, 256, 0, st>>>(g, c_in, c_out, sc, nw, s1);
  err = cudaGetLastError();
  if (err == cudaSuccess && state) err = cudaMemsetAsync(state, 0, (size_t)g.n[0] * g.n[1] * g.n[2], st);
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
