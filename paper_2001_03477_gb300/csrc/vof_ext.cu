// vof_ext.cu -- velocity extension across the interface (Malan et al.,
// arXiv:2001.03477, Sec. 3.3.1: Eq. press_inv, the correction u~ and
// u_l = u^{n+1} + u~).
//
// The sub-domain is the mixed cells and the pure gas cells of the first two
// layers around them (layers across cell faces).  Faces to pure liquid cells
// and zero-gradient walls are no-slip (no flux of p~, u~ = 0); faces to gas
// cells beyond the second layer are free flow (p~ = 0 there).  In every
// sub-domain cell
//     sum_faces beta_f (p~_Q - p~_P) = mdot (1/rho_g - 1/rho_l) A / h,
// beta_f = (dt / rho_f) / h^2, rho_f = rho_l c_f + rho_g (1 - c_f) with c_f
// the mean of the two cells' c, A the PLIC plane area of a mixed cell (cell
// units; gas cells have no source).  The negated system is symmetric
// positive definite and is solved by conjugate gradients with the diagonal
// as preconditioner; then u~ = -(dt / rho_f) (p~_R - p~_L) / h on every face
// with a sub-domain cell on one side and no liquid cell or wall.
//
// Kernels: k_ext_init / k_ext_dilate (layer codes, full grid, 1 B per
// cell), k_ext_list (compact the unknowns), k_ext_assemble (the six
// couplings and the source of each unknown, CG start), the CG iterations,
// and k_ext_faces (the face correction, full face grid per axis).  The CG
// iterations run in one cooperative launch, k_ext_cg: its CTAs pass three
// grid barriers per iteration (after the matrix product, the update and the
// new direction) and test the residual every iteration on the device; where
// a cooperative launch of that size is refused, the same three phases run as
// the kernels k_ext_spmv, k_ext_update, k_ext_dir with a host test every 8
// iterations.  Inner products are per-CTA partial sums that every CTA adds
// up in the same fixed order, so all CTAs use the same scalars.
#include <algorithm>
#include <vector>

#include "../../include/vofgb.h"
#include "vof_launch.h"

namespace vofgb {

namespace {

constexpr uint8_t kOut = 255;  // pure liquid
constexpr uint8_t kGas = 254;  // pure gas beyond the layers reached so far
constexpr int kExtThreads = 256;    // grid-wide cell and face kernels
constexpr int kSolveThreads = 256;   // the CG kernels: one CTA per SM (few warps per FP64 sum tree)
constexpr int kExtCTAs = 152;
constexpr int kNoNb = -1;       // no-slip face (liquid cell or wall)
constexpr int kFreeNb = -2;     // free-flow face (p~ = 0 beyond)

// face neighbour of (x, y, z) along `axis` in direction d (+-1): false
// across a zero-gradient wall
__device__ __forceinline__ bool face_nb(const GridDev& g, int x, int y, int z, int axis, int d, int& qx, int& qy,
                                        int& qz) {
  qx = x; qy = y; qz = z;
  int& p = axis == 0 ? qx : (axis == 1 ? qy : qz);
  const int n = g.n[axis];
  p += d;
  if (p < 0 || p >= n) {
    if (g.bc[axis] != 0) return false;
    p = p < 0 ? p + n : p - n;
  }
  return true;
}

__device__ __forceinline__ size_t cid(const GridDev& g, int x, int y, int z) {
  return ((size_t)z * g.n[1] + y) * g.n[0] + x;
}

__device__ __forceinline__ bool is_gas_b(double c, const GridDev& g) { return dbits(c) <= g.eps_bits; }

__global__ void k_ext_init(GridDev g, const double* __restrict__ c, uint8_t* __restrict__ code, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const double cv = __ldg(c + i);
    code[i] = is_mixed_b(cv, g) ? (uint8_t)0 : (is_gas_b(cv, g) ? kGas : kOut);
  }
}

// gas cells next (across a face) to layer L - 1 join layer L
__global__ void k_ext_dilate(GridDev g, uint8_t* __restrict__ code, int L, size_t N) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    if (code[i] != kGas) continue;
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    bool hit = false;
    for (int axis = 0; axis < 3 && !hit; ++axis)
      for (int d = -1; d <= 1 && !hit; d += 2) {
        int qx, qy, qz;
        if (face_nb(g, x, y, z, axis, d, qx, qy, qz) && code[cid(g, qx, qy, qz)] == (uint8_t)(L - 1)) hit = true;
      }
    if (hit) code[i] = (uint8_t)L;
  }
}

__device__ __forceinline__ void warp_append_ext(bool take, uint32_t v, uint32_t* list, int* counter, int* slot) {
  const unsigned mask = __ballot_sync(0xffffffffu, take);
  *slot = -1;
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (take) {
    *slot = base + __popc(mask & ((1u << lane) - 1u));
    list[*slot] = v;
  }
}

// the unknowns: every sub-domain cell (layer 0, 1, 2), and the map from
// cells to unknowns (-1 outside)
__global__ void k_ext_list(const uint8_t* __restrict__ code, uint32_t* __restrict__ list, int* __restrict__ map,
                           int* __restrict__ counter, size_t N) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t n_iter = (N + stride - 1) / stride;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t it = 0; it < n_iter; ++it, i += stride) {
    const bool take = i < N && code[i] <= 2;
    int slot;
    warp_append_ext(take, (uint32_t)i, list, counter, &slot);
    if (i < N) map[i] = slot;
  }
}

// area of the plane m . x = alpha inside the unit cube: the cut polygon
// projected on the coordinate plane normal to m's largest component,
// vertices ordered by angle about their mean, shoelace area, divided by
// that component of the unit normal
__device__ double cut_area(const double m[3], double alpha) {
  double px[24], py[24];
  const double am0 = fabs(m[0]), am1 = fabs(m[1]), am2 = fabs(m[2]);
  const int dom = (am0 >= am1 && am0 >= am2) ? 0 : (am1 >= am2 ? 1 : 2);
  const int ia = dom == 0 ? 1 : 0, ib = dom == 2 ? 1 : 2;
  int np = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3;
    for (int u = 0; u < 2; ++u)
      for (int v = 0; v < 2; ++v) {
        double p0[3], p1[3];
        p0[ax] = 0.0; p0[b1] = u; p0[b2] = v;
        p1[ax] = 1.0; p1[b1] = u; p1[b2] = v;
        const double f0 = (m[0] * p0[0] + m[1] * p0[1] + m[2] * p0[2]) - alpha;
        const double f1 = (m[0] * p1[0] + m[1] * p1[1] + m[2] * p1[2]) - alpha;
        if (f0 == 0.0 && np < 24) { px[np] = p0[ia]; py[np] = p0[ib]; ++np; }
        if (f1 == 0.0 && np < 24) { px[np] = p1[ia]; py[np] = p1[ib]; ++np; }
        if (((f0 < 0.0 && f1 > 0.0) || (f0 > 0.0 && f1 < 0.0)) && np < 24) {
          const double t = f0 / (f0 - f1);
          double q[3] = {p0[0], p0[1], p0[2]};
          q[ax] = t;
          px[np] = q[ia]; py[np] = q[ib]; ++np;
        }
      }
  }
  if (np < 3) return 0.0;
  double cx = 0.0, cy = 0.0;
  for (int q = 0; q < np; ++q) { cx += px[q]; cy += py[q]; }
  cx /= np; cy /= np;
  double ang[24];
  for (int q = 0; q < np; ++q) ang[q] = atan2(py[q] - cy, px[q] - cx);
  for (int a = 1; a < np; ++a) {  // insertion sort by angle
    const double ka = ang[a], kx = px[a], ky = py[a];
    int b = a - 1;
    while (b >= 0 && ang[b] > ka) {
      ang[b + 1] = ang[b]; px[b + 1] = px[b]; py[b + 1] = py[b];
      --b;
    }
    ang[b + 1] = ka; px[b + 1] = kx; py[b + 1] = ky;
  }
  double s = 0.0;
  for (int q = 0; q < np; ++q) {
    const int r = q + 1 == np ? 0 : q + 1;
    s += (px[q] - cx) * (py[r] - cy) - (px[r] - cx) * (py[q] - cy);
  }
  const double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  const double nd = fabs(m[dom]) / len;
  return 0.5 * fabs(s) / nd;
}

// Fixed-order sums of the per-CTA partials (the same values in every CTA):
// warp 0 alone, each lane its partials lane, lane + 32, ... in order, then a
// shuffle tree; K sums at once (one barrier).  L2: the partials were written
// by other CTAs of the same launch, so the loads skip L1 (not coherent
// across SMs).
template <int K, bool L2>
__device__ __forceinline__ void sum_partials_k(const double* const (&part)[K], int n, double (&out)[K]) {
  __shared__ double res[K];
  __syncthreads();  // res may still be read from the previous call
  if (threadIdx.x < 32) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    for (int i = threadIdx.x; i < n; i += 32)
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += L2 ? __ldcg(part[k] + i) : part[k][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; ++k) res[k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = res[k];
}
// The same sums in warp 0 alone (valid in its lane 0), for a scalar step
// that lane 0 takes before sharing the result.
template <int K, bool L2>
__device__ __forceinline__ void warp0_sums(const double* const (&part)[K], int n, double (&out)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = 0.0;
  for (int i = threadIdx.x; i < n; i += 32)
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] += L2 ? __ldcg(part[k] + i) : part[k][i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] += __shfl_down_sync(0xffffffffu, out[k], o);
}

// A CTA's partial sums of K values in a fixed order (the threads' values
// staged in shared memory; warp 0 sums them, each lane its entries lane,
// lane + 32, ... in order, then a shuffle tree: few FP64 instructions per
// value), written to out[k][blockIdx.x].
template <int K>
__device__ __forceinline__ void block_partial_k(const double (&v)[K], double* const (&out)[K]) {
  __shared__ double red[K][kSolveThreads];
  __syncthreads();  // red may still be read from the previous call
#pragma unroll
  for (int k = 0; k < K; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    double x[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      x[k] = 0.0;
      for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) x[k] += red[k][i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < K; ++k) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; ++k) out[k][blockIdx.x] = x[k];
  }
}
__device__ __forceinline__ void block_partial(double v, double* __restrict__ out) {
  const double vv[1] = {v};
  double* const o[1] = {out};
  block_partial_k<1>(vv, o);
}

struct ExtVec {
  int* nb;        // [6 n]: neighbour unknown, kNoNb, or kFreeNb
  double* beta;   // [6 n]
  double* diag;   // [n]
  double* rdiag;  // [n]: 1 / diag (0 where diag is 0), the Jacobi preconditioner
  double* x;      // p~
  double* r;
  double* d;
  double* d2;     // the cooperative solver's second direction buffer (the two take turns)
  double* q;
  double* part;   // [5][kExtCTAs]: b.b, r.z (two, alternating), d.q, r.r
  int* counters;  // [0] unknowns, [1] free-flow faces
};

__global__ void __launch_bounds__(kExtThreads)  // (heavy per unknown: no register cap)
k_ext_assemble(GridDev g, double h, double dt, double rho_l, double rho_g, const double* __restrict__ c,
               const double* __restrict__ mdot, const uint8_t* __restrict__ code, const int* __restrict__ map,
               const uint32_t* __restrict__ list, ExtVec v, unsigned char* __restrict__ cg_state) {
  const int n = v.counters[0];
  if (blockIdx.x == 0 && threadIdx.x < 32) reinterpret_cast<unsigned long long*>(cg_state)[threadIdx.x] = 0ull;
  double bb = 0.0, rz = 0.0;
  int free_faces = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t id = list[i];
    int x, y, z;
    cell_xyz(g, id, x, y, z);
    const double cp = __ldg(c + id);
    double dsum = 0.0;
    for (int f = 0; f < 6; ++f) {
      const int axis = f >> 1, dir = (f & 1) ? 1 : -1;
      int qx, qy, qz;
      int nb = kNoNb;
      double beta = 0.0;
      if (face_nb(g, x, y, z, axis, dir, qx, qy, qz)) {
        const size_t qid = cid(g, qx, qy, qz);
        const uint8_t qc = code[qid];
        if (qc != kOut) {
          const double cf = 0.5 * (cp + __ldg(c + qid));
          const double rho = rho_l * cf + rho_g * (1.0 - cf);
          beta = (dt / rho) / (h * h);
          nb = qc <= 2 ? map[qid] : kFreeNb;
          if (nb == kFreeNb) ++free_faces;
        }
      }
      v.nb[6 * (size_t)i + f] = nb;
      v.beta[6 * (size_t)i + f] = beta;
      dsum += beta;
    }
    double rhs = 0.0;
    if (code[id] == 0) {
      double s[27];
      for (int oz = 0; oz < 3; ++oz)
        for (int oy = 0; oy < 3; ++oy)
          for (int ox = 0; ox < 3; ++ox)
            s[(oz * 3 + oy) * 3 + ox] = __ldg(c + cid(g, map_idx(x + ox - 1, g.n[0], g.bc[0]),
                                                        map_idx(y + oy - 1, g.n[1], g.bc[1]),
                                                        map_idx(z + oz - 1, g.n[2], g.bc[2])));
      double m[3];
      myc_normal(s, m);
      const double al = plane_alpha(m[0], m[1], m[2], cp);
      rhs = __ldg(mdot + id) * (1.0 / rho_g - 1.0 / rho_l) * cut_area(m, al) / h;
    }
    // M = -A: diagonal sum beta, off-diagonal -beta; b = -rhs
    const double b = -rhs;
    const double rd = dsum > 0.0 ? 1.0 / dsum : 0.0;
    v.diag[i] = dsum;
    v.rdiag[i] = rd;
    v.x[i] = 0.0;
    v.r[i] = b;
    const double zi = b * rd;
    v.d[i] = zi;
    bb = fma(b, b, bb);
    rz = fma(b, zi, rz);
  }
  if (free_faces) atomicAdd(v.counters + 1, free_faces);
  const double pv[2] = {bb, rz};
  double* const po[2] = {v.part, v.part + kExtCTAs};
  block_partial_k<2>(pv, po);
}

// The element arithmetic of one CG iteration (both forms of the solver use
// it): q = M d with its partial d . q; x += alpha d, r -= alpha q, z = r /
// diag with the partials r . z and r . r; d = z + beta d.
__device__ __forceinline__ double ext_spmv_elem(const ExtVec& v, int i, bool l2) {
  double q = v.diag[i] * v.d[i];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = v.nb[6 * (size_t)i + f];
    if (nb >= 0) q = fma(-v.beta[6 * (size_t)i + f], l2 ? __ldcg(v.d + nb) : v.d[nb], q);  // another CTA's
  }
  v.q[i] = q;
  return q;
}

// q = M d, partial d . q
__global__ void __launch_bounds__(kSolveThreads) k_ext_spmv(ExtVec v) {
  const int n = v.counters[0];
  double dq = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dq = fma(v.d[i], ext_spmv_elem(v, i, false), dq);
  block_partial(dq, v.part + 3 * kExtCTAs);
}

// alpha = r.z / d.q; x += alpha d; r -= alpha q; partial r.z (new) and r.r
__device__ __forceinline__ void ext_update_elems(const ExtVec& v, int n, double alpha, double& rzn, double& rr) {
  rzn = 0.0;
  rr = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v.x[i] = fma(alpha, v.d[i], v.x[i]);
    const double r = fma(-alpha, v.q[i], v.r[i]);
    v.r[i] = r;
    rzn = fma(r, r * v.rdiag[i], rzn);
    rr = fma(r, r, rr);
  }
}
__global__ void __launch_bounds__(kSolveThreads) k_ext_update(ExtVec v, int cur) {
  const double* pp[2] = {v.part + (1 + cur) * kExtCTAs, v.part + 3 * kExtCTAs};
  double s2[2];
  sum_partials_k<2, false>(pp, kExtCTAs, s2);
  const double alpha = s2[1] > 0.0 ? s2[0] / s2[1] : 0.0;
  double rzn, rr;
  ext_update_elems(v, v.counters[0], alpha, rzn, rr);
  const double pv[2] = {rzn, rr};
  double* const po[2] = {v.part + (2 - cur) * kExtCTAs, v.part + 4 * kExtCTAs};
  block_partial_k<2>(pv, po);
}

// d = z + (r.z new / r.z old) d
__device__ __forceinline__ void ext_dir_elems(const ExtVec& v, int n, double beta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v.d[i] = fma(beta, v.d[i], v.r[i] * v.rdiag[i]);
}
__global__ void __launch_bounds__(kSolveThreads) k_ext_dir(ExtVec v, int cur) {
  const double* pp[2] = {v.part + (1 + cur) * kExtCTAs, v.part + (2 - cur) * kExtCTAs};
  double s2[2];
  sum_partials_k<2, false>(pp, kExtCTAs, s2);
  const double beta = s2[0] > 0.0 ? s2[1] / s2[0] : 0.0;
  ext_dir_elems(v, v.counters[0], beta);
}

// Device state of the persistent solver (in the workspace; the assemble
// kernel clears it).
constexpr int kBarGroup = 32;  // CTAs per first-level arrival counter
struct ExtCG {
  unsigned arrive;  // grid barrier: groups arrived at the current barrier
  unsigned gen;     // grid barrier: barriers completed
  int iters;        // iterations done
  int flag;         // 1 converged, 2 iteration limit, 3 a barrier wait gave up
  double res;       // |r| at the end
  unsigned sub[(kExtCTAs + kBarGroup - 1) / kBarGroup];  // CTAs arrived, per group
};
static_assert(sizeof(ExtCG) <= 256, "the solver state lives in 256 bytes of the workspace");

__device__ __forceinline__ unsigned long long ext_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch (all CTAs resident): each CTA
// arrives on its group's counter, the last of a group on the top counter,
// and the last group starts the next generation (two short chains of
// atomics instead of one of all CTAs).  The wait is bounded (1 s): on
// expiry the CTA records DEV_WAIT and returns false, and the solver stops.
__device__ __forceinline__ bool ext_grid_barrier(ExtCG* cg, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = &cg->gen;
    const unsigned g0 = *vgen;
    __threadfence();  // this CTA's writes, and g0, before its arrival
    const unsigned grp = blockIdx.x / kBarGroup, ngrp = (gridDim.x + kBarGroup - 1) / kBarGroup;
    const unsigned gsize = min((unsigned)kBarGroup, gridDim.x - grp * kBarGroup);
    bool last = false;
    if (atomicAdd(&cg->sub[grp], 1u) == gsize - 1) {
      atomicExch(&cg->sub[grp], 0u);
      __threadfence();
      last = atomicAdd(&cg->arrive, 1u) == ngrp - 1;
    }
    if (last) {
      atomicExch(&cg->arrive, 0u);
      __threadfence();
      atomicAdd(&cg->gen, 1u);
    } else {
      const unsigned long long t0 = ext_now_ns();
      while (*vgen == g0) {
        if (ext_now_ns() - t0 > 1000000000ull) {
          ok = 0;
          if (status) atomicOr(status, DEV_WAIT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();  // the other CTAs' writes before this CTA reads them
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The CG iterations in one launch, two grid barriers per iteration: the
// direction d_k = z_k + beta_k d_(k-1) (d_0 = z_0) is formed where the
// matrix product needs it -- each thread its own elements, written to the
// other of two buffers, and the neighbours' again from their r and previous
// d, the same arithmetic, so the values are the owners' -- and the product,
// its partial d . q, then (after a barrier) alpha, x += alpha d, r -=
// alpha q and the partials r . z, r . r (then a barrier) follow; beta and
// |r| are formed from those partials at the top of the next iteration.  The
// same element arithmetic, partial slots and grid as k_ext_spmv,
// k_ext_update and k_ext_dir, so both forms of the solver give the same
// iterates.  The iteration's scalars are formed once per CTA by thread 0
// and shared; partials written by other CTAs are read from L2.
__global__ void __launch_bounds__(kSolveThreads)
k_ext_cg(ExtVec v, ExtCG* cg, double tol, int max_iter, int* status) {
  // [0] alpha, [1] beta, [2] r.z, [3] |r|, [4] target
  __shared__ double scal[5];
  const int n = v.counters[0];
  if (threadIdx.x < 32) {
    const double* pp[2] = {v.part, v.part + kExtCTAs};
    double s2[2];
    warp0_sums<2, true>(pp, kExtCTAs, s2);
    if (threadIdx.x == 0) {
      scal[2] = s2[1];
      scal[3] = sqrt(s2[0]);
      scal[4] = tol * scal[3];
    }
  }
  __syncthreads();
  double rz = scal[2];  // r.z, carried between phases
  double res = scal[3];
  const double target = scal[4];
  double* dcur = v.d;   // d_(k-1); d_0 itself in the first iteration
  double* dnew = v.d2;  // d_k
  int cur = 0, it = 0;
  bool ok = true;
  double beta = 0.0;
  while (res > target && it < max_iter) {  // the same values in every CTA
    const bool first = it == 0;
    // d_k and q = M d_k, partial d_k . q
    double dq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double di = first ? dcur[i] : fma(beta, dcur[i], v.r[i] * v.rdiag[i]);
      dnew[i] = di;
      double q = v.diag[i] * di;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int nb = v.nb[6 * (size_t)i + f];
        if (nb >= 0) {
          const double dn = first ? __ldcg(dcur + nb)
                                  : fma(beta, __ldcg(dcur + nb), __ldcg(v.r + nb) * __ldcg(v.rdiag + nb));
          q = fma(-v.beta[6 * (size_t)i + f], dn, q);
        }
      }
      v.q[i] = q;
      dq = fma(di, q, dq);
    }
    block_partial(dq, v.part + 3 * kExtCTAs);
    if (!(ok = ext_grid_barrier(cg, status))) break;
    // alpha = r.z / d.q; x += alpha d; r -= alpha q; partial r.z and r.r
    if (threadIdx.x < 32) {
      const double* pp[1] = {v.part + 3 * kExtCTAs};
      double dqs[1];
      warp0_sums<1, true>(pp, kExtCTAs, dqs);
      if (threadIdx.x == 0) scal[0] = dqs[0] > 0.0 ? rz / dqs[0] : 0.0;
    }
    __syncthreads();
    {
      const double alpha = scal[0];
      double rzn = 0.0, rr = 0.0;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        v.x[i] = fma(alpha, dnew[i], v.x[i]);
        const double r = fma(-alpha, v.q[i], v.r[i]);
        v.r[i] = r;
        rzn = fma(r, r * v.rdiag[i], rzn);
        rr = fma(r, r, rr);
      }
      const double pv[2] = {rzn, rr};
      double* const po[2] = {v.part + (2 - cur) * kExtCTAs, v.part + 4 * kExtCTAs};
      block_partial_k<2>(pv, po);
    }
    if (!(ok = ext_grid_barrier(cg, status))) break;
    // beta = r.z new / r.z old, |r|
    if (threadIdx.x < 32) {
      const double* pp[2] = {v.part + (2 - cur) * kExtCTAs, v.part + 4 * kExtCTAs};
      double s2[2];
      warp0_sums<2, true>(pp, kExtCTAs, s2);
      if (threadIdx.x == 0) {
        scal[1] = rz > 0.0 ? s2[0] / rz : 0.0;
        scal[2] = s2[0];
        scal[3] = sqrt(s2[1]);
      }
    }
    __syncthreads();
    beta = scal[1];
    rz = scal[2];
    res = scal[3];
    double* t = dcur;  // the buffers take turns
    dcur = dnew;
    dnew = t;
    cur ^= 1;
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cg->iters = it;
    cg->res = res;
    cg->flag = !ok ? 3 : (res > target ? 2 : 1);
  }
}

// the face correction along AX over the whole face grid of that axis
template <int AX>
__global__ void __launch_bounds__(kExtThreads)
k_ext_faces(GridDev g, double h, double dt, double rho_l, double rho_g, const double* __restrict__ c,
            const uint8_t* __restrict__ code, const int* __restrict__ map, const double* __restrict__ x,
            double* __restrict__ uf, double* __restrict__ ut) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int fx = nx + (AX == 0), fy = ny + (AX == 1), fz = nz + (AX == 2);
  const size_t nf = (size_t)fx * fy * fz;
  const int n_ax = g.n[AX];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t ii = (uint32_t)i;
    int a = (int)(ii % (uint32_t)fx);
    const uint32_t rest = ii / (uint32_t)fx;
    int b = (int)(rest % (uint32_t)fy);
    int cc = (int)(rest / (uint32_t)fy);
    // face index f along AX, between cells f - 1 and f
    const int f = AX == 0 ? a : (AX == 1 ? b : cc);
    double val = 0.0;
    bool has = true;
    int fl = f - 1, fr = f;
    if (f == 0 || f == n_ax) {
      if (g.bc[AX] != 0) has = false;  // a wall: no-slip
      else { fl = n_ax - 1; fr = 0; }
    }
    if (has) {
      int lx = a, ly = b, lz = cc, rx = a, ry = b, rz = cc;
      if (AX == 0) { lx = fl; rx = fr; }
      else if (AX == 1) { ly = fl; ry = fr; }
      else { lz = fl; rz = fr; }
      const size_t L = cid(g, lx, ly, lz), R = cid(g, rx, ry, rz);
      const uint8_t cl = code[L], cr = code[R];
      if ((cl <= 2 || cr <= 2) && cl != kOut && cr != kOut) {
        const double pl = cl <= 2 ? x[map[L]] : 0.0;
        const double pr = cr <= 2 ? x[map[R]] : 0.0;
        const double cf = 0.5 * (__ldg(c + L) + __ldg(c + R));
        const double rho = rho_l * cf + rho_g * (1.0 - cf);
        val = -(dt / rho) * (pr - pl) / h;
      }
    }
    if (ut) ut[i] = val;
    if (uf) uf[i] += val;
  }
}

struct ExtLayout {
  size_t code, map, list, nb, beta, diag, rdiag, x, r, d, d2, q, part, counters, cg, total;
};

ExtLayout ext_layout(size_t N) {
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  ExtLayout L;
  size_t o = 0;
  L.code = o; o += a(N);
  L.map = o; o += a(N * 4);
  L.list = o; o += a(N * 4);
  L.nb = o; o += a(N * 6 * 4);
  L.beta = o; o += a(N * 6 * 8);
  L.diag = o; o += a(N * 8);
  L.rdiag = o; o += a(N * 8);
  L.x = o; o += a(N * 8);
  L.r = o; o += a(N * 8);
  L.d = o; o += a(N * 8);
  L.d2 = o; o += a(N * 8);
  L.q = o; o += a(N * 8);
  L.part = o; o += a(5 * kExtCTAs * 8);
  L.counters = o; o += a(4 * 4);
  L.cg = o; o += 256;
  L.total = o;
  return L;
}

}  // namespace

size_t ext_scratch_bytes(size_t N) { return ext_layout(N).total; }

cudaError_t launch_velocity_extension(const GridDev& g, double h, const double* c, const double* mdot, double rho_l,
                                      double rho_g, double dt, double tol, int max_iter, double* u, double* v,
                                      double* w, double* ut, double* vt, double* wt, void* workspace,
                                      cudaStream_t st, int* iters_out, double* res_out, int* status) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const ExtLayout L = ext_layout(N);
  char* ws = static_cast<char*>(workspace);
  uint8_t* code = reinterpret_cast<uint8_t*>(ws + L.code);
  int* map = reinterpret_cast<int*>(ws + L.map);
  uint32_t* list = reinterpret_cast<uint32_t*>(ws + L.list);
  ExtVec vec;
  vec.nb = reinterpret_cast<int*>(ws + L.nb);
  vec.beta = reinterpret_cast<double*>(ws + L.beta);
  vec.diag = reinterpret_cast<double*>(ws + L.diag);
  vec.rdiag = reinterpret_cast<double*>(ws + L.rdiag);
  vec.x = reinterpret_cast<double*>(ws + L.x);
  vec.r = reinterpret_cast<double*>(ws + L.r);
  vec.d = reinterpret_cast<double*>(ws + L.d);
  vec.d2 = reinterpret_cast<double*>(ws + L.d2);
  vec.q = reinterpret_cast<double*>(ws + L.q);
  vec.part = reinterpret_cast<double*>(ws + L.part);
  vec.counters = reinterpret_cast<int*>(ws + L.counters);
  *status = 0;
  cudaError_t err = cudaMemsetAsync(vec.counters, 0, 4 * sizeof(int), st);
  if (err != cudaSuccess) return err;
  const int grid_cells = (int)std::min<size_t>((N + kExtThreads - 1) / kExtThreads, (size_t)152 * 16);
  k_ext_init<<<grid_cells, kExtThreads, 0, st>>>(g, c, code, N);
  for (int layer = 1; layer <= 2; ++layer) k_ext_dilate<<<grid_cells, kExtThreads, 0, st>>>(g, code, layer, N);
  k_ext_list<<<grid_cells, kExtThreads, 0, st>>>(code, list, map, vec.counters, N);
  prof_mark("ext.layers", st);
  unsigned char* cg_state = reinterpret_cast<unsigned char*>(ws + L.cg);
  k_ext_assemble<<<kExtCTAs, kExtThreads, 0, st>>>(g, h, dt, rho_l, rho_g, c, mdot, code, map, list, vec, cg_state);
  prof_mark("ext.assemble", st);
  int host_counts[2] = {0, 0};
  err = cudaMemcpyAsync(host_counts, vec.counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return err;
  const int n = host_counts[0];
  std::vector<double> part(kExtCTAs);
  auto host_sum = [&](int slot, double* out) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(part.data(), vec.part + slot * kExtCTAs, kExtCTAs * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    double s = 0.0;
    for (int i = 0; i < kExtCTAs; ++i) s += part[i];
    *out = s;
    return e;
  };
  int it = 0;
  double res = 0.0;
  bool n_done = false;  // solved by the cooperative launch
  if (n > 0) {
    if (host_counts[1] == 0) {
      *status = 1;  // nothing fixes p~
      return cudaSuccess;
    }
    // one cooperative launch when all kExtCTAs CTAs fit at once (the grid
    // barriers need them resident); else the three kernels per iteration
    int dev = 0, nsm = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ext_cg, kSolveThreads, 0) == cudaSuccess && coop &&
        (long long)per_sm * nsm >= kExtCTAs) {
      ExtCG* cg = reinterpret_cast<ExtCG*>(cg_state);
      int* dstat = device_status_ptr();
      void* args[] = {&vec, &cg, &tol, &max_iter, &dstat};
      err = cudaLaunchCooperativeKernel((const void*)k_ext_cg, dim3(kExtCTAs), dim3(kSolveThreads), args, 0, st);
      if (err != cudaSuccess) return err;
      prof_mark("ext.cg", st);
      ExtCG hcg{};
      err = cudaMemcpyAsync(&hcg, cg, sizeof(ExtCG), cudaMemcpyDeviceToHost, st);
      if (err == cudaSuccess) err = cudaStreamSynchronize(st);
      if (err != cudaSuccess) return err;
      it = hcg.iters;
      res = hcg.res;
      if (hcg.flag != 1) *status = 2;  // not converged (or a barrier wait gave up: DEV_WAIT is set)
      n_done = true;
    }
  }
  if (n > 0 && !n_done) {
    double bb = 0.0;
    err = host_sum(0, &bb);
    if (err != cudaSuccess) return err;
    const double target = tol * sqrt(bb);
    res = sqrt(bb);
    int cur = 0;
    while (res > target && it < max_iter) {
      k_ext_spmv<<<kExtCTAs, kSolveThreads, 0, st>>>(vec);
      k_ext_update<<<kExtCTAs, kSolveThreads, 0, st>>>(vec, cur);
      k_ext_dir<<<kExtCTAs, kSolveThreads, 0, st>>>(vec, cur);
      cur ^= 1;
      ++it;
      if (it % 8 == 0 || it == max_iter) {
        double rr = 0.0;
        err = host_sum(4, &rr);
        if (err != cudaSuccess) return err;
        res = sqrt(rr);
      }
    }
    prof_mark("ext.cg", st);
    if (res > target) *status = 2;  // not converged within max_iter
  }
  k_ext_faces<0><<<grid_cells, kExtThreads, 0, st>>>(g, h, dt, rho_l, rho_g, c, code, map, vec.x, u, ut);
  k_ext_faces<1><<<grid_cells, kExtThreads, 0, st>>>(g, h, dt, rho_l, rho_g, c, code, map, vec.x, v, vt);
  k_ext_faces<2><<<grid_cells, kExtThreads, 0, st>>>(g, h, dt, rho_l, rho_g, c, code, map, vec.x, w, wt);
  prof_mark("ext.faces", st);
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = res;
  return cudaGetLastError();
}

}  // namespace vofgb
