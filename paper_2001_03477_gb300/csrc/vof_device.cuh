// vof_device.cuh -- device-side PLIC geometry, MYC normal and WENO5 face
// value for the GB300 library (sm_103a).  Method: Malan et al.,
// arXiv:2001.03477, Sec. 3.2 (PLIC: MYC normal, plane constant from the
// volume), Sec. 3.3 (geometric face fluxes), Sec. 3.4.1 (WENO5 face
// temperature).
//
// The library is compiled with -fmad=false: every expression below rounds
// each operation separately, in the order written, so that discrete
// decisions (which normal candidate wins, which cells are mixed, which
// face value shortcut applies) are taken on exactly the same numbers on any
// path that evaluates them.  Where a fused multiply-add is wanted it is
// written as fma().
#pragma once
#include <cstdint>

#include "vof_df.cuh"

namespace vofgb {

// ---------------------------------------------------------------------------
// Problem description passed to kernels by value
// ---------------------------------------------------------------------------
struct GridDev {
  int n[3];      // nx, ny, nz
  int bc[3];     // 0 periodic, 1 zero-gradient
  double lam;    // dt / h
  double Cp_l, Cp_g, T_sat, eps;
  long long eps_bits;     // bit pattern of eps
  long long one_m_eps;    // bit pattern of 1 - eps
  int f32;                // precision form: FP32 reconstruction and flux weights in the sweeps
  int le;                 // Lagrangian-explicit sweeps (Li's scheme) instead of Weymouth-Yue
  double rCp_l, rCp_g;    // 1 / Cp_l, 1 / Cp_g (T of pure cells by a multiply)
  int mlp;                // normal of the sweeps' reconstruction: 0 MYC, 1 learned
                          // (with MYC fallback), 2 Youngs
  const void* mlp_params; // packed network parameters (device)
};

// ---------------------------------------------------------------------------
// Comparisons on the integer pipe.  On this part FP64 compares issue on the
// FP64 unit (1/64 of the FP32 rate); the bit-pattern forms below give the
// same answer as the IEEE comparison for every non-NaN operand (and the same
// decision for the mixed-cell test with NaN), so decisions agree with the
// oracle's double compares.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// a == b (IEEE: +0 == -0)
__device__ __forceinline__ bool deq(double a, double b) {
  unsigned long long x = (unsigned long long)dbits(a), y = (unsigned long long)dbits(b);
  return x == y || ((x | y) << 1) == 0ull;
}
// a != 0 on the integer pipe.  The halves are taken with an opaque move: the
// one-word form ((bits << 1) != 0) is exactly an FP64 "not equal to zero"
// compare, and the compiler may emit it as one, which costs an FP64 unit
// slot (~80 cycles per warp) on this part.
__device__ __forceinline__ bool dnz(double a) {
  unsigned lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(a));
  return ((hi & 0x7fffffffu) | lo) != 0u;
}
__device__ __forceinline__ bool dgt0(double a) { return dbits(a) > 0; }
__device__ __forceinline__ bool dlt0(double a) { return dbits(a) < 0 && dnz(a); }
// a > 1.0
__device__ __forceinline__ bool dgt1(double a) { return dbits(a) > 0x3FF0000000000000LL; }
// a > 0.5
__device__ __forceinline__ bool dgthalf(double a) { return dbits(a) > 0x3FE0000000000000LL; }

// Exact scalings on the integer pipe, the same bits as the FP64 products
// (|x| < 2^1022).  2 x: a normal x by its exponent field, zero and subnormal
// x by a shift of the magnitude bits, which carries into the exponent field
// exactly as the product does.
__device__ __forceinline__ double dtwice(double x) {
  const unsigned long long b = (unsigned long long)dbits(x);
  const unsigned long long sg = b & 0x8000000000000000ull, mg = b & 0x7FFFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)((mg >> 52) ? b + (1ull << 52) : (sg | (mg << 1))));
}
// -x (the sign bit flipped)
__device__ __forceinline__ double dneg(double x) { return __longlong_as_double(dbits(x) ^ (long long)0x8000000000000000ull); }
// x / 2 where that is exact without rounding: x = 0, or the half a normal
// number (exponent field >= 2); ok = false otherwise (the caller multiplies)
__device__ __forceinline__ double dhalf_exact(double x, bool& ok) {
  const unsigned long long b = (unsigned long long)dbits(x);
  const unsigned e = (unsigned)((b >> 52) & 0x7FF);
  ok = e >= 2 || (b << 1) == 0ull;
  return __longlong_as_double((long long)(e >= 2 ? b - (1ull << 52) : b));
}

__device__ __forceinline__ int map_idx(int i, int n, int bc) {
  if (bc == 0) {
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

__device__ __forceinline__ double heat_cap(double Cp_l, double Cp_g, double c) {
  return Cp_l * c + Cp_g * (1.0 - c);
}

// T = e / C_p(c).  A pure cell (c exactly 0 or 1) multiplies by the
// phase's reciprocal heat capacity, within 2 ulps of the quotient, instead
// of dividing (an FP64 division costs ~10 FP64 instructions on this part);
// every kernel that needs T of a cell calls this one function, so equal
// (c, e) always give equal T.
__device__ __forceinline__ double temp_of(const GridDev& g, double e, double c) {
  const long long b = __double_as_longlong(c);
  if (b == 0x3FF0000000000000LL) return e * g.rCp_l;
  if (b == 0) return e * g.rCp_g;
  return e / heat_cap(g.Cp_l, g.Cp_g, c);
}

__device__ __forceinline__ bool is_mixed(double c, double eps) { return c > eps && c < 1.0 - eps; }
// the same test on the integer pipe (eps >= 0)
// cell coordinates of a cell index (grids hold fewer than 2^31 cells, so
// 32-bit division suffices; 64-bit division is a long software sequence)
__device__ __forceinline__ void cell_xyz(const GridDev& g, size_t id, int& x, int& y, int& z) {
  const uint32_t i = (uint32_t)id, nx = (uint32_t)g.n[0], ny = (uint32_t)g.n[1];
  const uint32_t r = i / nx;
  x = (int)(i - r * nx);
  const uint32_t q = r / ny;
  y = (int)(r - q * ny);
  z = (int)q;
}

__device__ __forceinline__ bool is_mixed_b(double c, const GridDev& g) {
  long long b = dbits(c);
  return b > g.eps_bits && b < g.one_m_eps;
}
__device__ __forceinline__ bool is_full_b(double c, const GridDev& g) { return dbits(c) >= g.one_m_eps; }

// ---------------------------------------------------------------------------
// Volume below a plane in the unit cube (Scardovelli & Zaleski 2000)
// ---------------------------------------------------------------------------
// sorted 0 <= m1 <= m2 <= m3, sum 1, 0 < a <= 1/2: inclusion-exclusion of the
// cube's corner terms, branch by branch, with the (a-m2)^3 and (a-m3)^3
// corrections kept bounded by m1 so nothing cancels catastrophically.
__device__ __forceinline__ double vol_low(double m1, double m2, double m3, double a) {
  double m12 = m1 + m2;
  if (a < m1) return a * a * a / (6.0 * m1 * m2 * m3);
  double v2 = a * (a - m1) / (2.0 * m2 * m3) + m1 * m1 / (6.0 * m2 * m3);
  if (a < m2) return v2;
  double t2 = a - m2;
  double v3 = v2 - t2 * t2 * t2 / (6.0 * m1 * m2 * m3);
  double top = m12 < m3 ? m12 : m3;
  if (a < top) return v3;
  if (m12 <= m3) return (2.0 * a - m12) / (2.0 * m3);
  double t3 = a - m3;
  return v3 - t3 * t3 * t3 / (6.0 * m1 * m2 * m3);
}

__device__ __forceinline__ void sort3(double& a, double& b, double& c) {
  double t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
}

// m >= 0, sum 1
__device__ __forceinline__ double vol_pos(double m0, double m1, double m2, double a) {
  if (a <= 0.0) return 0.0;
  if (a >= 1.0) return 1.0;
  sort3(m0, m1, m2);
  if (a <= 0.5) return vol_low(m0, m1, m2, a);
  return 1.0 - vol_low(m0, m1, m2, 1.0 - a);
}

struct Mirror {
  double mp[3];  // |m| / l1
  double sh;     // alpha_mirror = alpha + sh
  double l1;
};

__device__ __forceinline__ Mirror mirror_normalise(double m0, double m1, double m2) {
  Mirror r;
  double sh = 0.0;
  double a0, a1, a2;
  if (m0 < 0.0) { a0 = -m0; sh -= m0; } else a0 = m0;
  if (m1 < 0.0) { a1 = -m1; sh -= m1; } else a1 = m1;
  if (m2 < 0.0) { a2 = -m2; sh -= m2; } else a2 = m2;
  double s = a0 + a1 + a2;
  r.sh = sh;
  r.l1 = s;
  if (s > 0.0) { a0 /= s; a1 /= s; a2 /= s; }
  r.mp[0] = a0; r.mp[1] = a1; r.mp[2] = a2;
  return r;
}

// liquid fraction of {x in [0,1]^3 : m.x <= alpha}, any m
__device__ __forceinline__ double volume(double m0, double m1, double m2, double alpha) {
  Mirror r = mirror_normalise(m0, m1, m2);
  if (r.l1 == 0.0) return alpha >= 0.0 ? 1.0 : 0.0;
  return vol_pos(r.mp[0], r.mp[1], r.mp[2], (alpha + r.sh) / r.l1);
}

// derivative dV/da on the same branches (for the Newton polish)
__device__ __forceinline__ double dvol_low(double m1, double m2, double m3, double a) {
  double m12 = m1 + m2;
  if (a < m1) return a * a / (2.0 * m1 * m2 * m3);
  double d2 = (2.0 * a - m1) / (2.0 * m2 * m3);
  if (a < m2) return d2;
  double t2 = a - m2;
  double d3 = d2 - t2 * t2 / (2.0 * m1 * m2 * m3);
  double top = m12 < m3 ? m12 : m3;
  if (a < top) return d3;
  if (m12 <= m3) return 1.0 / m3;
  double t3 = a - m3;
  return d3 - t3 * t3 / (2.0 * m1 * m2 * m3);
}

// Plane constant for sorted m (sum 1) and 0 < c <= 1/2, analytic per branch
// (Scardovelli & Zaleski 2000): cube root, quadratic, linear, or the
// trigonometric root of the branch cubic; then one safeguarded Newton step.
static __device__ __noinline__ double alpha_low_analytic(double m1, double m2, double m3, double c) {
  double m12 = m1 + m2;
  double P6 = 6.0 * m1 * m2 * m3;
  double V1 = (m1 > 0.0) ? m1 * m1 / (6.0 * m2 * m3) : 0.0;
  double V2 = V1 + (m2 - m1) / (2.0 * m3);
  double a, lo, hi;
  if (c < V1) {
    a = cbrt(P6 * c);
    lo = 0.0; hi = m1;
  } else if (c < V2) {
    double disc = 2.0 * m2 * m3 * c - m1 * m1 / 12.0;
    a = 0.5 * m1 + sqrt(disc > 0.0 ? disc : 0.0);
    lo = m1; hi = m2;
  } else {
    bool lin = (m12 <= m3);
    double Vt = lin ? m12 / (2.0 * m3) : vol_low(m1, m2, m3, m3);
    if (c < Vt) {
      // a^3 - 3 m12 a^2 + 3 (m1^2 + m2^2) a - (m1^3 + m2^3 - 6 P c) = 0
      double a2 = -3.0 * m12, a1 = 3.0 * (m1 * m1 + m2 * m2);
      double a0 = -(m1 * m1 * m1 + m2 * m2 * m2 - P6 * c);
      lo = m2; hi = lin ? m12 : m3;
      double p = a1 - a2 * a2 / 3.0;
      double q = 2.0 * a2 * a2 * a2 / 27.0 - a2 * a1 / 3.0 + a0;
      double best = 0.5 * (lo + hi);
      if (p < 0.0) {
        double r = 2.0 * sqrt(-p / 3.0);
        double arg = 3.0 * q / (p * r);
        arg = arg > 1.0 ? 1.0 : (arg < -1.0 ? -1.0 : arg);
        double th = acos(arg) / 3.0;
        double bd = 1e300;
        for (int k = 0; k < 3; ++k) {
          double t = r * cos(th - 2.0943951023931957 * k) - a2 / 3.0;
          double d = t < lo ? lo - t : (t > hi ? t - hi : 0.0);
          if (d < bd) { bd = d; best = t; }
        }
      }
      a = best;
    } else if (lin) {
      a = m3 * c + 0.5 * m12;
      lo = m12; hi = 0.5;
    } else {
      // a^3 - 1.5 a^2 + 1.5 S2 a - 0.5 (S3 - 6 P c) = 0
      double S2 = m1 * m1 + m2 * m2 + m3 * m3;
      double S3 = m1 * m1 * m1 + m2 * m2 * m2 + m3 * m3 * m3;
      double a2 = -1.5, a1 = 1.5 * S2, a0 = -0.5 * (S3 - P6 * c);
      lo = m3; hi = 0.5;
      double p = a1 - a2 * a2 / 3.0;
      double q = 2.0 * a2 * a2 * a2 / 27.0 - a2 * a1 / 3.0 + a0;
      double best = 0.5 * (lo + hi);
      if (p < 0.0) {
        double r = 2.0 * sqrt(-p / 3.0);
        double arg = 3.0 * q / (p * r);
        arg = arg > 1.0 ? 1.0 : (arg < -1.0 ? -1.0 : arg);
        double th = acos(arg) / 3.0;
        double bd = 1e300;
        for (int k = 0; k < 3; ++k) {
          double t = r * cos(th - 2.0943951023931957 * k) - a2 / 3.0;
          double d = t < lo ? lo - t : (t > hi ? t - hi : 0.0);
          if (d < bd) { bd = d; best = t; }
        }
      }
      a = best;
    }
  }
  a = a < lo ? lo : (a > hi ? hi : a);
  // polish: Newton on the monotone volume, kept inside a shrinking bracket
  // (a bisection step whenever Newton would leave it); at most 8 steps
  // and the best point seen is returned
  double blo = lo, bhi = hi, best = a, bestf = 1e300;
  for (int it = 0; it < 8; ++it) {
    const double f = vol_low(m1, m2, m3, a) - c;
    if (fabs(f) < bestf) { bestf = fabs(f); best = a; }
    if (f == 0.0) break;
    if (f < 0.0) blo = a; else bhi = a;
    const double d = dvol_low(m1, m2, m3, a);
    double an = (d > 0.0) ? a - f / d : a;
    if (an == a) break;  // converged to the last bit
    if (!(an >= blo && an <= bhi)) an = 0.5 * (blo + bhi);
    if (an == a) break;
    a = an;
  }
  return best;
}

// Non-negative doubles order like their bit patterns read as integers: a
// compare that needs no FP64 instruction (an FP64 compare occupies the FP64
// unit as long as an add on this part).
__device__ __forceinline__ bool nn_lt(double a, double b) { return dbits(a) < dbits(b); }

// Single-precision guess of the plane constant for sorted m (sum 1) and
// 0 < c <= 1/2: bisection of the volume's branch form in float (the float
// unit is ~64x wider than the FP64 one here, and bisection has no
// branch-dependent convergence), on u with a = u^3 / 2, which resolves the
// small constants of nearly empty or nearly axis-aligned cells in relative
// terms.
__device__ __forceinline__ float alpha_guess_f(float m1, float m2, float m3, float c) {
  const float m12 = m1 + m2;
  const float top = m12 < m3 ? m12 : m3;
  const bool lin = m12 <= m3;
  const float r6 = 1.0f / (6.0f * m1 * m2 * m3), r2 = 1.0f / (2.0f * m2 * m3), r3 = 1.0f / m3;
  const float v2c = m1 * m1 * r2 * (1.0f / 3.0f);
  float lo = 0.0f, hi = 1.0f;
#pragma unroll 1
  for (int it = 0; it < 22; ++it) {
    const float u = 0.5f * (lo + hi);
    const float a = 0.5f * u * u * u;
    // every branch's value, then the branch's (no divergent paths; the
    // same operations, so the same floats, as taking the branch)
    const float v1 = a * a * a * r6;
    const float v2 = a * (a - m1) * r2 + v2c;
    const float t2 = a - m2;
    const float v3 = v2 - t2 * t2 * t2 * r6;
    const float v4 = (2.0f * a - m12) * 0.5f * r3;
    const float t3 = a - m3;
    const float v5 = v3 - t3 * t3 * t3 * r6;
    const float v = a < m1 ? v1 : (a < m2 ? v2 : (a < top ? v3 : (lin ? v4 : v5)));
    if (v < c) lo = u; else hi = u;
  }
  const float u = 0.5f * (lo + hi);
  return 0.5f * u * u * u;
}

// Plane constant for sorted m (sum 1) and 0 < c <= 1/2: float guess, then
// three Newton steps in FP64 on the volume's branch form evaluated without
// branches (all branches computed, the right one selected, reciprocals of
// the branch denominators formed once), so the lanes of a warp stay
// together.  The best of the iterates is kept; if it misses c by more than
// rounding, the analytic solution with its safeguarded polish is used.
__device__ __forceinline__ double alpha_low(double m1, double m2, double m3, double c) {
  const double m12 = m1 + m2;
  const double top = m12 < m3 ? m12 : m3;
  const bool lin = !nn_lt(m3, m12);  // m12 <= m3
  const double r6 = 1.0 / (6.0 * m1 * m2 * m3);  // inf when m1 = 0: that branch is then never selected
  const double r2 = 1.0 / (2.0 * m2 * m3);
  const double r3 = 1.0 / m3;
  const double v2c = m1 * m1 * r2 / 3.0;
  double a = (double)alpha_guess_f((float)m1, (float)m2, (float)m3, (float)c);
  double best = a;
  long long bestf = 0x7FF0000000000000LL;  // |f| bits
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const double t1 = a - m1, t2 = a - m2, t3 = a - m3;
    const double v1 = a * a * a * r6, d1 = 3.0 * a * a * r6;
    const double v2 = a * t1 * r2 + v2c, d2 = (a + t1) * r2;
    const double v3 = v2 - t2 * t2 * t2 * r6, d3 = d2 - 3.0 * t2 * t2 * r6;
    const double v4 = (a + (a - m12)) * 0.5 * r3, d4 = r3;
    const double v5 = v3 - t3 * t3 * t3 * r6, d5 = d3 - 3.0 * t3 * t3 * r6;
    double v, d;
    if (nn_lt(a, m1)) { v = v1; d = d1; }
    else if (nn_lt(a, m2)) { v = v2; d = d2; }
    else if (nn_lt(a, top)) { v = v3; d = d3; }
    else if (lin) { v = v4; d = d4; }
    else { v = v5; d = d5; }
    const double f = v - c;
    const long long af = dbits(f) & 0x7FFFFFFFFFFFFFFFLL;
    if (af < bestf) { bestf = af; best = a; }
    if (it == 3) break;
    double an = a - f / d;
    // stay in [0, 1/2] (a > 0 keeps the cubic corner's derivative nonzero)
    if (!(dbits(an) > 0)) an = 0.5 * a;
    if (nn_lt(0.5, an)) an = 0.5;
    a = an;
  }
  // converged to rounding: |f| within a few ulps of the volume
  const double tol = 32.0 * 1.1102230246251565e-16 * c;
  if (!(__longlong_as_double(bestf) <= tol)) best = alpha_low_analytic(m1, m2, m3, c);
  return best;
}

// An estimate of the same plane constant (float guess, two Newton steps on
// the same branch form; no check of the result), for callers that verify it.
__device__ __forceinline__ double alpha_low_est(double m1, double m2, double m3, double c) {
  const double m12 = m1 + m2;
  const double top = nn_lt(m12, m3) ? m12 : m3;
  const bool lin = !nn_lt(m3, m12);
  const double r6 = 1.0 / (6.0 * m1 * m2 * m3);
  const double r2 = 1.0 / (2.0 * m2 * m3);
  const double r3 = 1.0 / m3;
  const double v2c = m1 * m1 * r2 * (1.0 / 3.0);
  double a = (double)alpha_guess_f((float)m1, (float)m2, (float)m3, (float)c);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double t1 = a - m1, t2 = a - m2, t3 = a - m3;
    const double v1 = a * a * a * r6, d1 = 3.0 * a * a * r6;
    const double v2 = a * t1 * r2 + v2c, d2 = (a + t1) * r2;
    const double v3 = v2 - t2 * t2 * t2 * r6, d3 = d2 - 3.0 * t2 * t2 * r6;
    const double v4 = (a + (a - m12)) * 0.5 * r3, d4 = r3;
    const double v5 = v3 - t3 * t3 * t3 * r6, d5 = d3 - 3.0 * t3 * t3 * r6;
    double v, d;
    if (nn_lt(a, m1)) { v = v1; d = d1; }
    else if (nn_lt(a, m2)) { v = v2; d = d2; }
    else if (nn_lt(a, top)) { v = v3; d = d3; }
    else if (lin) { v = v4; d = d4; }
    else { v = v5; d = d5; }
    double an = a - (v - c) / d;
    if (!(dbits(an) > 0)) an = 0.5 * a;
    if (nn_lt(0.5, an)) an = 0.5;
    a = an;
  }
  return a;
}

// alpha with volume(m, alpha) = c for any m (mirror, normalise, invert,
// undo): the same outer steps as the volume function.
__device__ __forceinline__ double plane_alpha(double m0, double m1, double m2, double c) {
  Mirror r = mirror_normalise(m0, m1, m2);
  if (r.l1 == 0.0) return 0.0;
  if (c <= 0.0) return 0.0 - r.sh;
  if (c >= 1.0) return r.l1 - r.sh;
  double s0 = r.mp[0], s1 = r.mp[1], s2 = r.mp[2];
  sort3(s0, s1, s2);
  // one call for both halves (c or 1 - c picked per lane): an FP64
  // instruction costs its full issue time whatever the active lanes, so a
  // warp that took both branches would pay for the inversion twice
  const bool up = !(c <= 0.5);
  const double al = alpha_low(s0, s1, s2, up ? 1.0 - c : c);
  const double am = up ? 1.0 - al : al;
  return am * r.l1 - r.sh;
}

// The same plane constant by bisection on the monotone volume, step for
// step the plain algorithm (interval [0,1] of the mirrored normalised plane,
// halving until the bracket is two adjacent doubles, then the end whose
// volume is closer to c).  Used where alpha(c) is ill-conditioned (c within
// 1e-3 of 0 or 1) and the plane is extrapolated into neighbouring cells,
// which would amplify the last-bit differences of any other inversion.
//
// Two bounds on the FP64 volume (these operations, no contraction) make it
// cheaper without changing a midpoint or a decision: (1) it is within 256
// ulps of the exact volume V (relative below the cube's middle, relative to
// 1 - V above it, plus an ulp); a rounding analysis of the branch forms
// gives ~54 ulps, 4.4 were seen over 3.2e5 normals and constants spanning
// every branch, the branch boundaries and degenerate normals against exact
// rational arithmetic; (2) its form with rounded reciprocals is within 256
// ulps of it (5 seen); with the branch forms' cancellation bounds (v2 <=
// 1.5 v3, (a - m2)^3 / d6 <= v3 / 2, and in the last branch v3 <= 1.04 v5,
// (a - m3)^3 / d6 <= 0.04 v5) the rounding analysis gives ~14 ulps, so a
// 64-ulp margin decides.
//
// LANES = 3: three lanes of a warp (lanes leader .. leader + 2, mask gmask,
// sub = lane - leader) share one cell and take two levels per round -- the
// midpoint and both midpoints of the level after it, each lane deciding
// one, so a round costs one volume per lane -- with the same midpoints and
// decisions as the one-lane loop.
template <int LANES>
static __device__ __noinline__ double plane_alpha_bisect_t(double m0, double m1, double m2, double c, unsigned gmask,
                                                           int leader, int sub) {
  Mirror r = mirror_normalise(m0, m1, m2);
  if (r.l1 == 0.0) return 0.0;
  if (c <= 0.0) return 0.0 - r.sh;
  if (c >= 1.0) return r.l1 - r.sh;
  // the volume function's own steps, with the sort of the (fixed) normal
  // done once and its compares of non-negative values made on integers:
  // the same values at every midpoint as the plain volume function
  double s0 = r.mp[0], s1 = r.mp[1], s2 = r.mp[2];
  sort3(s0, s1, s2);
  const double m12 = s0 + s1;
  const double top = nn_lt(m12, s2) ? m12 : s2;
  const bool lin = !nn_lt(s2, m12);
  const double d6 = 6.0 * s0 * s1 * s2, d2 = 2.0 * s1 * s2, d2m3 = 2.0 * s2;
  const double v2c = s0 * s0 / (6.0 * s1 * s2);
  auto vlow = [&](double a) -> double {
    if (nn_lt(a, s0)) return a * a * a / d6;
    const double v2 = a * (a - s0) / d2 + v2c;
    if (nn_lt(a, s1)) return v2;
    const double t2 = a - s1;
    const double v3 = v2 - t2 * t2 * t2 / d6;
    if (nn_lt(a, top)) return v3;
    if (lin) return (2.0 * a - m12) / d2m3;
    const double t3 = a - s2;
    return v3 - t3 * t3 * t3 / d6;
  };
  auto vpos = [&](double a) -> double {  // a in (0, 1) here; one vlow for both halves
    const bool up = nn_lt(0.5, a);
    const double w = vlow(up ? 1.0 - a : a);
    return up ? 1.0 - w : w;
  };
  // The same volume with the divisions replaced by products with the
  // rounded reciprocals: within a few ulps of it (relative below the middle
  // of the cell, of 1 above).  A midpoint whose fast volume is farther from
  // c than a margin ~500 times that is decided from it -- the exact volume
  // is on the same side of c -- and only midpoints near the root pay for the
  // exact volume's divisions (slow on this part).  The decisions, and so the
  // result, are those of the plain bisection.
  const double r6 = 1.0 / d6, r2 = 1.0 / d2, r2m3 = 1.0 / d2m3;
  auto vlow_fast = [&](double a) -> double {
    if (nn_lt(a, s0)) return a * a * a * r6;
    const double v2 = a * (a - s0) * r2 + v2c;
    if (nn_lt(a, s1)) return v2;
    const double t2 = a - s1;
    const double v3 = v2 - t2 * t2 * t2 * r6;
    if (nn_lt(a, top)) return v3;
    if (lin) return (2.0 * a - m12) * r2m3;
    const double t3 = a - s2;
    return v3 - t3 * t3 * t3 * r6;
  };
  // Above the cube's middle the decision vpos(mid) < c, vpos = RN(1 - w)
  // with w the volume at 1 - mid, is w > t exactly, t = (1 - c) + 2^-54 (c
  // in [1/2, 1): 1 - c exact, RN(1 - w) < c iff 1 - w lies below the
  // midpoint between c and its predecessor; w = t is a tie and goes to the
  // exact evaluation), a comparison with relative bounds only.
  const double t = (1.0 - c) + 0x1p-54;
  // bound (2): a fast volume farther from its threshold than this is on the
  // exact volume's side of it
  const double margin_low = 0x1p-47 * c, margin_high = 0x1p-47 * t;
  double lo = 0.0, hi = 1.0;
  int it = 0;
  // Levels whose midpoint lies clear of the root are decided without a
  // volume: with the Newton root ae, bound (1) and the monotone exact volume
  // show that every a < aL is below and every a > aR is not (else nothing
  // is skipped).  Until a midpoint falls in [aL, aR] the bisection's
  // decisions are then known; its midpoints are computed as it computes
  // them, and the loop below resumes at that midpoint.  (For c <= 1/4 every
  // a > 1/2 has a volume >= 1/2 - 2^-45 > c; for c >= 3/4 every a <= 1/2 one
  // <= 1/2 + 2^-45 < c.)
  if (nn_lt(c, 0.25) || nn_lt(0.75, c)) {
    // (every step below is taken by every lane, the halves picked per
    // lane, so a warp evaluates each volume once)
    const bool low_c = nn_lt(c, 0.25);
    const double al = alpha_low_est(s0, s1, s2, low_c ? c : 1.0 - c);
    const double ae = low_c ? al : 1.0 - al;
    double dz = (low_c ? ae : 1.0 - ae) * 0x1p-36;
    if (!low_c && nn_lt(dz, 0x1p-50)) dz = 0x1p-50;  // a few ulps of 1 at least
    const double aL = ae - dz, aR = ae + dz;
    // below the middle: vlow(aL) < c <= vlow(aR); above it, with w(a) =
    // vlow(1 - a) falling in a (1 - aL and 1 - aR exact): w(aL) > t > w(aR)
    const double wL = vlow(low_c ? aL : 1.0 - aL), wR = vlow(low_c ? aR : 1.0 - aR);
    bool ok;
    if (low_c) {
      ok = dgt0(aL) && nn_lt(aL, aR) && !nn_lt(0.5, aR) && nn_lt(wL * (1.0 + 0x1p-43), c) &&
           !nn_lt(wR * (1.0 - 0x1p-43), c);
    } else {
      ok = !nn_lt(aL, 0.5) && nn_lt(aL, aR) && nn_lt(aR, 1.0) && nn_lt(t, wL * (1.0 - 0x1p-43)) &&
           nn_lt(wR * (1.0 + 0x1p-43), t);
    }
    if (ok && !(low_c && nn_lt(aR, 0x1p-900))) {  // (the units stay normal doubles)
      // The skipped levels on integers.  Below the middle the bisection
      // first halves [0, 1] to [0, 2^(e+1)] (e: aR's exponent; the midpoints
      // 2^-1 .. 2^(e+1) all exceed aR); then, as above the middle from [0, 1],
      // the bracket is [L, L + H] in units 2^(e+1-62) (2^-62): midpoints
      // L + H/2 exact, compared with ceil(aL / unit) and floor(aR / unit).
      // While H >= 2^10 every midpoint has at most 53 significant bits, so
      // the doubles the bisection would compute are these integers times
      // the unit.
      const int e = (int)((dbits(aR) >> 52) & 0x7FF) - 1023;
      const int k0 = low_c ? -e - 1 : 0;       // halvings of hi from 1
      const int sc = low_c ? 61 - e : 62;      // 1 / unit = 2^sc
      const double up = __longlong_as_double((long long)(sc + 1023) << 52);
      const double dn = __longlong_as_double((long long)(1023 - sc) << 52);
      const unsigned long long ZL = __double2ull_ru(aL * up), ZR = __double2ull_rd(aR * up);
      unsigned long long L = 0ull, H = 1ull << 62;
      it = k0;
      for (; it < 200 && H >= (1ull << 10); ++it) {
        const unsigned long long M = L + (H >> 1);
        if (M < ZL) L = M;
        else if (M > ZR) {}
        else break;
        H >>= 1;
      }
      lo = (double)L * dn;
      hi = (double)(L + H) * dn;
    }
  }
  // below the middle: mid is below iff the volume at mid is < c; above it
  // iff the volume at 1 - mid is > t (one fast volume per lane either way)
  auto below_at = [&](double mid) -> bool {
    const bool up = nn_lt(0.5, mid);
    const double d = vlow_fast(up ? 1.0 - mid : mid) - (up ? t : c);
    if (nn_lt(up ? margin_high : margin_low, fabs(d))) return up ? dgt0(d) : dlt0(d);
    return nn_lt(vpos(mid), c);
  };
  if (LANES == 1) {
    for (; it < 200; ++it) {
      double mid = lo + 0.5 * (hi - lo);
      if (!(nn_lt(lo, mid) && nn_lt(mid, hi))) break;
      if (below_at(mid)) lo = mid;
      else hi = mid;
    }
  } else {
    while (it < 200) {
      const double mid = lo + 0.5 * (hi - lo);
      if (!(nn_lt(lo, mid) && nn_lt(mid, hi))) break;
      // the next level's midpoint after either decision, as the loop above
      // would compute it from its new bracket
      const double midL = lo + 0.5 * (mid - lo), midR = mid + 0.5 * (hi - mid);
      const bool b = below_at(sub == 0 ? mid : (sub == 1 ? midL : midR));
      const bool bA = __shfl_sync(gmask, b, leader), bL = __shfl_sync(gmask, b, leader + 1),
                 bR = __shfl_sync(gmask, b, leader + 2);
      if (bA) lo = mid;
      else hi = mid;
      if (++it >= 200) break;
      const double m2n = bA ? midR : midL;
      if (!(nn_lt(lo, m2n) && nn_lt(m2n, hi))) break;
      if (bA ? bR : bL) lo = m2n;
      else hi = m2n;
      ++it;
    }
  }
  // lo and hi are 0 or 1 only at a bracket end never left (vpos's end cases)
  const double vlo = dbits(lo) == 0 ? 0.0 : vpos(lo);
  const double vhi = dbits(hi) == 0x3FF0000000000000LL ? 1.0 : vpos(hi);
  const long long el = dbits(vlo - c) & 0x7FFFFFFFFFFFFFFFLL, eh = dbits(vhi - c) & 0x7FFFFFFFFFFFFFFFLL;
  double am = (eh < el) ? hi : lo;
  return am * r.l1 - r.sh;
}
static __device__ __forceinline__ double plane_alpha_bisect(double m0, double m1, double m2, double c) {
  return plane_alpha_bisect_t<1>(m0, m1, m2, c, 0u, 0, 0);
}

// The volume function with every compare on the integer pipe: the normal is
// mirrored to |m_i| (a -0 component becomes +0, which changes no volume), so
// all compared values are non-negative and order like their bit patterns.
// Not bit-for-bit the plain routine's steps at a zero component's sign, so
// the oracle-identical bisection keeps the plain one.
__device__ __forceinline__ double vol_low_nn(double m1, double m2, double m3, double a) {
  const double m12 = m1 + m2;
  if (nn_lt(a, m1)) return a * a * a / (6.0 * m1 * m2 * m3);
  const double v2 = a * (a - m1) / (2.0 * m2 * m3) + m1 * m1 / (6.0 * m2 * m3);
  if (nn_lt(a, m2)) return v2;
  const double t2 = a - m2;
  const double v3 = v2 - t2 * t2 * t2 / (6.0 * m1 * m2 * m3);
  const double top = nn_lt(m12, m3) ? m12 : m3;
  if (nn_lt(a, top)) return v3;
  if (!nn_lt(m3, m12)) return (2.0 * a - m12) / (2.0 * m3);
  const double t3 = a - m3;
  return v3 - t3 * t3 * t3 / (6.0 * m1 * m2 * m3);
}

// The volume function split in two: the normal's mirror, normalisation and
// sort (once per normal), then the volume at a plane constant.  volume_nn is
// the two in a row, so several volumes of one normal are bit for bit the
// single calls'.
struct VolNormal {
  double sh, l1, a0, a1, a2;
};
__device__ __forceinline__ VolNormal volume_normal_nn(double m0, double m1, double m2) {
  VolNormal p;
  p.sh = 0.0;
  if (dlt0(m0)) p.sh -= m0;
  if (dlt0(m1)) p.sh -= m1;
  if (dlt0(m2)) p.sh -= m2;
  double a0 = fabs(m0), a1 = fabs(m1), a2 = fabs(m2);
  p.l1 = a0 + a1 + a2;
  if (dnz(p.l1)) {
    a0 /= p.l1; a1 /= p.l1; a2 /= p.l1;
    // sort the three non-negative components
    double t;
    if (nn_lt(a1, a0)) { t = a0; a0 = a1; a1 = t; }
    if (nn_lt(a2, a1)) { t = a1; a1 = a2; a2 = t; }
    if (nn_lt(a1, a0)) { t = a0; a0 = a1; a1 = t; }
  }
  p.a0 = a0; p.a1 = a1; p.a2 = a2;
  return p;
}

__device__ __forceinline__ double volume_at_nn(const VolNormal& p, double alpha) {
  if (!dnz(p.l1)) return dlt0(alpha) ? 0.0 : 1.0;
  const double a = (alpha + p.sh) / p.l1;
  if (!dgt0(a)) return 0.0;
  if (!nn_lt(a, 1.0)) return 1.0;
  // one call for both halves (the argument picked per lane, as above)
  const bool up = nn_lt(0.5, a);
  const double v = vol_low_nn(p.a0, p.a1, p.a2, up ? 1.0 - a : a);
  return up ? 1.0 - v : v;
}

__device__ __forceinline__ double volume_nn(double m0, double m1, double m2, double alpha) {
  return volume_at_nn(volume_normal_nn(m0, m1, m2), alpha);
}

// liquid volume (cell units) in the slab x_axis in [x0, x0+delta], any m,
// with the integer-pipe volume function
__device__ __forceinline__ double slab_volume_nn(const double m[3], double alpha, int axis, double x0, double delta) {
  if (!dgt0(delta)) return 0.0;
  double mm0 = m[0], mm1 = m[1], mm2 = m[2];
  const double ma = m[axis];
  if (axis == 0) mm0 = ma * delta;
  else if (axis == 1) mm1 = ma * delta;
  else mm2 = ma * delta;
  return delta * volume_nn(mm0, mm1, mm2, alpha - ma * x0);
}

// liquid volume (cell units) in the slab x_axis in [x0, x0+delta]
__device__ __forceinline__ double slab_volume(const double m[3], double alpha, int axis, double x0, double delta) {
  if (delta <= 0.0) return 0.0;
  double mm0 = m[0], mm1 = m[1], mm2 = m[2];
  double ma = m[axis];
  if (axis == 0) mm0 = ma * delta;
  else if (axis == 1) mm1 = ma * delta;
  else mm2 = ma * delta;
  double a2 = alpha - ma * x0;
  return delta * volume(mm0, mm1, mm2, a2);
}

// ---------------------------------------------------------------------------
// MYC normal (Aulisa et al. 2007): stencil s[(dz*3+dy)*3+dx], offsets 0..2
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sax(const double* s, int d, int r, int p, int q) {
  // value at offset r along d, p along t1, q along t2 (t1 < t2 the other axes)
  int o0, o1, o2;
  if (d == 0) { o0 = r; o1 = p; o2 = q; }
  else if (d == 1) { o1 = r; o0 = p; o2 = q; }
  else { o2 = r; o0 = p; o1 = q; }
  return s[((o2 + 1) * 3 + (o1 + 1)) * 3 + (o0 + 1)];
}

__device__ __forceinline__ void youngs_normal(const double* s, double m[3]) {
  const double w[3] = {1.0, 2.0, 1.0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double g = 0.0;
#pragma unroll
    for (int q = -1; q <= 1; ++q)
#pragma unroll
      for (int p = -1; p <= 1; ++p) {
        double diff = sax(s, d, 1, p, q) - sax(s, d, -1, p, q);
        g = g + (w[p + 1] * w[q + 1]) * diff;
      }
    m[d] = -g;
  }
  double l1 = fabs(m[0]) + fabs(m[1]) + fabs(m[2]);
  if (l1 > 0.0) { m[0] /= l1; m[1] /= l1; m[2] /= l1; }
  else { m[0] = 1.0; m[1] = 0.0; m[2] = 0.0; }
}

__device__ __forceinline__ void cc_candidate(const double* s, int d, double m[3]) {
  double h[3][3];
#pragma unroll
  for (int q = -1; q <= 1; ++q)
#pragma unroll
    for (int p = -1; p <= 1; ++p) {
      double col = sax(s, d, -1, p, q);
      col = col + sax(s, d, 0, p, q);
      col = col + sax(s, d, 1, p, q);
      h[p + 1][q + 1] = col;
    }
  double lower = 0.0, upper = 0.0;
#pragma unroll
  for (int q = -1; q <= 1; ++q)
#pragma unroll
    for (int p = -1; p <= 1; ++p) {
      lower = lower + sax(s, d, -1, p, q);
      upper = upper + sax(s, d, 1, p, q);
    }
  double sg = (lower >= upper) ? 1.0 : -1.0;
  double a1 = -(h[2][1] - h[0][1]) * 0.5;
  double a2 = -(h[1][2] - h[1][0]) * 0.5;
  double l1 = fabs(a1) + fabs(a2) + 1.0;
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  m[t1] = a1 / l1;
  m[t2] = a2 / l1;
  m[d] = sg / l1;
}

// Centred-columns candidate along d without its divisions: the two
// tangential slopes a1, a2 (along t1 < t2), the L1 norm l1 = |a1|+|a2|+1 and
// the sign of the own-axis component.
struct CCParts {
  double a1, a2, l1, sg;
};

__device__ __forceinline__ CCParts cc_parts(const double* s, int d) {
  double h[3][3];
#pragma unroll
  for (int q = -1; q <= 1; ++q)
#pragma unroll
    for (int p = -1; p <= 1; ++p) {
      double col = sax(s, d, -1, p, q);
      col = col + sax(s, d, 0, p, q);
      col = col + sax(s, d, 1, p, q);
      h[p + 1][q + 1] = col;
    }
  double lower = 0.0, upper = 0.0;
#pragma unroll
  for (int q = -1; q <= 1; ++q)
#pragma unroll
    for (int p = -1; p <= 1; ++p) {
      lower = lower + sax(s, d, -1, p, q);
      upper = upper + sax(s, d, 1, p, q);
    }
  CCParts r;
  r.sg = !nn_lt(lower, upper) ? 1.0 : -1.0;  // lower >= upper (both >= 0)
  // the central differences' halves on the integer pipe; a difference
  // whose half would be subnormal (never met in practice) takes the product
  // (a1 = -(h21 - h01) / 2, a2 = -(h12 - h10) / 2, the sign flipped on the
  // bit pattern)
  const double d1 = h[2][1] - h[0][1], d2 = h[1][2] - h[1][0];
  bool ok1, ok2;
  double e1 = dhalf_exact(d1, ok1), e2 = dhalf_exact(d2, ok2);
  if (__any_sync(__activemask(), !(ok1 && ok2))) {
    e1 = ok1 ? e1 : d1 * 0.5;
    e2 = ok2 ? e2 : d2 * 0.5;
  }
  r.a1 = dneg(e1);
  r.a2 = dneg(e2);
  r.l1 = fabs(r.a1) + fabs(r.a2) + 1.0;
  return r;
}

// The choices of the MYC rule from the candidates' L1 norms l1_d (own-axis
// components 1 / l1_d) and Youngs' largest |g| over its L1 norm, with the
// divisions the plain rule takes: the best candidate bd (largest own-axis
// component, lowest axis on ties) and whether it is kept (its component not
// below Youngs' largest).
static __device__ __noinline__ void myc_choice_exact(double l10, double l11, double l12, double amax, double l1y, int& bd,
                                              bool& use_cc) {
  const double d0 = 1.0 / l10, d1 = 1.0 / l11, d2 = 1.0 / l12;
  bd = 0;
  double dm = d0;
  if (nn_lt(dm, d1)) { bd = 1; dm = d1; }
  if (nn_lt(dm, d2)) { bd = 2; dm = d2; }
  const double ymax = dnz(l1y) ? amax / l1y : 1.0;
  use_cc = !nn_lt(ymax, dm);
}

// Best centred-columns candidate (largest own-axis component, lowest axis on
// ties), kept unless its dominant component exceeds the Youngs normal's, in
// which case Youngs is taken.  The same values as normalising every
// candidate and comparing their components, with fewer divisions: a
// candidate's own-axis component is +-1/l1 exactly, and the largest Youngs
// component is the largest |g| over l1 (division is monotone).  Non-negative
// values are compared as integers.
__device__ __forceinline__ void myc_normal(const double* s, double m[3]) {
  CCParts c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) c[d] = cc_parts(s, d);
  // Youngs gradient; the weights 2 and 4 applied on the integer pipe
  double y[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double g = 0.0;
#pragma unroll
    for (int q = -1; q <= 1; ++q)
#pragma unroll
      for (int p = -1; p <= 1; ++p) {
        const double diff = sax(s, d, 1, p, q) - sax(s, d, -1, p, q);
        const int k = (p == 0) + (q == 0);  // weight 2^k
        const double wd = k == 0 ? diff : (k == 1 ? dtwice(diff) : dtwice(dtwice(diff)));
        g = g + wd;
      }
    y[d] = -g;
  }
  const double ay0 = fabs(y[0]), ay1 = fabs(y[1]), ay2 = fabs(y[2]);
  const double l1y = ay0 + ay1 + ay2;
  double amax = ay0;
  if (nn_lt(amax, ay1)) amax = ay1;
  if (nn_lt(amax, ay2)) amax = ay2;
  // The rule's choices compare rounded quotients (1 / l1_d, amax / l1y);
  // they are taken here from the operands wherever those are far enough
  // apart that the quotients' rounding cannot tie or reorder them (L1 norms
  // >= 1 and non-negative values compare as integers; 8 units in the last
  // place is a relative gap > 2^-50, 4 roundings' worth), else with the
  // divisions themselves.
  const long long b0 = dbits(c[0].l1), b1 = dbits(c[1].l1), b2 = dbits(c[2].l1);
  bool amb = false;
  // 1/l1_a < 1/l1_b  <=>  l1_a > l1_b, unless they are within 8 ulps
  auto dom_lt = [&](long long la, long long lb) {
    if (la - lb > 0 && la - lb < 8) amb = true;
    return la - lb >= 8;
  };
  int bd = dom_lt(b0, b1) ? 1 : 0;
  const long long bb = bd ? b1 : b0;
  if (dom_lt(bb, b2)) bd = 2;
  const double lbd = bd == 0 ? c[0].l1 : (bd == 1 ? c[1].l1 : c[2].l1);
  // amax / l1y < 1 / l1_bd  <=>  amax l1_bd < l1y (the product within an
  // ulp; 16 ulps apart decides)
  bool use_cc = true;  // l1y = 0: Youngs' largest component is 1, not below
  if (dnz(l1y)) {
    const long long pb = dbits(amax * lbd), yb = dbits(l1y);
    if (pb + 16 <= yb) use_cc = false;
    else if (!(pb >= yb + 16)) amb = true;
  }
  if (__any_sync(__activemask(), amb)) {
    int bx;
    bool ux;
    myc_choice_exact(c[0].l1, c[1].l1, c[2].l1, amax, l1y, bx, ux);
    if (amb) { bd = bx; use_cc = ux; }
  }
  // the centred-columns candidate (a1, a2 on the transverse axes, +-1 on
  // its own, over l1) or Youngs' (y / l1y; (1, 0, 0) when y = 0).
  // Numerators and denominator are picked first, so both cases share three
  // divisions (a warp whose lanes took both branches would pay for five).
  const CCParts cb = bd == 0 ? c[0] : (bd == 1 ? c[1] : c[2]);
  const double own = dbits(cb.sg) < 0 ? -1.0 : 1.0;
  // transverse axes of bd: t1 = bd == 0 ? 1 : 0, t2 = bd == 2 ? 1 : 2
  const double n0 = bd == 0 ? own : cb.a1;
  const double n1 = bd == 1 ? own : (bd == 0 ? cb.a1 : cb.a2);
  const double n2 = bd == 2 ? own : cb.a2;
  const double den = use_cc ? cb.l1 : l1y;
  const double q0 = (use_cc ? n0 : y[0]) / den, q1 = (use_cc ? n1 : y[1]) / den, q2 = (use_cc ? n2 : y[2]) / den;
  const bool deg = !use_cc && !dnz(l1y);
  m[0] = deg ? 1.0 : q0;
  m[1] = deg ? 0.0 : q1;
  m[2] = deg ? 0.0 : q2;
}

// ---------------------------------------------------------------------------
// WENO5 face value (Jiang-Shu weights, eps 1e-6), upwind-ordered stencil:
// weno5_df (vof_df.cuh), the weights and the correction to the donor value
// in double-float pairs (FP64-accurate, a fraction of the FP64 instructions).
// Five equal values return the donor value exactly.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Precision form (vof_grid.precision = VOF_F32_FLUX): the sweeps'
// reconstruction and flux weights in FP32, on the FP32 unit (~64x the FP64
// rate on this part).  The plane constant is still inverted in FP64 from the
// FP32 normal, stencil differences and cell updates stay FP64, so the fluxes
// still telescope and volume and energy stay conserved to FP64 round-off.
// ---------------------------------------------------------------------------
// MYC normal in FP32.  The three decisions of the method (which
// centred-columns candidate dominates, its own-axis sign, candidate or
// Youngs) are taken in FP32 only where FP32 round-off cannot change them; a
// cell within the error bounds below of any decision takes the FP64 normal,
// so the precision form makes every decision the FP64 form makes.  Bounds,
// with stencil values in [0, 1] rounded to FP32 (unit round-off u = 2^-24):
// a column sum is off by <= 9u, a slope by <= 11u, l1 = |a1| + |a2| + 1 <= 4
// by <= 30u, so dom = 1/l1 by <= 31u relative; the lower and upper sums of
// 9 values by <= 60u each; a Youngs component (weights 1, 2, 4, magnitude
// <= 16) by <= 190u and l1y by <= 670u, so ymax = max|y| / l1y by
// <= 860u / l1y + u.  The margins below are about twice these.
__device__ __forceinline__ void myc_normal_f(const double* sd, double m[3]) {
  float s[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) s[i] = (float)sd[i];
  auto at = [&](int d, int r, int p, int q) -> float {
    int o0, o1, o2;
    if (d == 0) { o0 = r; o1 = p; o2 = q; }
    else if (d == 1) { o1 = r; o0 = p; o2 = q; }
    else { o2 = r; o0 = p; o1 = q; }
    return s[((o2 + 1) * 3 + (o1 + 1)) * 3 + (o0 + 1)];
  };
  float best[3] = {0.f, 0.f, 0.f}, dom[3];
  float bdom = -1.f, bsep = 0.f;
  int bd = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float h[3][3], lower = 0.f, upper = 0.f;
#pragma unroll
    for (int q = -1; q <= 1; ++q)
#pragma unroll
      for (int p = -1; p <= 1; ++p) {
        h[p + 1][q + 1] = (at(d, -1, p, q) + at(d, 0, p, q)) + at(d, 1, p, q);
        lower += at(d, -1, p, q);
        upper += at(d, 1, p, q);
      }
    const float sg = lower >= upper ? 1.f : -1.f;
    const float a1 = -(h[2][1] - h[0][1]) * 0.5f, a2 = -(h[1][2] - h[1][0]) * 0.5f;
    const float l1 = fabsf(a1) + fabsf(a2) + 1.f;
    dom[d] = 1.f / l1;
    if (dom[d] > bdom) {
      bdom = dom[d];
      bd = d;
      bsep = fabsf(lower - upper);
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      best[t1] = a1 * dom[d];
      best[t2] = a2 * dom[d];
      best[d] = sg * dom[d];
    }
  }
  const float w[3] = {1.f, 2.f, 1.f};
  float y[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float gsum = 0.f;
#pragma unroll
    for (int q = -1; q <= 1; ++q)
#pragma unroll
      for (int p = -1; p <= 1; ++p) gsum += (w[p + 1] * w[q + 1]) * (at(d, 1, p, q) - at(d, -1, p, q));
    y[d] = -gsum;
  }
  const float l1y = fabsf(y[0]) + fabsf(y[1]) + fabsf(y[2]);
  const float amax = fmaxf(fabsf(y[0]), fmaxf(fabsf(y[1]), fabsf(y[2])));
  const float ymax = l1y > 0.f ? amax / l1y : 1.f;
  bool near = bsep <= 2e-5f;                                    // own-axis sign
  near |= fabsf(bdom - ymax) * l1y <= 5e-6f * l1y + 1e-4f;      // candidate or Youngs
#pragma unroll
  for (int d = 0; d < 3; ++d) near |= d != bd && bdom - dom[d] <= 8e-6f * bdom;  // dominance
  if (near) {
    myc_normal(sd, m);
    return;
  }
  if (bdom <= ymax) {
    m[0] = best[0]; m[1] = best[1]; m[2] = best[2];
  } else {
    m[0] = y[0] / l1y; m[1] = y[1] / l1y; m[2] = y[2] / l1y;
  }
}

__device__ __forceinline__ float vol_low_f(float m1, float m2, float m3, float a) {
  const float m12 = m1 + m2;
  if (a < m1) return a * a * a / (6.f * m1 * m2 * m3);
  const float v2 = a * (a - m1) / (2.f * m2 * m3) + m1 * m1 / (6.f * m2 * m3);
  if (a < m2) return v2;
  const float t2 = a - m2;
  const float v3 = v2 - t2 * t2 * t2 / (6.f * m1 * m2 * m3);
  const float top = m12 < m3 ? m12 : m3;
  if (a < top) return v3;
  if (m12 <= m3) return (2.f * a - m12) / (2.f * m3);
  const float t3 = a - m3;
  return v3 - t3 * t3 * t3 / (6.f * m1 * m2 * m3);
}

// donor-slab volume with the cut geometry in FP32.  The plane's offset from
// the slab's lowest corner (alpha - m_axis x0 + shift) and its complement
// l1 - offset are formed in FP64, so whichever of the two is small keeps its
// relative accuracy when rounded to FP32, the slab is empty or full exactly
// when the FP64 form finds it so, and a slab that is nearly full returns
// 1 - (FP32 deficit) in FP64: cells next to a full or empty slab are not left
// with FP32 round-off of size 1e-8, which would exceed the mixed threshold
// and make them mixed cells that the FP64 form keeps pure.  The result is
// held to what the slab can hold of the donor's liquid c and gas 1 - c,
// [c - (1 - delta), c] (exact bounds that FP32 round-off would otherwise
// cross): a donor emptied of either phase is emptied exactly, as in FP64,
// and not left a few 1e-9 beyond it for the update to clip (clipping c
// without e moves T by C_pl / C_pg times the clipped volume).
__device__ __forceinline__ double slab_volume_f(const double m[3], double alpha, int axis, double x0, double delta,
                                                double c) {
  if (!dgt0(delta)) return 0.0;
  float mm0 = (float)m[0], mm1 = (float)m[1], mm2 = (float)m[2];
  const double ma = m[axis];
  const float md = (float)(ma * delta);
  if (axis == 0) mm0 = md;
  else if (axis == 1) mm1 = md;
  else mm2 = md;
  float sh = 0.f;
  if (mm0 < 0.f) sh -= mm0;
  if (mm1 < 0.f) sh -= mm1;
  if (mm2 < 0.f) sh -= mm2;
  float a0 = fabsf(mm0), a1 = fabsf(mm1), a2 = fabsf(mm2);
  const float l1 = (a0 + a1) + a2;
  const double num = fma(-ma, x0, alpha) + (double)sh;  // offset, cell units
  const double numc = (double)l1 - num;                // complement
  if (!dgt0(num)) return 0.0;
  if (!dgt0(numc)) return delta;
  const float r = 1.f / l1;
  a0 *= r; a1 *= r; a2 *= r;
  float t;
  if (a1 < a0) { t = a0; a0 = a1; a1 = t; }
  if (a2 < a1) { t = a1; a1 = a2; a2 = t; }
  if (a1 < a0) { t = a0; a0 = a1; a1 = t; }
  const float alo = (float)num * r, ahi = (float)numc * r;
  double v = alo <= ahi ? delta * (double)vol_low_f(a0, a1, a2, alo)
                        : delta * (1.0 - (double)vol_low_f(a0, a1, a2, ahi));
  if (nn_lt(c, v)) v = c;  // both >= 0
  const double lo = c - (1.0 - delta);
  if (dgt0(lo) && nn_lt(v, lo)) v = lo;
  return v;
}

// WENO5 with the neighbour differences in FP64 and the nonlinear weights and
// the correction to v0 in FP32: T_f = v0 + correction
__device__ __forceinline__ double weno5_f(double vm2, double vm1, double v0, double vp1, double vp2) {
  if (deq(vm2, v0) && deq(vm1, v0) && deq(vp1, v0) && deq(vp2, v0)) return v0;
  const float D0 = (float)(vm1 - vm2), D1 = (float)(v0 - vm1), D2 = (float)(vp1 - v0), D3 = (float)(vp2 - vp1);
  const float epsw = 1e-6f;
  const float d0 = D1 - D0, d1 = D2 - D1, d2 = D3 - D2;
  const float e0 = 3.f * D1 - D0, e1 = D1 + D2, e2 = D3 - 3.f * D2;
  const float b0 = (13.f / 12.f) * d0 * d0 + 0.25f * e0 * e0;
  const float b1 = (13.f / 12.f) * d1 * d1 + 0.25f * e1 * e1;
  const float b2 = (13.f / 12.f) * d2 * d2 + 0.25f * e2 * e2;
  // alpha_k = d_k / (eps + beta_k)^2 (bounded by d_k / eps^2: no float
  // overflow for any stencil), omega = alpha / sum alpha
  const float i0 = 1.f / (epsw + b0), i1 = 1.f / (epsw + b1), i2 = 1.f / (epsw + b2);
  const float w0 = 0.1f * i0 * i0, w1 = 0.6f * i1 * i1, w2 = 0.3f * i2 * i2;
  const float r0 = 5.f * D1 - 2.f * D0, r1 = 2.f * D2 + D1, r2 = 4.f * D2 - D3;
  const float corr = (w0 * r0 + w1 * r1 + w2 * r2) / (6.f * (w0 + w1 + w2));
  return v0 + (double)corr;
}

}  // namespace vofgb
