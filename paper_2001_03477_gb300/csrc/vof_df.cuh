// vof_df.cuh -- double-float arithmetic (unevaluated sums of two FP32
// numbers, ~48 significant bits) for FP64 arithmetic that decides nothing,
// and the WENO5 face value built on it.
//
// On this part an FP64 instruction occupies an SM partition's FP64 unit as
// long as ~64 FP32 instructions occupy the FP32 units, so a value computed
// with a few dozen FP32 instructions to FP64-like accuracy is far cheaper
// than the same value in FP64.  The error-free transformations are the
// classical ones: TwoSum (Knuth), FastTwoSum (Dekker), TwoProduct with a
// fused multiply-add; the pair operations follow Dekker (1971) and the
// double-double algorithms of Hida, Li & Bailey (QD library paper, 2001),
// restated here.  Conversions between FP64 and pairs are done on the bits
// (integer instructions), not by FP64 conversion instructions.
//
// The file is compiled with -fmad=false: no multiply-add is formed except
// where fmaf() is written, which the error-free transformations rely on.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define VOF_HD __host__ __device__ __forceinline__
#else
#define VOF_HD inline
#endif

namespace vofgb {
namespace df {

struct f2 {
  float hi, lo;
};

VOF_HD uint64_t d_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
VOF_HD double bits_d(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
VOF_HD float bits_f(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
VOF_HD uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
VOF_HD float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return fmaf(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// FP32 value of x * 2^-k with x's significand truncated to 24 bits, from the
// bits (sign, exponent shifted by -k, top 23 stored bits); 0 when the result
// would be below the normal FP32 range.  The caller keeps x * 2^-k below
// 2^127.
VOF_HD float trunc_scale(double x, int k) {
  const uint64_t b = d_bits(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023 - k + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return bits_f((uint32_t)((b >> 32) & 0x80000000u) | 0x7F800000u);  // beyond FP32: infinity
  const uint32_t f = (uint32_t)((b >> 32) & 0x80000000u) | ((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu);
  return bits_f(f);
}

// x * 2^-k as a pair: hi = x with its significand truncated to 24 bits
// (exact in FP32), lo = the rest (one FP64 subtraction, exact), truncated to
// 24 bits: |x 2^-k - (hi + lo)| <= 2^-47 |x 2^-k| (and below 2^-126 for
// parts under the FP32 normal range)
VOF_HD f2 split_scaled(double x, int k) {
  const double xh = bits_d(d_bits(x) & 0xFFFFFFFFE0000000ull);
  const double xl = x - xh;
  return {trunc_scale(xh, k), trunc_scale(xl, k)};
}

// FP64 value of the FP32 number f * 2^k (exact; f normal or zero)
VOF_HD double widen_scaled(float f, int k) {
  const uint32_t b = f_bits(f);
  const uint32_t ef = (b >> 23) & 0xFF;
  if (ef == 0) return 0.0;
  const uint64_t d = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(ef + k - 127 + 1023) << 52) |
                     ((uint64_t)(b & 0x7FFFFFu) << 29);
  return bits_d(d);
}

// error-free transformations
VOF_HD f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
VOF_HD f2 fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = a + b;
  return {s, b - (s - a)};
}
VOF_HD f2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fma_f(a, b, -p)};
}

// pair arithmetic (relative error ~2^-46 without cancellation; the sum's
// error is bounded by ~2^-46 of the operands' magnitudes)
VOF_HD f2 add(f2 x, f2 y) {
  f2 s = two_sum(x.hi, y.hi);
  const f2 t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
VOF_HD f2 neg(f2 x) { return {-x.hi, -x.lo}; }
VOF_HD f2 sub(f2 x, f2 y) { return add(x, neg(y)); }
VOF_HD f2 mul(f2 x, f2 y) {
  f2 p = two_prod(x.hi, y.hi);
  p.lo = fma_f(x.hi, y.lo, fma_f(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// times a small integer constant (exact in FP32)
VOF_HD f2 mul_k(f2 x, float k) {
  f2 p = two_prod(x.hi, k);
  p.lo = fma_f(x.lo, k, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
VOF_HD f2 sqr(f2 x) {
  f2 p = two_prod(x.hi, x.hi);
  p.lo = fma_f(2.0f * x.hi, x.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// x / y: the FP32 quotient, its remainder by one pair product, a correction
VOF_HD f2 div(f2 x, f2 y) {
  const float q1 = x.hi / y.hi;
  const f2 r = sub(x, mul({q1, 0.0f}, y));
  const float q2 = r.hi / y.hi;
  return fast_two_sum(q1, q2);
}

}  // namespace df

// WENO5 face value (Jiang-Shu weights, eps = 1e-6, linear weights 0.1, 0.6,
// 0.3) of the upwind-ordered stencil: the four neighbour differences in FP64,
// the weights and the correction to v0 in pairs, T_f = v0 + correction in
// FP64.  The same reformulation as the FP64 form: candidate values 6 v0 +
// r_k, smoothness indicators scaled by 12/13 with eps (weights unchanged),
// linear weights scaled by 10.  The differences are scaled by a power of
// two 2^-k with the largest near 1 (k >= -20) and eps by 2^-2k, both exact,
// so that no pair overflows or underflows where it matters; the correction
// is scaled back exactly.  Error: ~1e-14 of the largest difference, far
// below the FP64 form's parity bound.
VOF_HD double weno5_df(double vm2, double vm1, double v0, double vp1, double vp2) {
  using namespace df;
  const double D0 = vm1 - vm2, D1 = v0 - vm1, D2 = vp1 - v0, D3 = vp2 - vp1;
  // exponent of the largest |D| (from the bits)
  uint64_t mb = d_bits(D0) & 0x7FFFFFFFFFFFFFFFull;
  uint64_t b1 = d_bits(D1) & 0x7FFFFFFFFFFFFFFFull, b2 = d_bits(D2) & 0x7FFFFFFFFFFFFFFFull,
           b3 = d_bits(D3) & 0x7FFFFFFFFFFFFFFFull;
  mb = mb > b1 ? mb : b1;
  mb = mb > b2 ? mb : b2;
  mb = mb > b3 ? mb : b3;
  if (mb == 0) return v0;
  int k = (int)(mb >> 52) - 1023 + 1;  // max |D| < 2^k
  if (k < -20) k = -20;
  const f2 a0 = split_scaled(D0, k), a1 = split_scaled(D1, k), a2 = split_scaled(D2, k), a3 = split_scaled(D3, k);
  // eps' = 1e-6 * 12/13 * 2^-2k, exact scaling of the FP32 pair of eps'
  const double epsd = 1e-6 * (12.0 / 13.0);
  const f2 eps = split_scaled(epsd, 2 * k);
  const f2 d0 = sub(a1, a0), d1 = sub(a2, a1), d2 = sub(a3, a2);
  const f2 e0 = sub(mul_k(a1, 3.0f), a0), e1 = add(a1, a2), e2 = sub(a3, mul_k(a2, 3.0f));
  const f2 c3 = split_scaled(3.0 / 13.0, 0);  // the ratio of the indicators' two terms, to pair accuracy
  const f2 t0 = add(add(sqr(d0), mul(sqr(e0), c3)), eps);
  const f2 t1 = add(add(sqr(d1), mul(sqr(e1), c3)), eps);
  const f2 t2 = add(add(sqr(d2), mul(sqr(e2), c3)), eps);
  const f2 s0 = sqr(t0), s1 = sqr(t1), s2 = sqr(t2);
  const f2 w0 = mul(s1, s2), w1 = mul_k(mul(s0, s2), 6.0f), w2 = mul_k(mul(s0, s1), 3.0f);
  const f2 r0 = sub(mul_k(a1, 5.0f), mul_k(a0, 2.0f)), r1 = add(mul_k(a2, 2.0f), a1),
           r2 = sub(mul_k(a2, 4.0f), a3);
  const f2 num = add(add(mul(w0, r0), mul(w1, r1)), mul(w2, r2));
  const f2 den = mul_k(add(add(w0, w1), w2), 6.0f);
  const f2 q = div(num, den);
  return v0 + (widen_scaled(q.hi, k) + widen_scaled(q.lo, k));
}

}  // namespace vofgb
