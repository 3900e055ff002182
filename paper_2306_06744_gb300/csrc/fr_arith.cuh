// fr_arith.cuh -- arithmetic types of the FR kernels.
//
//   double : native FP64 (precision 0).
//   float  : FP32 operators, fluxes, traces and common fluxes (precision 1, and the tensor-core
//            forms 2 and 3 outside their operator contraction); the Runge-Kutta combination
//            stays FP64.
//   ff     : an unevaluated sum hi + lo of two floats ("double-word" arithmetic, precision 4),
//            ~48-bit significand on the FP32 pipes.  GB300 runs FP64 at 1/58 of its FP32 rate, so
//            double-word arithmetic executes FP64-class accuracy several times faster.
//
// The double-word algorithms are the classical error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum and the FMA-based exact product (TwoProd), combined as in Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of double-word arithmetic"
// (ACM TOMS 2017): the "sloppy" sum (error bounded relative to |a|+|b|), the product with one
// FastTwoSum renormalisation, and Newton-corrected quotient and square root.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace frg {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = ff_two_sum(a.h, b.h);
  float e = s.l + (a.l + b.l);
  return ff_fast_two_sum(s.h, e);
}
__device__ __forceinline__ ff operator-(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);  // exact error of the leading product
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff fma_t(ff a, ff b, ff c) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  ff s = ff_two_sum(p, c.h);
  float t = s.l + (e + c.l);
  return ff_fast_two_sum(s.h, t);
}
// quotient: q1 = a/b in float, one Newton correction with the exact residual a - q1*b
__device__ __forceinline__ ff operator/(ff a, ff b) {
  float q1 = __fdividef(a.h, b.h);
  ff r = a - ff{q1, 0.f} * b;
  float q2 = __fdividef(r.h, b.h);
  ff q = ff_fast_two_sum(q1, q2);
  r = a - q * b;
  float q3 = __fdividef(r.h, b.h);
  return q + ff{q3, 0.f};
}
__device__ __forceinline__ ff sqrt_t(ff a) {
  if (a.h <= 0.f) return {0.f, 0.f};
  float s = sqrtf(a.h);
  ff r = a - ff{s, 0.f} * ff{s, 0.f};
  float c = __fdividef(r.h, 2.f * s);
  ff q = ff_fast_two_sum(s, c);
  r = a - q * q;
  return q + ff{__fdividef(r.h, 2.f * q.h), 0.f};
}
__device__ __forceinline__ ff fabs_t(ff a) { return a.h < 0.f ? -a : a; }
__device__ __forceinline__ bool lt_t(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ ff fmax_t(ff a, ff b) { return lt_t(a, b) ? b : a; }

// Dot-product accumulator for double-word operands (the compensated dot product of Ogita, Rump
// and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005, with double-word
// operands): the running sum of the leading products in one float, every rounding error (the
// exact error of each leading product, the cross terms, the TwoSum error of each addition)
// gathered in a second float, and one renormalisation at the end instead of one per term.
struct ffacc {
  float s, c;
};
__device__ __forceinline__ void ffacc_fma(ffacc& A, ff a, ff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const ff t = ff_two_sum(A.s, p);
  A.s = t.h;
  A.c += t.l + e;
}
__device__ __forceinline__ ff ffacc_fin(ffacc A) { return ff_two_sum(A.s, A.c); }

// double -> ff by integer manipulation of the bit pattern (no FP64 instruction): hi keeps the
// leading 24 significand bits (truncated), lo the next bits of the remainder; exact to 2^-47
// relative for normal doubles whose exponent lies in [-74, 127]; smaller magnitudes keep hi only.
__device__ __forceinline__ ff ff_from_double(double x) {
  uint64_t b = uint64_t(__double_as_longlong(x));
  uint32_t sign = uint32_t(b >> 63) << 31;
  int E = int((b >> 52) & 0x7FF) - 1023;
  uint64_t m = b & 0xFFFFFFFFFFFFFull;
  if (E < -126) return {__int_as_float(int(sign)), 0.f};  // zero or below float range
  float hi = __int_as_float(int(sign | (uint32_t(E + 127) << 23) | uint32_t(m >> 29)));
  uint32_t r = uint32_t(m & 0x1FFFFFFFu);  // remaining 29 bits, weight 2^(E-52)
  float lo = 0.f;
  if (r != 0u && E >= -74) {
    float scale = __int_as_float((E - 52 + 127) << 23);
    lo = __uint2float_rz(r) * scale;
    if (sign) lo = -lo;
  }
  return ff_fast_two_sum(hi, lo);  // renormalise: |lo| <= ulp(hi)/2
}

// float -> double by integer widening (normal floats and zero; subnormal floats become zero)
__device__ __forceinline__ double f_to_double_bits(float f) {
  uint32_t u = uint32_t(__float_as_int(f));
  uint32_t e = (u >> 23) & 0xFF;
  if (e == 0u) return __longlong_as_double((long long)(uint64_t(u >> 31) << 63));
  uint64_t db = (uint64_t(u >> 31) << 63) | (uint64_t(e - 127 + 1023) << 52) |
                (uint64_t(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)db);
}
__device__ __forceinline__ double ff_to_double(ff a) {
  return f_to_double_bits(a.h) + f_to_double_bits(a.l);  // one FP64 add
}

// ---- uniform interface over the three types ----
template <class T>
struct Ar;

template <>
struct Ar<double> {
  static __device__ __forceinline__ double from_d(double x) { return x; }
  static __device__ __forceinline__ double to_d(double x) { return x; }
  static __device__ __forceinline__ double c(double x) { return x; }
};
// double -> float by integer manipulation of the bit pattern (no FP64-rate conversion): the
// significand is cut to 24 bits and rounded half away from zero (a carry moves into the exponent);
// magnitudes below 2^-126 become a signed zero, above the float range infinity, NaN stays NaN.
__device__ __forceinline__ float f32_from_double_bits(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const uint32_t sign = uint32_t(b >> 63) << 31;
  const int E = int((b >> 52) & 0x7FF) - 1023;
  if (E < -126) return __int_as_float(int(sign));
  if (E > 127)
    return __int_as_float(int(sign | ((E == 1024 && (b & 0xFFFFFFFFFFFFFull)) ? 0x7FC00000u : 0x7F800000u)));
  uint32_t mag = (uint32_t(E + 127) << 23) | uint32_t((b >> 29) & 0x7FFFFFu);
  mag += uint32_t((b >> 28) & 1u);
  return __int_as_float(int(sign | mag));
}

template <>
struct Ar<float> {
  static __device__ __forceinline__ float from_d(double x) { return f32_from_double_bits(x); }
  static __device__ __forceinline__ double to_d(float x) { return f_to_double_bits(x); }
};
template <>
struct Ar<ff> {
  static __device__ __forceinline__ ff from_d(double x) { return ff_from_double(x); }
  static __device__ __forceinline__ double to_d(ff x) { return ff_to_double(x); }
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
// reciprocals: FP64 by Newton-Raphson from the hardware approximation (two iterations square the
// relative error twice, from ~2^-23 to below the FP64 rounding error); FP32 by the fast divide;
// double-word by the corrected quotient above.
__device__ __forceinline__ double rcp_t(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ ff rcp_t(ff x) { return ff{1.f, 0.f} / x; }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double sqrt_t(double a) { return sqrt(a); }
__device__ __forceinline__ float sqrt_t(float a) { return sqrtf(a); }
__device__ __forceinline__ double fabs_t(double a) { return fabs(a); }
__device__ __forceinline__ float fabs_t(float a) { return fabsf(a); }
__device__ __forceinline__ double fmax_t(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmax_t(float a, float b) { return fmaxf(a, b); }

// zero / constant helpers
template <class T>
__device__ __forceinline__ T zero_t() {
  return T(0);
}
template <>
__device__ __forceinline__ ff zero_t<ff>() {
  return ff{0.f, 0.f};
}

}  // namespace frg
