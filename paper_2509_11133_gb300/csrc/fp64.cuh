// FP64 helpers of the element kernels (device code only).
#pragma once

#include <cuda_runtime.h>

namespace ph {

// On this part FP64 arithmetic issues at 2 operations per clock per SM, 1/32
// of the integer ALU rate, and the element kernels are bound by it.  Sign
// flips and range tests are therefore done on the bit pattern with integer
// instructions (IEEE negation is a flip of the sign bit), and 1/x uses a
// short Newton iteration instead of a correctly rounded divide.

// n ? -x : x, bit-exact with IEEE negation
__device__ __forceinline__ double neg_if(double x, bool n) {
  const unsigned hi = (unsigned)__double2hiint(x) ^ ((unsigned)n << 31);
  return __hiloint2double((int)hi, __double2loint(x));
}
__device__ __forceinline__ double negate(double x) { return neg_if(x, true); }

// 0 < x < +inf (false for zeros, negatives, infinities and NaN)
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}

// 1/x by the Newton-Raphson iteration for the reciprocal, y <- y + y (1 - x y)
// (quadratic convergence), seeded from the single-precision hardware
// approximation rcp.approx of the top 20 mantissa bits of x (relative error
// below 2^-19, so two steps reach full double precision: relative error of
// the result below 2^-52, i.e. within an ulp of the rounded quotient).
// x outside [2^-1020, 2^1021) -- including zero, negative, infinite and NaN
// x -- takes the IEEE divide.
__device__ __forceinline__ double rcp_newton(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const int ex = (int)(hi >> 20);  // biased exponent; >= 2048 when the sign bit is set
  if (ex < 3 || ex > 2043) return 1.0 / x;
  const float m = __uint_as_float(0x3F800000u | ((hi & 0x000FFFFFu) << 3));  // mantissa in [1, 2)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));  // r in (0.5, 1]
  const unsigned rb = __float_as_uint(r);
  const int e_out = (int)(rb >> 23) - 127 - (ex - 1023) + 1023;  // in [2, 2043]
  const unsigned yhi = ((unsigned)e_out << 20) | ((rb & 0x007FFFFFu) >> 3);
  double y = __hiloint2double((int)yhi, (int)((rb & 0x7u) << 29));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// sqrt(x)/2 (a triangle's area from the squared norm x of its edge cross
// product) by the coupled Newton iteration for sqrt(q) and 1/(2 sqrt(q)),
// q = x/4 (Goldschmidt's method, as in Markstein, IBM J. Res. Dev. 34(1),
// 1990).  The seed y ~ 1/sqrt(q) is the single-precision hardware
// approximation rsqrt.approx of q's top 23 mantissa bits with q's exponent
// halved (relative error below 2^-22); then, with g = q y and h = y/2,
//     r = 1/2 - g h,   g <- g + g r,   h <- h + h r    (error ~1.5 e^2 < 2^-43)
//     d = q - g g (exact by fma),   g <- g + d h      (error ~e^2, then rounding)
// so the result is within an ulp of sqrt(x)/2: 6 FP64 operations.  x outside
// [2^-960, 2^960) -- including zero, subnormal, negative, infinite and NaN x
// -- takes 0.5 * sqrt(x).
__device__ __forceinline__ double half_sqrt(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)(hi >> 20);  // biased exponent; >= 2048 when the sign bit is set
  if (ex < 63 || ex > 1982) return 0.5 * sqrt(x);
  const double q = __hiloint2double((int)(hi - (2u << 20)), (int)lo);  // x/4, exact
  const int e = ex - 2 - 1023;                                          // q = m 2^e, m in [1, 2)
  const int k = e >> 1, p = e & 1;                                      // e = 2k + p
  const float f = __uint_as_float(((unsigned)(127 + p) << 23) | ((hi & 0x000FFFFFu) << 3) | (lo >> 29));
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));  // f = m 2^p in [1, 4), r about 1/sqrt(f)
  const unsigned rb = __float_as_uint(r);
  // y = r 2^-k, built on the bit pattern (biased exponent in [500, 1550])
  const unsigned yhi = ((unsigned)((int)(rb >> 23) - 127 - k + 1023) << 20) | ((rb & 0x007FFFFFu) >> 3);
  const int ylo = (int)((rb & 0x7u) << 29);
  double h = __hiloint2double((int)(yhi - (1u << 20)), ylo);  // y/2
  double g = q * __hiloint2double((int)yhi, ylo);
  const double t = fma(-g, h, 0.5);
  g = fma(g, t, g);
  h = fma(h, t, h);
  return fma(fma(-g, g, q), h, g);
}

}  // namespace ph
