// Double-word arithmetic on the FP32 pipe (device code only).
//
// On this part the FP64 pipe issues ~528 G operations/s, the FP32 pipe ~38
// T/s: a double-word operation -- a value held as an unevaluated pair (h, l)
// of floats, h = RN(h + l) -- costs 6 to 20 FP32 instructions, several times
// less than one FP64 operation.  The algorithms are Dekker's (1971) exact
// transforms and the double-word building blocks of Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017 (u = 2^-24):
//   add(DW, DW)  their AccurateDWPlusDW,  relative error <= 3u^2 + 13u^3
//   add(DW, FP)  DWPlusFP,                <= 2u^2
//   mul(DW, DW)  DWTimesDW3 (with fma),   <= 4u^2
//   mul(DW, FP)  DWTimesFP3,              <= 2u^2
// so a double-word value carries ~48 bits, against fp64's 53.  Every float
// operation below is an explicit round-to-nearest intrinsic, so the compiler
// cannot contract or reorder what the transforms rely on.
//
// Conversions from and to fp64 work on the bit patterns with integer
// instructions (the F2F conversion instructions run at the FP64 pipe's rate
// on this part), and take a power-of-two scale 2^shift on the way, so callers
// keep the float exponents in a safe range and carry the scale separately.
#pragma once

#include <cuda_runtime.h>

namespace dw {

struct f2 {
  float h, l;
};

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return {s, __fsub_rn(b, z)};
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  return {s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}

__device__ __forceinline__ f2 add(f2 x, f2 y) {
  const f2 s = two_sum(x.h, y.h);
  const f2 t = two_sum(x.l, y.l);
  const f2 v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}

__device__ __forceinline__ f2 add(f2 x, float y) {
  const f2 s = two_sum(x.h, y);
  return fast_two_sum(s.h, __fadd_rn(x.l, s.l));
}

__device__ __forceinline__ f2 neg(f2 x) { return {-x.h, -x.l}; }
__device__ __forceinline__ f2 sub(f2 x, f2 y) { return add(x, neg(y)); }

__device__ __forceinline__ f2 mul(f2 x, f2 y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

__device__ __forceinline__ f2 mul(f2 x, float y) {
  const float ch = __fmul_rn(x.h, y);
  const float cl1 = __fmaf_rn(x.h, y, -ch);
  return fast_two_sum(ch, __fmaf_rn(x.l, y, cl1));
}

// x * y + z
__device__ __forceinline__ f2 fma(f2 x, f2 y, f2 z) { return add(mul(x, y), z); }

// 1/y: the float reciprocal t, then one Newton step in double-word,
// t + t (1 - y t); relative error ~ (2^-23)^2 + a few u^2.  y normal, nonzero.
__device__ __forceinline__ f2 rcp(f2 y) {
  const float t = __frcp_rn(y.h);
  const f2 e = add(neg(mul(y, t)), 1.0f);  // 1 - y t, small
  return add(mul(e, t), t);
}

// Binade of a nonzero normal float (bit pattern).
__device__ __forceinline__ int exponent(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF) - 127; }

// x * 2^p for an integer p in [-126, 127] (exact while the result is normal)
__device__ __forceinline__ f2 ldexp(f2 x, int p) {
  const float s = __uint_as_float((unsigned)(p + 127) << 23);
  return {__fmul_rn(x.h, s), __fmul_rn(x.l, s)};
}

// Unbiased binary exponent of a finite nonzero double (bit pattern).
__device__ __forceinline__ int exponent(double x) { return (int)((__double2hiint(x) >> 20) & 0x7FF) - 1023; }

// x 2^shift as a double-word: h = x 2^shift rounded to 24 bits, l = the
// remainder (29 bits, rounded to 24 by the integer-to-float conversion), so
// h + l = x 2^shift to a relative 2^-49.  Requires the result's exponent
// E = exponent(x) + shift <= 126; a result below 2^-74 (and zero) gives 0,
// so callers scale their data to magnitudes near 1 first.
__device__ __forceinline__ f2 from_double(double x, int shift = 0) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int E = e - 1023 + shift;
  if (e == 0 || E < -74) return {0.f, 0.f};
  const unsigned sign = hi & 0x80000000u;
  const unsigned top = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // 23 fraction bits
  const unsigned r = lo & 0x1FFFFFFFu;                       // the other 29
  const unsigned up = r >> 28;                               // round h to nearest
  const int rs = (int)r - (int)(up << 29);                   // |rs| <= 2^28
  const float h = __uint_as_float(sign | ((((unsigned)(E + 127)) << 23) + top + up));
  const float l = __fmul_rn(__int2float_rn(rs), __uint_as_float((unsigned)(E - 52 + 127) << 23));
  return {h, __uint_as_float(__float_as_uint(l) ^ sign)};
}

// (h + l) 2^shift rounded to fp64 (faithfully: to one of the two neighbours),
// for a normalized pair (|l| <= ulp(h)/2) whose result is a normal double.
__device__ __forceinline__ double to_double(f2 x, int shift = 0) {
  const unsigned hb = __float_as_uint(x.h), lb = __float_as_uint(x.l);
  const int eh = (int)((hb >> 23) & 0xFFu);
  if (eh == 0) return 0.0;
  // value = M 2^(E - 62) with h's 24-bit significand at bits 62..39 of M
  long long M = (long long)(((hb & 0x7FFFFFu) | 0x800000u)) << 39;
  const int el = (int)((lb >> 23) & 0xFFu);
  if (el != 0) {
    const long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
    const int d = eh - el;  // >= 24 for a normalized pair
    const long long a = d <= 39 ? (ml << (39 - d)) : (d < 63 ? (ml >> (d - 39)) : 0);
    M = ((hb ^ lb) & 0x80000000u) ? M - a : M + a;
  }
  int E = eh - 127 + shift;
  if (M < (1LL << 62)) {  // h a power of two and l < 0: one bit lower
    M <<= 1;
    E -= 1;
  }
  unsigned long long R = (unsigned long long)M + (1ull << 9);  // round at bit 10
  if (R >> 63) {
    R >>= 1;
    E += 1;
  }
  const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                  ((unsigned long long)(E + 1023) << 52) | ((R >> 10) & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

}  // namespace dw
