// Double-float arithmetic: a value is an unevaluated sum h + l of two FP32
// numbers with |l| <= ulp(h)/2, about 48 significant bits.  GB300 runs FP64
// at a small fraction of its FP32 rate, so the FP64-accurate sweep keeps
// FP64 bytes in HBM and does its arithmetic here, on the FP32 pipes, with
// error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   * FastTwoSum (Dekker 1971): the same when |a| >= |b|;
//   * TwoProd with an FMA (Ogita, Rump and Oishi, "Accurate sum and dot
//     product", SIAM J. Sci. Comput. 26, 2005): p + e = a b exactly;
//   * the double-word additions and products of Joldes, Muller and Popescu,
//     "Tight and rigorous error bounds for basic building blocks of
//     double-word arithmetic", ACM TOMS 44, 2017 (AccurateDWPlusDW,
//     DWTimesFP3, DWTimesDW1);
//   * dot products accumulated as in Dot2 (Ogita, Rump and Oishi): the high
//     parts of the products summed with TwoSum, every error term in a second
//     FP32 accumulator.
// Every operation is rounded to nearest by the compiler's plain operators;
// nothing here may be contracted or reassociated (the expressions rely on
// the exact rounding of each step), hence the explicit __fadd_rn / __fmul_rn.
#pragma once

#include <stdint.h>

namespace vtm {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// (a.h + a.l) + (b.h + b.l), relative error below 3 u^2 (u = 2^-24)
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  const df t = two_sum(a.l, b.l);
  const df v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// (a.h + a.l) y, relative error below 2 u^2
__device__ __forceinline__ df df_mul_f(df a, float y) {
  const df c = two_prod(a.h, y);
  return fast_two_sum(c.h, __fmaf_rn(a.l, y, c.l));
}

// (a.h + a.l)(b.h + b.l), relative error below 7 u^2
__device__ __forceinline__ df df_mul(df a, df b) {
  const df c = two_prod(a.h, b.h);
  const float tl = __fmaf_rn(a.l, b.h, __fmul_rn(a.h, b.l));
  return fast_two_sum(c.h, __fadd_rn(c.l, tl));
}

// Dot2 accumulator: S collects the high parts of the terms exactly (TwoSum
// errors moved to E), E everything else; the value is S + E.
struct dacc {
  float S, E;
};

// acc += (th + tl)(wh + wl): the product's high part p = rn(th wh) and its
// exact error, plus the two cross terms (tl wl is below the precision kept)
__device__ __forceinline__ void dacc_fma(dacc& a, float th, float tl, float wh, float wl) {
  const float p = __fmul_rn(th, wh);
  float e = __fmaf_rn(th, wh, -p);
  e = __fmaf_rn(th, wl, e);
  e = __fmaf_rn(tl, wh, e);
  const df s = two_sum(a.S, p);
  a.S = s.h;
  a.E = __fadd_rn(a.E, __fadd_rn(s.l, e));
}

// the first term of a fresh accumulator
__device__ __forceinline__ dacc dacc_first(float th, float tl, float wh, float wl) {
  const float p = __fmul_rn(th, wh);
  float e = __fmaf_rn(th, wh, -p);
  e = __fmaf_rn(th, wl, e);
  e = __fmaf_rn(tl, wh, e);
  return {p, e};
}

// a + b of two accumulators
__device__ __forceinline__ dacc dacc_add(dacc a, dacc b) {
  const df s = two_sum(a.S, b.S);
  return {s.h, __fadd_rn(__fadd_rn(a.E, b.E), s.l)};
}

// the accumulator's value as a normalised double-float (TwoSum: S may have
// cancelled below E)
__device__ __forceinline__ df dacc_value(dacc a) { return two_sum(a.S, a.E); }

// Paired forms (two independent values in the two halves of a 64-bit
// register, one FADD2 / FMUL2 / FFMA2 instruction for both): the same
// roundings as dacc_first / dacc_fma, value by value, at half the
// instructions.  A subtraction x - y is the exactly rounded fma(y, -1, x).
struct dacc2 {
  float2 S, E;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ dacc2 dacc2_first(float2 th, float2 tl, float2 wh, float2 wl) {
  const float2 p = __fmul2_rn(th, wh);
  float2 e = __ffma2_rn(th, wh, f2neg(p));
  e = __ffma2_rn(th, wl, e);
  e = __ffma2_rn(tl, wh, e);
  return {p, e};
}

// a += (th + tl)(wh + wl); whn = -wh (the negated product's high part is
// formed directly, so that p = -pn needs no extra instruction)
__device__ __forceinline__ void dacc2_fma(dacc2& a, float2 th, float2 tl, float2 wh, float2 whn, float2 wl) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 pn = __fmul2_rn(th, whn);           // -rn(th wh)
  float2 e = __ffma2_rn(th, wh, pn);               // th wh - p, exact
  e = __ffma2_rn(th, wl, e);
  e = __ffma2_rn(tl, wh, e);
  const float2 s = __ffma2_rn(pn, m1, a.S);        // S + p
  const float2 bb = __ffma2_rn(a.S, m1, s);        // s - S
  const float2 t1 = __ffma2_rn(bb, m1, s);         // s - bb
  const float2 a1 = __ffma2_rn(t1, m1, a.S);       // S - t1
  const float2 a2n = __fadd2_rn(pn, bb);           // -(p - bb)
  const float2 err = __ffma2_rn(a2n, m1, a1);      // (S - t1) + (p - bb)
  a.S = s;
  a.E = __fadd2_rn(a.E, __fadd2_rn(err, e));
}

// Conversions by the bits alone (integer instructions, no FP64 pipe), with
// an exact power-of-two scale.
//
// v 2^-f as a double-float: h = v's leading 24 significant bits (truncated,
// so |l| < ulp(h) rather than ulp(h)/2), l = the next 29 bits (rounded to
// FP32, so h + l keeps about 48 of v's 53 bits).  |v 2^-f| below 2^-126 reads
// as a signed zero, at or above 2^128 as an infinity; an infinity or NaN
// stays one.
__device__ __forceinline__ float2 df_from_double(double v, int f) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((u >> 52) & 0x7ff);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  const unsigned long long M = u & 0xfffffffffffffull;
  if (E == 0x7ff) return make_float2(__uint_as_float(sign | 0x7f800000u | (M ? 0x400000u : 0u)), 0.f);
  const int e = E - 1023 - f;
  if (E == 0 || e < -126) return make_float2(__uint_as_float(sign), 0.f);
  if (e > 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float h = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(M >> 29));
  const float rm = __uint2float_rn((uint32_t)(M & 0x1fffffffu));  // l = rm 2^(e - 52)
  float l = e >= -74 ? __fmul_rn(rm, __uint_as_float((uint32_t)(e - 52 + 127) << 23))
                     : __fmul_rn(__fmul_rn(rm, __uint_as_float((uint32_t)(e + 12 + 127) << 23)),
                                 __uint_as_float((uint32_t)(-64 + 127) << 23));
  return make_float2(h, sign ? -l : l);
}

// x 2^f as a double (exact for a normal x whose scaled exponent fits a
// double; anything else through the FP64 pipe)
__device__ __forceinline__ double double_from_float(float x, int f) {
  const uint32_t u = __float_as_uint(x);
  const int E = (int)((u >> 23) & 0xff);
  const int Ed = E - 127 + f + 1023;
  if (E == 0 || E == 0xff || Ed <= 0 || Ed >= 0x7ff) return ldexp((double)x, f);
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)Ed << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ dacc dacc2_lo(const dacc2& a) { return {a.S.x, a.E.x}; }
__device__ __forceinline__ dacc dacc2_hi(const dacc2& a) { return {a.S.y, a.E.y}; }

}  // namespace vtm
