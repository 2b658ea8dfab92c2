// Float-float ("double-float") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// a 48-bit significand (unit roundoff 2^-48 ~ 3.6e-15).  GB300 issues FP64
// FMAs at ~1/70 of its FP32 rate, so the "FP64" vectors of the Newton loop are
// stored and updated in this format: the same 8 bytes per value as a double,
// with arithmetic that stays under the HBM roofline.
//
// The error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, the
// FMA-based TwoProd) use explicitly rounded intrinsics so that the compiler
// can neither contract nor reassociate them.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

struct __align__(8) df {
  float hi, lo;
};

__device__ __forceinline__ df df_from_float(float a) { return df{a, 0.0f}; }

// exact: s + e == a + b
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// exact when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// acc + a*b with one renormalisation
__device__ __forceinline__ df df_mac(df acc, df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  t = __fadd_rn(t, __fadd_rn(acc.lo, e));
  df r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}

// a*a accumulated: acc + a^2 (used for squared norms)
__device__ __forceinline__ df df_sqr_acc(df acc, df a) { return df_mac(acc, a, a); }

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_from_double(double x) {
  float hi = __double2float_rn(x);
  float lo = __double2float_rn(x - (double)hi);
  return df{hi, lo};
}

__host__ inline df df_from_double_host(double x) {
  float hi = (float)x;
  float lo = (float)(x - (double)hi);
  return df{hi, lo};
}

// ---- lazily normalised accumulation ------------------------------------------
// An unevaluated pair s + t whose t collects the exact rounding errors of the
// running sum s (TwoSum) and of each product (FMA-TwoProd plus the two cross
// terms); one renormalisation at the end.  Per multiply-add 12 FP32 operations
// instead of 15, with the same 2^-48-relative error on the terms.
struct dfacc {
  float s, t;
};

__device__ __forceinline__ dfacc dfa_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfacc{p, e};
}

__device__ __forceinline__ dfacc dfa_mac(dfacc c, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, err;
  two_sum(c.s, p, s, err);
  return dfacc{s, __fadd_rn(c.t, __fadd_rn(err, e))};
}

__device__ __forceinline__ dfacc dfa_add(dfacc a, dfacc b) {
  float s, err;
  two_sum(a.s, b.s, s, err);
  return dfacc{s, __fadd_rn(__fadd_rn(a.t, b.t), err)};
}

// s + t renormalised with TwoSum (no ordering assumption on |s|, |t|)
__device__ __forceinline__ df dfa_norm(dfacc c) {
  df r;
  two_sum(c.s, c.t, r.hi, r.lo);
  return r;
}

// ---- reciprocal and exponential -------------------------------------------
// 1/a: Newton-Raphson from the float reciprocal, q = q0 + q0 (1 - a q0), one
// step doubling the 24 correct bits of q0 to the format's 48.
__device__ __forceinline__ df df_recip(df a) {
  const float q0 = 1.0f / a.hi;
  const df e = df_add(df{1.0f, 0.0f}, df_neg(df_mul(a, df{q0, 0.0f})));
  return df_mac(df{q0, 0.0f}, df{q0, 0.0f}, e);
}

// e^x, written from the mathematics:
// - Cody-Waite argument reduction x = k ln2 + r, k = rint(x / ln2), with ln 2
//   split in three floats.  The first carries 16 significant bits, so k*L1 is
//   exact for |k| < 256, and k*L2 is formed exactly by an FMA.
// - The Taylor series of e^r for |r| <= ln2/2 to degree 12 in Horner form.
//   Truncation is below 2e-16 relative.
// - 2^k applied to both halves.
// The split constants are ln 2 to 60 digits cut into floats:
//   L1 = 0x1.62e4p-1, L2 = 0x1.7f7d1cp-20, L3 = 0x1.ef357ap-45.
// The residual of the split is 1.3e-21.  The coefficients are 1/i!, rounded
// from double.  The float exponent range limits the result: +inf above
// x = 88, 0 below x = -87.
struct df_fact_inv {
  static constexpr __host__ __device__ double v(int i) { return i <= 1 ? 1.0 : v(i - 1) / i; }
  // 1/i! as a float-float pair, formed at compile time
  static constexpr __host__ __device__ float hi(int i) { return (float)v(i); }
  static constexpr __host__ __device__ float lo(int i) { return (float)(v(i) - (double)(float)v(i)); }
};
__device__ __forceinline__ df df_exp(df x) {
  if (x.hi > 88.0f) return df{INFINITY, 0.0f};
  if (!(x.hi >= -87.0f)) return x.hi != x.hi ? x : df{0.0f, 0.0f};  // NaN passes through
  constexpr float L1 = 0x1.62e4p-1f, L2 = 0x1.7f7d1cp-20f, L3 = 0x1.ef357ap-45f;
  const float k = rintf(x.hi * 1.44269504088896341f);
  df r = df_add(x, df{-k * L1, 0.0f});
  const float p2 = k * L2;
  r = df_add(r, df{-p2, -__fmaf_rn(k, L2, -p2)});
  r = df_add(r, df{-k * L3, 0.0f});
#define EI_DF_C(i) df{df_fact_inv::hi(i), df_fact_inv::lo(i)}
  df p = EI_DF_C(12);
  p = df_mac(EI_DF_C(11), p, r);
  p = df_mac(EI_DF_C(10), p, r);
  p = df_mac(EI_DF_C(9), p, r);
  p = df_mac(EI_DF_C(8), p, r);
  p = df_mac(EI_DF_C(7), p, r);
  p = df_mac(EI_DF_C(6), p, r);
  p = df_mac(EI_DF_C(5), p, r);
  p = df_mac(EI_DF_C(4), p, r);
  p = df_mac(EI_DF_C(3), p, r);
  p = df_mac(EI_DF_C(2), p, r);
  p = df_mac(df{1.0f, 0.0f}, p, r);
  p = df_mac(df{1.0f, 0.0f}, p, r);
#undef EI_DF_C
  const int ki = (int)k;
  return df{ldexpf(p.hi, ki), ldexpf(p.lo, ki)};
}

// ---- double -> float-float without the FP64 pipe ----------------------------
// From the IEEE-754 fields: hi = sign, exponent and the top 23 fraction bits
// (x cut to 24 significant bits, exact as a float); lo = the remaining 29
// fraction bits as an integer converted to float and scaled by 2^(e - 52),
// exact up to its single rounding; a fast two-sum renormalises the pair
// (|lo| < ulp(hi)).  Zeros, and magnitudes below 2^-150 (zero in the format's
// range), give signed zeros; the few others outside [2^-96, 2^128) -- float
// subnormal range, huge, infinite, NaN -- take df_from_double.  The result agrees with df_from_double
// to the format's precision (both keep 48 of the 53 bits).
__device__ __forceinline__ float df_pow2f(int k) {  // 2^k as a float, k >= -149
  return k >= -126 ? __uint_as_float((unsigned)(k + 127) << 23)
                   : __uint_as_float(1u << (k + 149));
}
__device__ __forceinline__ df df_split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  if ((b << 1) == 0ull) return df{__uint_as_float(hw & 0x80000000u), 0.0f};  // +-0
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
  // below 2^-150 the float-float value is a signed zero (the format's range)
  if (e < -150) return df{__uint_as_float(hw & 0x80000000u), 0.0f};
  if (e < -96 || e > 127) return df_from_double(x);
  const unsigned sgn = hw & 0x80000000u;
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) |
                                   ((hw & 0xfffffu) << 3) | (lw >> 29));
  float lo = __uint2float_rn(lw & 0x1fffffffu) * df_pow2f(e - 52);
  lo = sgn ? -lo : lo;
  df r;
  fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}
