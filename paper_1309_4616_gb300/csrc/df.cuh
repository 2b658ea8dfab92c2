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
