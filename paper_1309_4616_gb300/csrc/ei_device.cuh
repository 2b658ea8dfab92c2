// Device-side building blocks shared by the kernel translation units:
// arithmetic over the three vector formats (float-float pairs, double,
// float), loads and stores, block reductions and the last-block pattern.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "df.cuh"
#include "ei_internal.h"

namespace ei {

#define EI_BX 32
#define EI_BY 8
#define EI_ZC 16
#define EI_TPB 256

// ---------------------------------------------------------------------------
// scalar arithmetic over the three formats
// ---------------------------------------------------------------------------
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double mac(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ float mac(float acc, float a, float b) { return fmaf(a, b, acc); }
__device__ __forceinline__ df add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df sub(df a, df b) { return df_sub(a, b); }
__device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df mac(df acc, df a, df b) { return df_mac(acc, a, b); }

template <class T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ df zero<df>() { return df{0.0f, 0.0f}; }

template <class T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ df from_d<df>(double x) { return df_from_double(x); }

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(df x) { return df_to_double(x); }

// widen a vector value to the Newton-sum type
__device__ __forceinline__ df to_p(df x) { return x; }
__device__ __forceinline__ df to_p(float x) { return df{x, 0.0f}; }
__device__ __forceinline__ double to_p(double x) { return x; }

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// A double as a signed 64-bit key whose integer order is the value order:
// negative values get their magnitude bits inverted (-0 sorts just below +0).
// A NaN sorts beyond the infinity of its sign bit.  The transform is its own
// inverse.  Running min/max on keys keep the comparisons off the FP64 pipe.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_value(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}


// Verdict after the Newton step reaching degree `deg`, with squared norms nw2
// of w_deg and np2 of p_deg and coefficient d = d_deg.  Adaptive mode: stop
// at the first degree whose estimate |d| ||w|| <= tol ||p|| holds (done = 1),
// or at m_max (done = 2).  Fixed-count mode: only deg == m_max is judged, and
// a failed check also counts into ctl->fixfail.  Non-finite norms stop with
// done = 4 in both modes, and a bounded device wait that ran out (ctl->err)
// with done = 5.  Returns true when the iteration stops at `deg`.  Called by
// one thread after the grid-wide reduction.
// Bracket steps (s.bracket, adaptive mode): the squared norms are known only
// to lie in [nw2, nw2_hi] and [np2, np2_hi].  The test is decided where the
// brackets decide it for every value inside them (with a 1e-9 margin for the
// rounding of the comparison); otherwise, or where a bracket left FP64's
// normal range (an Inf or NaN among the values included), the step stops
// with done = 6 and the host forms both norms and takes the test.
__device__ __forceinline__ bool newton_verdict(DevCtl* ctl, const NewtonScalars& s, int deg,
                                               double d, double nw2, double np2,
                                               double nw2_hi = -1.0, double np2_hi = -1.0) {
  const bool last = deg >= s.m_max;
  if (*(volatile int*)&ctl->err) {
    ctl->done = 5;
    ctl->degree = deg;
    if (s.fixed) atomicAdd(&ctl->fixfail, 1);
    return true;
  }
  if (s.bracket && nw2_hi >= 0.0) {
    const bool normal = nw2_hi < INFINITY && np2_hi < INFINITY && nw2 >= 0x1p-1000 &&
                        np2 >= 0x1p-1000;
    if (normal) {
      const double a_lo = fabs(d) * sqrt(nw2), a_hi = fabs(d) * sqrt(nw2_hi);
      const double b_lo = s.tol * sqrt(np2), b_hi = s.tol * sqrt(np2_hi);
      if (a_hi * (1.0 + 1e-9) <= b_lo) {  // converged for every value in the brackets
        ctl->done = 1;
        ctl->degree = deg;
        return true;
      }
      if (a_lo > b_hi * (1.0 + 1e-9)) {  // fails for every value in the brackets
        if (!last) return false;
        ctl->done = 2;
        ctl->degree = deg;
        return true;
      }
    }
    ctl->done = 6;
    ctl->degree = deg;
    return true;
  }
  if (!finite_d(nw2) || !finite_d(np2)) {
    ctl->done = 4;
    ctl->degree = deg;
    if (s.fixed) atomicAdd(&ctl->fixfail, 1);
    return true;
  }
  if (deg == 1 && s.j == 0 && np2 == 0.0 && nw2 == 0.0) {  // zero input: p = 0 at degree 0
    ctl->done = 1;
    ctl->degree = 0;
    return true;
  }
  if (s.fixed && !last) return false;
  if (fabs(d) * sqrt(nw2) <= s.tol * sqrt(np2)) {
    ctl->done = 1;
    ctl->degree = deg;
    return true;
  }
  if (last) {
    ctl->done = 2;
    ctl->degree = deg;
    if (s.fixed) atomicAdd(&ctl->fixfail, 1);
    return true;
  }
  return false;
}

// Bracket steps of the native FP64 Newton kernels (NewtonScalars::bracket):
// ||w_{j+1}||^2 and ||p_{j+1}||^2 are bracketed by FP32 sums of t^2, t being
// the value cut to its high word by integer operations: sign cleared, exponent
// rebiased so that the previous step's root mean square lands near 1 (scale
// 2^k, from ctl->nw2 and ctl->np2), 20 mantissa bits kept.  Then
// t <= |v| 2^k < t (1 + 2^-20) wherever t is a normal float; a |v| below that
// range gives t = 0, one above it (or an Inf or NaN) t = Inf.  The FP64 pipe
// is left to the iteration itself.
struct NormBrackets {
  int kw = 0, kp = 0, rw = 896 << 20, rp = 896 << 20;  // 896: FP64's exponent bias less FP32's
  float aw = 0.f, ap = 0.f;
  double npts = 1.0;
  // the scale exponent that brings a mean square ms to about 1, 0 where ms
  // is 0 or not finite
  static __device__ __forceinline__ int scale_exp(double ms) {
    if (!(ms > 0.0 && ms < INFINITY)) return 0;
    return max(-480, min(480, -(ilogb(ms) >> 1)));
  }
  // |v| 2^k cut to a float (rebias = (896 - k) << 20)
  static __device__ __forceinline__ float cut(double v, int rebias) {
    const int r = min(max((__double2hiint(v) & 0x7fffffff) - rebias, 0), 0x0ff00000);
    return __int_as_float(r << 3);
  }
  // 2^(-2k), exact
  static __device__ __forceinline__ double unscale(int k) {
    return __hiloint2double((1023 - 2 * k) << 20, 0);
  }
  __device__ __forceinline__ void init(const DevCtl* ctl, double n) {
    npts = n;
    kw = scale_exp(ctl->nw2 / n);
    kp = scale_exp(ctl->np2 / n);
    rw = (896 - kw) << 20;
    rp = (896 - kp) << 20;
  }
  __device__ __forceinline__ void add(double w, double p) {
    const float tw = cut(w, rw), tp = cut(p, rp);
    aw = fmaf(tw, tw, aw);
    ap = fmaf(tp, tp, ap);
  }
  // this thread's sums back in the unscaled units (exact)
  __device__ __forceinline__ double sum_w() const { return (double)aw * unscale(kw); }
  __device__ __forceinline__ double sum_p() const { return (double)ap * unscale(kp); }
  // The verdict on the grid's sums nw2, np2 of sum_w, sum_p, `terms` the most
  // values one thread added.  Each thread's FP32 sum has at most `terms`
  // roundings of relative 2^-24 (gam bounds their effect), each cut value
  // lies within a factor 1 + 2^-20 below the true magnitude, and a value that
  // left FP32's normal range or a square that went subnormal is off by less
  // than 2^-140 in the rebiased scale (slack).  The FP64 reductions of the
  // thread sums add far less than the 1e-9 margins.
  __device__ __forceinline__ bool verdict(DevCtl* ctl, const NewtonScalars& s, double nw2,
                                          double np2, double terms) const {
    const double gam = terms * 0x1p-24 / (1.0 - terms * 0x1p-24);
    const double cut2 = (1.0 + 0x1p-20) * (1.0 + 0x1p-20);
    const double sw = npts * 0x1p-140 * unscale(kw), sp = npts * 0x1p-140 * unscale(kp);
    auto lo = [&](double v, double slack) {
      return fmax(v - slack, 0.0) / (1.0 + gam) * (1.0 - 1e-9);
    };
    auto hi = [&](double v, double slack) {
      return (v / (1.0 - gam) * (1.0 + 1e-9) + slack) * cut2;
    };
    return newton_verdict(ctl, s, s.j + 1, s.d_next, lo(nw2, sw), lo(np2, sp), hi(nw2, sw),
                          hi(np2, sp));
  }
};

// Gershgorin min/max accumulation of one row's bounds.  fmin/fmax drop a NaN
// operand, so a row with a NaN bound widens the pair to (-inf, +inf) instead:
// the host's finiteness check of the interval then sees it.
__device__ __forceinline__ void minmax_row(double& mn, double& mx, double lo, double hi) {
  if (isnan(lo) || isnan(hi)) {
    mn = -INFINITY;
    mx = INFINITY;
    return;
  }
  mn = fmin(mn, lo);
  mx = fmax(mx, hi);
}

// loads / stores (read-only path for data the kernel does not write)
__device__ __forceinline__ df ldg(const df* p, int64_t i) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
  return df{v.x, v.y};
}
__device__ __forceinline__ double ldg(const double* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float ldg(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ df ld(const df* p, int64_t i) {
  float2 v = reinterpret_cast<const float2*>(p)[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ double ld(const double* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ void st(df* p, int64_t i, df v) {
  reinterpret_cast<float2*>(p)[i] = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ void st(double* p, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ void st(float* p, int64_t i, float v) { p[i] = v; }

// 7-point sum diag*wc + sum_k a_k*w_k and the Newton update
// w' = (A w)*inv_gamma - shift*wc.  Float-float: two lazily normalised
// accumulators (independent chains for instruction-level parallelism);
// float: two chains of FMAs; double: one chain.
__device__ __forceinline__ df stencil7(df dg, df wc, df a0, df w0, df a1, df w1, df a2, df w2,
                                       df a3, df w3, df a4, df w4, df a5, df w5) {
  dfacc s1 = dfa_mul(dg, wc);
  dfacc s2 = dfa_mul(a3, w3);
  s1 = dfa_mac(s1, a0, w0);
  s2 = dfa_mac(s2, a4, w4);
  s1 = dfa_mac(s1, a1, w1);
  s2 = dfa_mac(s2, a5, w5);
  s1 = dfa_mac(s1, a2, w2);
  return dfa_norm(dfa_add(s1, s2));
}
// Native FP64: one chain of a multiply and six FMAs.  The FP64 pipe, not the
// latency of the chain, bounds these kernels (a GB300 SM retires about two FP64
// FMA lanes a clock), so the shortest instruction count wins.
__device__ __forceinline__ double stencil7(double dg, double wc, double a0, double w0, double a1,
                                           double w1, double a2, double w2, double a3, double w3,
                                           double a4, double w4, double a5, double w5) {
  double s = dg * wc;
  s = fma(a0, w0, s);
  s = fma(a1, w1, s);
  s = fma(a2, w2, s);
  s = fma(a3, w3, s);
  s = fma(a4, w4, s);
  return fma(a5, w5, s);
}
__device__ __forceinline__ float stencil7(float dg, float wc, float a0, float w0, float a1,
                                          float w1, float a2, float w2, float a3, float w3,
                                          float a4, float w4, float a5, float w5) {
  float s1 = dg * wc, s2 = a3 * w3;
  s1 = fmaf(a0, w0, s1);
  s2 = fmaf(a4, w4, s2);
  s1 = fmaf(a1, w1, s1);
  s2 = fmaf(a5, w5, s2);
  s1 = fmaf(a2, w2, s1);
  return s1 + s2;
}
__device__ __forceinline__ df newton_update(df Aw, df invg, df nshift, df wc) {
  return dfa_norm(dfa_mac(dfa_mul(Aw, invg), nshift, wc));
}
__device__ __forceinline__ double newton_update(double Aw, double invg, double nshift,
                                                double wc) {
  return fma(nshift, wc, Aw * invg);
}
__device__ __forceinline__ float newton_update(float Aw, float invg, float nshift, float wc) {
  return fmaf(nshift, wc, Aw * invg);
}
// ---------------------------------------------------------------------------
// The combustion term of Sec. III-C, g(u) = (2 - u) e^{20 (1 - 1/u)} / 4, and
// g'(u) = e^{20 (1 - 1/u)} (20 (2 - u) / u^2 - 1) / 4; both 0 for u <= 0.025
// (their limit as u -> 0+).  A NaN u gives NaN.
// - float-float: the format's own reciprocal and exponential (df.cuh);
// - double (the native FP64 format): the math library's exp and IEEE division;
// - float: expf and IEEE division;
// - fast (any format): __expf and __fdividef in FP32, the hardware
//   approximations (the paper's "fast math" variant).
// ---------------------------------------------------------------------------
constexpr float COMBUSTION_CUT = 0.025f;
__device__ __forceinline__ void combustion_eval(df u, df& g, df& dg) {
  if (u.hi <= COMBUSTION_CUT) {
    g = df{0.0f, 0.0f};
    dg = df{0.0f, 0.0f};
    return;
  }
  const df q = df_recip(u);
  const df e4 = df_mul(df{0.25f, 0.0f}, df_exp(df_mul(df{20.0f, 0.0f}, df_add(df{1.0f, 0.0f}, df_neg(q)))));
  const df tm = df_add(df{2.0f, 0.0f}, df_neg(u));
  g = df_mul(e4, tm);
  const df t = df_mul(df_mul(df{20.0f, 0.0f}, tm), df_mul(q, q));
  dg = df_mul(e4, df_add(t, df{-1.0f, 0.0f}));
}
__device__ __forceinline__ void combustion_eval(double u, double& g, double& dg) {
  if (u <= (double)COMBUSTION_CUT) {
    g = 0.0;
    dg = 0.0;
    return;
  }
  const double q = 1.0 / u;
  const double e4 = 0.25 * exp(20.0 * (1.0 - q));
  g = e4 * (2.0 - u);
  dg = e4 * (20.0 * (2.0 - u) * q * q - 1.0);
}
__device__ __forceinline__ void combustion_eval(float u, float& g, float& dg) {
  if (u <= COMBUSTION_CUT) {
    g = 0.0f;
    dg = 0.0f;
    return;
  }
  const float q = 1.0f / u;
  const float e4 = 0.25f * expf(20.0f * (1.0f - q));
  g = e4 * (2.0f - u);
  dg = e4 * (20.0f * (2.0f - u) * q * q - 1.0f);
}
__device__ __forceinline__ void combustion_fast(float u, float& g, float& dg) {
  if (u <= COMBUSTION_CUT) {
    g = 0.0f;
    dg = 0.0f;
    return;
  }
  const float q = __fdividef(1.0f, u);
  const float e4 = 0.25f * __expf(20.0f * (1.0f - q));
  g = e4 * (2.0f - u);
  dg = e4 * (20.0f * (2.0f - u) * q * q - 1.0f);
}
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(df x) { return x.hi; }
// g(u) and g'(u) of a combustion nonlinearity (EI_NONLIN_COMBUSTION or
// EI_NONLIN_COMBUSTION_FAST) in the vector format T
template <class T>
__device__ __forceinline__ void combustion_term(int nonlin, T u, T& g, T& dg) {
  if (nonlin == EI_NONLIN_COMBUSTION_FAST) {
    float gf, dgf;
    combustion_fast(to_f(u), gf, dgf);
    g = from_d<T>((double)gf);
    dg = from_d<T>((double)dgf);
  } else {
    combustion_eval(u, g, dg);
  }
}

// squared-norm accumulators: lazily normalised pairs for float-float values
template <class T> struct Acc {
  using type = T;
  static __device__ __forceinline__ T zero() { return T(0); }
};
template <> struct Acc<df> {
  using type = dfacc;
  static __device__ __forceinline__ dfacc zero() { return dfacc{0.0f, 0.0f}; }
};
__device__ __forceinline__ double acc_sq(double a, double x) { return fma(x, x, a); }
__device__ __forceinline__ float acc_sq(float a, float x) { return fmaf(x, x, a); }
__device__ __forceinline__ dfacc acc_sq(dfacc a, df x) { return dfa_mac(a, x, x); }
__device__ __forceinline__ double acc_d(double a) { return a; }
__device__ __forceinline__ double acc_d(float a) { return (double)a; }
__device__ __forceinline__ double acc_d(dfacc a) { return (double)a.s + (double)a.t; }

// accumulate / finish a row sum (two independent chains; float-float lazily
// normalised)
__device__ __forceinline__ dfacc lmac(dfacc c, df a, df b) { return dfa_mac(c, a, b); }
__device__ __forceinline__ double lmac(double c, double a, double b) { return fma(a, b, c); }
__device__ __forceinline__ float lmac(float c, float a, float b) { return fmaf(a, b, c); }
__device__ __forceinline__ df lsum(dfacc a, dfacc b) { return dfa_norm(dfa_add(a, b)); }
__device__ __forceinline__ double lsum(double a, double b) { return a + b; }
__device__ __forceinline__ float lsum(float a, float b) { return a + b; }

// butterfly exchange within a warp (all 32 lanes take part)
__device__ __forceinline__ double shfl_x(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float shfl_x(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df shfl_x(df v, int m) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// CSR row pipelining (ei_kernels.cu, ei_complex.cu): rows walk a grid-stride
// loop; each thread prefetches the first CSR_PFC columns of its next row into
// its own shared-memory slots with cp.async.
constexpr int CSR_PF = 12;
constexpr int CSR_PFC = 20;
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// the first CSR_PFC columns of entries [b, e) into this thread's slots
__device__ __forceinline__ void csr_prefetch_cols(int32_t (*slot)[EI_TPB], const int32_t* col,
                                                  int64_t b, int64_t e) {
#pragma unroll
  for (int q = 0; q < CSR_PFC; ++q)
    if (b + q < e) cp_async4(&slot[q][threadIdx.x], col + b + q);
}


template <int FMT> struct VT;
template <> struct VT<VF_DF> { using T = df; using P = df; };
template <> struct VT<VF_F64> { using T = double; using P = double; };
template <> struct VT<VF_F32> { using T = float; using P = df; };

// ---------------------------------------------------------------------------
// block reductions and the last-block pattern
// ---------------------------------------------------------------------------
// RED_SUM: (a, b) summed; RED_MINMAX: min of a, max of b; RED_SUMMAX: a summed,
// max of b (b >= 0)
enum { RED_SUM = 0, RED_MINMAX = 1, RED_SUMMAX = 2 };

template <int OP>
__device__ __forceinline__ void comb(double& a, double& b, double a2, double b2) {
  if (OP == RED_SUM) {
    a += a2;
    b += b2;
  } else if (OP == RED_SUMMAX) {
    a += a2;
    b = fmax(b, b2);
  } else {
    a = fmin(a, a2);
    b = fmax(b, b2);
  }
}

// Reduce (a, b) over the block; result valid in thread 0.  Fixed order.
// Blocks of 256 threads first halve through shared memory (128, 64, then 32
// threads add), then one warp finishes by shuffles: about 12 warp-wide adds a
// value instead of 45 for eight warps of shuffles, which matters on GB300's
// narrow FP64 pipe.  Other block sizes shuffle in every warp.
template <int OP>
__device__ __forceinline__ void block_reduce2(double& a, double& b) {
  __shared__ double sa[256], sb[256];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  if (nthr == 256) {
    sa[tid] = a;
    sb[tid] = b;
    __syncthreads();
#pragma unroll
    for (int h = 128; h >= 32; h >>= 1) {
      if (tid < h) {
        double a2 = sa[tid + h], b2 = sb[tid + h];
        comb<OP>(a, b, a2, b2);
        if (h > 32) {
          sa[tid] = a;
          sb[tid] = b;
        }
      }
      if (h > 32) __syncthreads();
    }
    if (tid < 32) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        double a2 = __shfl_down_sync(0xffffffffu, a, off);
        double b2 = __shfl_down_sync(0xffffffffu, b, off);
        comb<OP>(a, b, a2, b2);
      }
    }
    __syncthreads();
    return;
  }
  const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double a2 = __shfl_down_sync(0xffffffffu, a, off);
    double b2 = __shfl_down_sync(0xffffffffu, b, off);
    comb<OP>(a, b, a2, b2);
  }
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  const int nw = (nthr + 31) >> 5;
  if (wid == 0) {
    if (OP == RED_SUM || OP == RED_SUMMAX) {
      a = lane < nw ? sa[lane] : 0.0;
      b = lane < nw ? sb[lane] : 0.0;
    } else {
      a = lane < nw ? sa[lane] : INFINITY;
      b = lane < nw ? sb[lane] : -INFINITY;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double a2 = __shfl_down_sync(0xffffffffu, a, off);
      double b2 = __shfl_down_sync(0xffffffffu, b, off);
      comb<OP>(a, b, a2, b2);
    }
  }
  __syncthreads();
}

// Every block publishes its pair; the last block to arrive reduces all pairs
// in block order and returns true (in all its threads) with the totals.
template <int OP>
__device__ bool last_block_reduce2(double& a, double& b, double* partials, DevCtl* ctl) {
  __shared__ bool am_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_reduce2<OP>(a, b);
  if (tid == 0) {
    partials[2 * bid] = a;
    partials[2 * bid + 1] = b;
    __threadfence();
    unsigned t = atomicAdd(&ctl->count, 1u);
    am_last = (t == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double ra = (OP == RED_MINMAX) ? INFINITY : 0.0, rb = (OP == RED_MINMAX) ? -INFINITY : 0.0;
  for (unsigned i = tid; i < nblk; i += nthr) {
    comb<OP>(ra, rb, __ldcg(partials + 2 * i), __ldcg(partials + 2 * i + 1));
  }
  block_reduce2<OP>(ra, rb);
  __shared__ double fa, fb;
  if (tid == 0) {
    fa = ra;
    fb = rb;
    ctl->count = 0;
  }
  __syncthreads();
  a = fa;
  b = fb;
  return true;
}


// Four values in two pairs, v[0..1] combined by OPA and v[2..3] by OPB (sums
// by default): every block publishes its four partials; the last block to
// arrive combines them in block order.  Returns true (in all its threads)
// there.
template <int OPA = RED_SUM, int OPB = RED_SUM>
__device__ inline bool last_block_reduce4(double v[4], double* partials, DevCtl* ctl) {
  __shared__ bool am_last4;
  __shared__ double f4[4];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
  const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_reduce2<OPA>(v[0], v[1]);
  block_reduce2<OPB>(v[2], v[3]);
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) partials[4 * bid + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(&ctl->count, 1u);
    am_last4 = (t == nblk - 1);
  }
  __syncthreads();
  if (!am_last4) return false;
  __threadfence();
  double r[4] = {OPA == RED_MINMAX ? INFINITY : 0.0, OPA == RED_MINMAX ? -INFINITY : 0.0,
                 OPB == RED_MINMAX ? INFINITY : 0.0, OPB == RED_MINMAX ? -INFINITY : 0.0};
  for (unsigned i = tid; i < nblk; i += nthr) {
    comb<OPA>(r[0], r[1], __ldcg(partials + 4 * i), __ldcg(partials + 4 * i + 1));
    comb<OPB>(r[2], r[3], __ldcg(partials + 4 * i + 2), __ldcg(partials + 4 * i + 3));
  }
  block_reduce2<OPA>(r[0], r[1]);
  block_reduce2<OPB>(r[2], r[3]);
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) f4[k] = r[k];
    ctl->count = 0;
  }
  __syncthreads();
  for (int k = 0; k < 4; ++k) v[k] = f4[k];
  return true;
}

}  // namespace ei
