// CUDA kernels of the Leja exponential-integrator hot path (sm_103a).
//
// The hot loop is one fused kernel per Newton iteration (Eq. (3): products
// (alpha*A + beta*I)x with alpha = 1/gamma, beta = -(c/gamma + xi_j)):
//     w_{j+1} = (A w_j)/gamma - (c/gamma + xi_j) w_j,   p += d_{j+1} w_{j+1},
// fused with the squared norms ||w_{j+1}||^2, ||p||^2 (block partials, a
// fixed-order last-block reduction) and the device-side stop test, so that a
// whole Newton loop can be launched without host round trips.  A is a
// matrix-free stencil with the boundary conditions folded in (Sec. III-A) and
// position-dependent coefficients read from arrays (Sec. III-B), or CSR
// (Sec. III-D).
//
// Vector formats: float-float pairs (FP64-accurate on the FP32 pipes), IEEE
// double (for comparison), float (reduced-precision form).  The Newton sum p
// is float-float except in the double format.
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
__device__ __forceinline__ void st(df* p, int64_t i, df v) {
  reinterpret_cast<float2*>(p)[i] = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ void st(double* p, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ void st(float* p, int64_t i, float v) { p[i] = v; }

template <int FMT> struct VT;
template <> struct VT<VF_DF> { using T = df; using P = df; };
template <> struct VT<VF_F64> { using T = double; using P = double; };
template <> struct VT<VF_F32> { using T = float; using P = df; };

// ---------------------------------------------------------------------------
// block reductions and the last-block pattern
// ---------------------------------------------------------------------------
enum { RED_SUM = 0, RED_MINMAX = 1 };

template <int OP>
__device__ __forceinline__ void comb(double& a, double& b, double a2, double b2) {
  if (OP == RED_SUM) {
    a += a2;
    b += b2;
  } else {
    a = fmin(a, a2);
    b = fmax(b, b2);
  }
}

// Reduce (a, b) over the block; result valid in thread 0.  Fixed order.
template <int OP>
__device__ __forceinline__ void block_reduce2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
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
    if (OP == RED_SUM) {
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
  double ra = (OP == RED_SUM) ? 0.0 : INFINITY, rb = (OP == RED_SUM) ? 0.0 : -INFINITY;
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

// ---------------------------------------------------------------------------
// the stencil operator at one grid point
// ---------------------------------------------------------------------------
// (A w)_i = sum_e r_e [ (D_i + D_{i+e})(w_{i+e} - w_i) + (D_i + D_{i-e})(w_{i-e} - w_i) ]
//         + sum_e B_e,i (w_{i+e} - w_{i-e}) + qc_i w_i
// with D pre-scaled by 1/(2 dx_x^2) and B_e by 1/(2 dx_e).  A missing
// neighbour is a ghost: 0 (Dirichlet) or w_i (Neumann); its D is D_i.
template <class T, int DIM>
__device__ __forceinline__ T stencil_apply(const StencilDev& op, const T* __restrict__ w,
                                           const T* __restrict__ qc, int x, int y, int z,
                                           int64_t idx, T& wc) {
  const T* __restrict__ D = static_cast<const T*>(op.D);
  wc = ldg(w, idx);
  const T Dc = ldg(D, idx);
  const T zro = zero<T>();
  T acc;
  {  // x
    const bool hm = x > 0, hp = x < op.nx - 1;
    const T wm = hm ? ldg(w, idx - 1) : (op.bc[0] ? wc : zro);
    const T wp = hp ? ldg(w, idx + 1) : (op.bc[1] ? wc : zro);
    const T Dm = hm ? ldg(D, idx - 1) : Dc;
    const T Dp = hp ? ldg(D, idx + 1) : Dc;
    acc = mul(add(Dc, Dp), sub(wp, wc));
    acc = mac(acc, add(Dc, Dm), sub(wm, wc));
    acc = mac(acc, ldg(static_cast<const T*>(op.B[0]), idx), sub(wp, wm));
  }
  {  // y
    const int64_t s = op.nx;
    const bool hm = y > 0, hp = y < op.ny - 1;
    const T wm = hm ? ldg(w, idx - s) : (op.bc[2] ? wc : zro);
    const T wp = hp ? ldg(w, idx + s) : (op.bc[3] ? wc : zro);
    const T Dm = hm ? ldg(D, idx - s) : Dc;
    const T Dp = hp ? ldg(D, idx + s) : Dc;
    T ay = mul(add(Dc, Dp), sub(wp, wc));
    ay = mac(ay, add(Dc, Dm), sub(wm, wc));
    acc = op.uniform ? add(acc, ay) : mac(acc, from_d<T>(op.ratio[1]), ay);
    acc = mac(acc, ldg(static_cast<const T*>(op.B[1]), idx), sub(wp, wm));
  }
  if (DIM == 3) {  // z
    const int64_t s = (int64_t)op.nx * op.ny;
    const bool hm = z > 0, hp = z < op.nz - 1;
    const T wm = hm ? ldg(w, idx - s) : (op.bc[4] ? wc : zro);
    const T wp = hp ? ldg(w, idx + s) : (op.bc[5] ? wc : zro);
    const T Dm = hm ? ldg(D, idx - s) : Dc;
    const T Dp = hp ? ldg(D, idx + s) : Dc;
    T az = mul(add(Dc, Dp), sub(wp, wc));
    az = mac(az, add(Dc, Dm), sub(wm, wc));
    acc = op.uniform ? add(acc, az) : mac(acc, from_d<T>(op.ratio[2]), az);
    acc = mac(acc, ldg(static_cast<const T*>(op.B[2]), idx), sub(wp, wm));
  }
  return mac(acc, ldg(qc, idx), wc);
}

// ---------------------------------------------------------------------------
// the fused Newton iteration, stencil
// ---------------------------------------------------------------------------
template <int FMT, int DIM>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_newton(StencilDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
                 void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const T* __restrict__ w_in = static_cast<const T*>(w_in_);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const int x = blockIdx.x * EI_BX + threadIdx.x;
  const int y = blockIdx.y * EI_BY + threadIdx.y;
  const int z0 = blockIdx.z * EI_ZC;
  const int z1 = min(z0 + EI_ZC, op.nz);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  T aw = zero<T>();
  P ap = zero<P>();
  if (x < op.nx && y < op.ny) {
    for (int z = z0; z < z1; ++z) {
      const int64_t idx = ((int64_t)z * op.ny + y) * op.nx + x;
      T wc;
      const T Aw = stencil_apply<T, DIM>(op, w_in, qc, x, y, z, idx, wc);
      const T wn = mac(mul(Aw, invg), nshift, wc);
      const P pold = (s.j == 0) ? mul(d0, to_p(wc)) : ld(p, idx);
      const P pn = mac(pold, dn, to_p(wn));
      st(w_out, idx, wn);
      st(p, idx, pn);
      aw = mac(aw, wn, wn);
      ap = mac(ap, pn, pn);
    }
  }
  double nw2 = to_d(aw), np2 = to_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      if (!finite_d(nw2) || !finite_d(np2)) {
        ctl->done = 4;
        ctl->degree = s.j + 1;
      } else if (s.j == 0 && np2 == 0.0) {  // zero input: p = 0 at degree 0
        ctl->done = 1;
        ctl->degree = 0;
      } else if (fabs(s.d_next) * sqrt(nw2) <= s.tol * sqrt(np2)) {
        ctl->done = 1;
        ctl->degree = s.j + 1;
      } else if (s.j + 1 >= s.m_max) {
        ctl->done = 2;
        ctl->degree = s.j + 1;
      }
    }
  }
}

// r = A y + v, ||r||^2
template <int FMT, int DIM>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_residual(StencilDev op, const void* __restrict__ y_, const void* __restrict__ v_,
                   void* __restrict__ r_, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ yv = static_cast<const T*>(y_);
  const T* __restrict__ v = static_cast<const T*>(v_);
  T* __restrict__ r = static_cast<T*>(r_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const int x = blockIdx.x * EI_BX + threadIdx.x;
  const int y = blockIdx.y * EI_BY + threadIdx.y;
  const int z0 = blockIdx.z * EI_ZC;
  const int z1 = min(z0 + EI_ZC, op.nz);
  T ar = zero<T>();
  if (x < op.nx && y < op.ny) {
    for (int z = z0; z < z1; ++z) {
      const int64_t idx = ((int64_t)z * op.ny + y) * op.nx + x;
      T yc;
      const T Ay = stencil_apply<T, DIM>(op, yv, qc, x, y, z, idx, yc);
      const T rv = add(Ay, ldg(v, idx));
      st(r, idx, rv);
      ar = mac(ar, rv, rv);
    }
  }
  double a = to_d(ar), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) ctl->sum0 = a;
  }
}

// F = A u + g(u) (A with the base diagonal c), qc_out = c + g'(u) (Rosenbrock) or c
template <int FMT, int DIM>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_F(StencilDev op, const void* __restrict__ u_, void* __restrict__ F_,
            void* __restrict__ qc_out_, const void* __restrict__ cbase_, int nonlin,
            int rosenbrock, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ u = static_cast<const T*>(u_);
  const T* __restrict__ cb = static_cast<const T*>(cbase_);
  T* __restrict__ F = static_cast<T*>(F_);
  T* __restrict__ qo = static_cast<T*>(qc_out_);
  const int x = blockIdx.x * EI_BX + threadIdx.x;
  const int y = blockIdx.y * EI_BY + threadIdx.y;
  const int z0 = blockIdx.z * EI_ZC;
  const int z1 = min(z0 + EI_ZC, op.nz);
  const T one = from_d<T>(1.0);
  T af = zero<T>();
  if (x < op.nx && y < op.ny) {
    for (int z = z0; z < z1; ++z) {
      const int64_t idx = ((int64_t)z * op.ny + y) * op.nx + x;
      T uc;
      T Fv = stencil_apply<T, DIM>(op, u, cb, x, y, z, idx, uc);
      if (nonlin) Fv = mac(Fv, uc, sub(one, uc));  // g(u) = u(1-u)
      st(F, idx, Fv);
      if (rosenbrock) {
        T q = ldg(cb, idx);
        if (nonlin) q = add(q, mac(one, from_d<T>(-2.0), uc));  // g'(u) = 1 - 2u
        st(qo, idx, q);
      }
      af = mac(af, Fv, Fv);
    }
  }
  double a = to_d(af), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      ctl->sum0 = a;
      ctl->sum1 = finite_d(a) ? 1.0 : 0.0;
    }
  }
}


// ---------------------------------------------------------------------------
// CSR operator (Sec. III-D): a group of EI_LPR lanes per row.  The paper found
// four threads per row best for its matrix; rows of the random geometric graph
// carry ~12 entries, so a 4-lane group reads three entries per lane.
// ---------------------------------------------------------------------------
#define EI_LPR 4

template <class T>
__device__ __forceinline__ T shfl_xor_T(T v, int m);
template <> __device__ __forceinline__ double shfl_xor_T<double>(double v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
template <> __device__ __forceinline__ float shfl_xor_T<float>(float v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
template <> __device__ __forceinline__ df shfl_xor_T<df>(df v, int m) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// (W x)_row over the lane group; every lane of the group gets the full sum
template <class T>
__device__ __forceinline__ T csr_row(const CsrDev& op, const T* __restrict__ x, int64_t row,
                                     bool valid, int lane) {
  T acc = zero<T>();
  if (valid) {
    const T* __restrict__ val = static_cast<const T*>(op.val);
    const int64_t b = __ldg(op.rowptr + row), e = __ldg(op.rowptr + row + 1);
    for (int64_t k = b + lane; k < e; k += EI_LPR) acc = mac(acc, ldg(val, k), ldg(x, __ldg(op.col + k)));
  }
#pragma unroll
  for (int m = EI_LPR / 2; m > 0; m >>= 1) acc = add(acc, shfl_xor_T(acc, m));
  return acc;
}

template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_csr_newton(CsrDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
             void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const T* __restrict__ w_in = static_cast<const T*>(w_in_);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const int lane = threadIdx.x % EI_LPR;
  const int64_t rows_per_iter = (int64_t)gridDim.x * (EI_TPB / EI_LPR);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  T aw = zero<T>();
  P ap = zero<P>();
  for (int64_t base = (int64_t)blockIdx.x * (EI_TPB / EI_LPR); base < op.n; base += rows_per_iter) {
    const int64_t row = base + threadIdx.x / EI_LPR;
    const bool valid = row < op.n;
    const T Wx = csr_row<T>(op, w_in, row, valid, lane);
    if (valid && lane == 0) {
      const T wc = ldg(w_in, row);
      const T Aw = mac(Wx, ldg(qc, row), wc);
      const T wn = mac(mul(Aw, invg), nshift, wc);
      const P pold = (s.j == 0) ? mul(d0, to_p(wc)) : ld(p, row);
      const P pn = mac(pold, dn, to_p(wn));
      st(w_out, row, wn);
      st(p, row, pn);
      aw = mac(aw, wn, wn);
      ap = mac(ap, pn, pn);
    }
  }
  double nw2 = to_d(aw), np2 = to_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      if (!finite_d(nw2) || !finite_d(np2)) {
        ctl->done = 4;
        ctl->degree = s.j + 1;
      } else if (s.j == 0 && np2 == 0.0) {
        ctl->done = 1;
        ctl->degree = 0;
      } else if (fabs(s.d_next) * sqrt(nw2) <= s.tol * sqrt(np2)) {
        ctl->done = 1;
        ctl->degree = s.j + 1;
      } else if (s.j + 1 >= s.m_max) {
        ctl->done = 2;
        ctl->degree = s.j + 1;
      }
    }
  }
}

template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_csr_residual(CsrDev op, const void* __restrict__ y_, const void* __restrict__ v_,
               void* __restrict__ r_, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ yv = static_cast<const T*>(y_);
  const T* __restrict__ v = static_cast<const T*>(v_);
  T* __restrict__ r = static_cast<T*>(r_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const int lane = threadIdx.x % EI_LPR;
  const int64_t rows_per_iter = (int64_t)gridDim.x * (EI_TPB / EI_LPR);
  T ar = zero<T>();
  for (int64_t base = (int64_t)blockIdx.x * (EI_TPB / EI_LPR); base < op.n; base += rows_per_iter) {
    const int64_t row = base + threadIdx.x / EI_LPR;
    const bool valid = row < op.n;
    const T Wy = csr_row<T>(op, yv, row, valid, lane);
    if (valid && lane == 0) {
      const T rv = add(mac(Wy, ldg(qc, row), ldg(yv, row)), ldg(v, row));
      st(r, row, rv);
      ar = mac(ar, rv, rv);
    }
  }
  double a = to_d(ar), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) ctl->sum0 = a;
  }
}

template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_csr_F(CsrDev op, const void* __restrict__ u_, void* __restrict__ F_, void* __restrict__ qo_,
        const void* __restrict__ cb_, int nonlin, int rosenbrock, double* partials,
        DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ u = static_cast<const T*>(u_);
  const T* __restrict__ cb = static_cast<const T*>(cb_);
  T* __restrict__ F = static_cast<T*>(F_);
  T* __restrict__ qo = static_cast<T*>(qo_);
  const int lane = threadIdx.x % EI_LPR;
  const int64_t rows_per_iter = (int64_t)gridDim.x * (EI_TPB / EI_LPR);
  const T one = from_d<T>(1.0);
  T af = zero<T>();
  for (int64_t base = (int64_t)blockIdx.x * (EI_TPB / EI_LPR); base < op.n; base += rows_per_iter) {
    const int64_t row = base + threadIdx.x / EI_LPR;
    const bool valid = row < op.n;
    const T Wu = csr_row<T>(op, u, row, valid, lane);
    if (valid && lane == 0) {
      const T uc = ldg(u, row);
      T Fv = mac(Wu, ldg(cb, row), uc);
      if (nonlin) Fv = mac(Fv, uc, sub(one, uc));
      st(F, row, Fv);
      if (rosenbrock) {
        T q = ldg(cb, row);
        if (nonlin) q = add(q, mac(one, from_d<T>(-2.0), uc));
        st(qo, row, q);
      }
      af = mac(af, Fv, Fv);
    }
  }
  double a = to_d(af), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->sum0 = a;
      ctl->sum1 = finite_d(a) ? 1.0 : 0.0;
    }
  }
}

// Gershgorin rows of A = W + diag: a_ii = diag_i + sum_{col==row} w, r_i = sum_{col!=row} |w|
template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_csr_gershgorin(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                 const U* __restrict__ val, const U* __restrict__ diag, double* lo, double* hi,
                 double* partials, DevCtl* ctl) {
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = diag ? (double)diag[i] : 0.0, r = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double a = (double)val[k];
      if (col[k] == i) d += a; else r += fabs(a);
    }
    lo[i] = d - r;
    hi[i] = d + r;
    mn = fmin(mn, d - r);
    mx = fmax(mx, d + r);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

// ---------------------------------------------------------------------------
// Gershgorin interval (FP64, from the caller's arrays)
// ---------------------------------------------------------------------------
template <class U>
__device__ __forceinline__ double uval(const void* p, double cst, int64_t i) {
  return p ? (double)__ldg(static_cast<const U*>(p) + i) : cst;
}

template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_gershgorin(int dim, int nx, int ny, int nz, int bc0, int bc1, int bc2, int bc3,
                     int bc4, int bc5, double dx0, double dx1, double dx2, const void* D,
                     double Dc, const void* b0, const void* b1, const void* b2, double bc_0,
                     double bc_1, double bc_2, const void* c, double cc, double* lo,
                     double* hi, double* partials, DevCtl* ctl) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int bcs[6] = {bc0, bc1, bc2, bc3, bc4, bc5};
  const double dxs[3] = {dx0, dx1, dx2};
  const void* bs[3] = {b0, b1, b2};
  const double bcst[3] = {bc_0, bc_1, bc_2};
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((int64_t)nx * ny));
    const int crd[3] = {x, y, z};
    const int ext[3] = {nx, ny, nz};
    const int64_t str[3] = {1, nx, (int64_t)nx * ny};
    const double Di = uval<U>(D, Dc, i);
    double diag = uval<U>(c, cc, i), rad = 0.0;
    for (int e = 0; e < dim; ++e) {
      const double h2 = dxs[e] * dxs[e];
      const double be = uval<U>(bs[e], bcst[e], i);
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const bool has = sgn < 0 ? crd[e] > 0 : crd[e] < ext[e] - 1;
        const int face = 2 * e + (sgn > 0);
        if (has) {
          const double Df = 0.5 * (Di + uval<U>(D, Dc, i + sgn * str[e]));
          rad += fabs(Df / h2 + sgn * be / (2.0 * dxs[e]));
          diag -= Df / h2;
        } else if (bcs[face] == 1) {
          diag += sgn * be / (2.0 * dxs[e]);
        } else {
          diag -= Di / h2;
        }
      }
    }
    lo[i] = diag - rad;
    hi[i] = diag + rad;
    mn = fmin(mn, diag - rad);
    mx = fmax(mx, diag + rad);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

// min/max of (lo + q), (hi + q), q = g'(u) = 1 - 2u for the logistic g
template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_shifted_minmax(int64_t n, const double* __restrict__ lo, const double* __restrict__ hi,
                 const U* __restrict__ u, int nonlin, double* partials, DevCtl* ctl) {
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double q = nonlin ? 1.0 - 2.0 * (double)u[i] : 0.0;
    mn = fmin(mn, lo[i] + q);
    mx = fmax(mx, hi[i] + q);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

// ---------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------
template <int FMT, class U>
__global__ void k_fill_coef(void* dst_, int64_t n, const U* src, double cst, double scale) {
  using T = typename VT<FMT>::T;
  T* dst = static_cast<T*>(dst_);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (src ? (double)src[i] : cst) * scale;
    st(dst, i, from_d<T>(v));
  }
}

template <int FMT, class U>
__global__ void __launch_bounds__(EI_TPB)
k_import(void* dst_, const U* __restrict__ src, int64_t n, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  T* dst = static_cast<T*>(dst_);
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i];
    st(dst, i, from_d<T>(v));
    a = fma(v, v, a);
  }
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->sum0 = a;
      ctl->sum1 = finite_d(a) ? 1.0 : 0.0;
    }
  }
}

template <class S, class U>
__global__ void k_export(U* dst, const S* __restrict__ src, int64_t n, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dst[i] = (U)(to_d(ldg(src, i)) * scale);
  }
}

template <class S, class U>
__global__ void k_add_export(U* u, const S* __restrict__ y, int64_t n, double scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    u[i] = (U)fma(to_d(ldg(y, i)), scale, (double)u[i]);
  }
}

template <int FMT>
__global__ void k_p_to_vec(void* dst_, const void* p_, int64_t n) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  T* dst = static_cast<T*>(dst_);
  const P* p = static_cast<const P*>(p_);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (FMT == VF_F32) {
      st(dst, i, (float)to_d(ldg(p, i)));
    } else {
      st(dst, i, ldg(p, i));
    }
  }
}

// y += tau * p  (y in vector format, p in the Newton-sum format)
template <int FMT>
__global__ void k_axpy(void* y_, const void* p_, int64_t n, double tau) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  T* y = static_cast<T*>(y_);
  const P* p = static_cast<const P*>(p_);
  const P t = from_d<P>(tau);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const P v = mac(to_p(ldg(y, i)), t, ldg(p, i));
    if constexpr (FMT == VF_F32) {
      st(y, i, (float)to_d(v));
    } else {
      st(y, i, v);
    }
  }
}

template <int FMT>
__global__ void k_zero(void* x_, int64_t n) {
  using T = typename VT<FMT>::T;
  T* x = static_cast<T*>(x_);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    st(x, i, zero<T>());
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static int ew_blocks(int64_t n) {
  int64_t b = (n + EI_TPB - 1) / EI_TPB;
  int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

static dim3 stencil_grid(const StencilDev& op) {
  return dim3((op.nx + EI_BX - 1) / EI_BX, (op.ny + EI_BY - 1) / EI_BY,
              (op.nz + EI_ZC - 1) / EI_ZC);
}

int stencil_blocks(const StencilDev& op) {
  dim3 g = stencil_grid(op);
  return (int)(g.x * g.y * g.z);
}

int reduction_capacity() { return num_sms() * 8; }

int csr_blocks(int64_t n) {
  int64_t b = (n + (EI_TPB / 4) - 1) / (EI_TPB / 4);
  int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

#define EI_DISPATCH_FMT(fmt, KERNEL_CALL)        \
  switch (fmt) {                                 \
    case VF_DF: { constexpr int F_ = VF_DF; KERNEL_CALL; } break;   \
    case VF_F64: { constexpr int F_ = VF_F64; KERNEL_CALL; } break; \
    default: { constexpr int F_ = VF_F32; KERNEL_CALL; } break;     \
  }

cudaError_t launch_stencil_newton(const StencilDev& op, const void* w_in, void* w_out, void* p,
                                  const NewtonScalars& s, int fmt, double* partials,
                                  DevCtl* ctl, cudaStream_t stm) {
  dim3 g = stencil_grid(op), b(EI_BX, EI_BY, 1);
  if (op.dim == 3) {
    EI_DISPATCH_FMT(fmt, (k_stencil_newton<F_, 3><<<g, b, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_stencil_newton<F_, 2><<<g, b, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl)));
  }
  return cudaGetLastError();
}

cudaError_t launch_stencil_residual(const StencilDev& op, const void* y, const void* v, void* r,
                                    int fmt, double* partials, DevCtl* ctl, cudaStream_t stm) {
  dim3 g = stencil_grid(op), b(EI_BX, EI_BY, 1);
  if (op.dim == 3) {
    EI_DISPATCH_FMT(fmt, (k_stencil_residual<F_, 3><<<g, b, 0, stm>>>(op, y, v, r, partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_stencil_residual<F_, 2><<<g, b, 0, stm>>>(op, y, v, r, partials, ctl)));
  }
  return cudaGetLastError();
}

cudaError_t launch_stencil_F(const StencilDev& op, const void* u, void* F, void* qc_out,
                             const void* c_base, int nonlin, int rosenbrock, int fmt,
                             double* partials, DevCtl* ctl, cudaStream_t stm) {
  dim3 g = stencil_grid(op), b(EI_BX, EI_BY, 1);
  if (op.dim == 3) {
    EI_DISPATCH_FMT(fmt, (k_stencil_F<F_, 3><<<g, b, 0, stm>>>(op, u, F, qc_out, c_base, nonlin, rosenbrock, partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_stencil_F<F_, 2><<<g, b, 0, stm>>>(op, u, F, qc_out, c_base, nonlin, rosenbrock, partials, ctl)));
  }
  return cudaGetLastError();
}


cudaError_t launch_csr_newton(const CsrDev& op, const void* w_in, void* w_out, void* p,
                              const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                              cudaStream_t stm) {
  const int nb = csr_blocks(op.n);
  EI_DISPATCH_FMT(fmt, (k_csr_newton<F_><<<nb, EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl)));
  return cudaGetLastError();
}

cudaError_t launch_csr_residual(const CsrDev& op, const void* y, const void* v, void* r, int fmt,
                                double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = csr_blocks(op.n);
  EI_DISPATCH_FMT(fmt, (k_csr_residual<F_><<<nb, EI_TPB, 0, stm>>>(op, y, v, r, partials, ctl)));
  return cudaGetLastError();
}

cudaError_t launch_csr_F(const CsrDev& op, const void* u, void* F, void* qc_out,
                         const void* c_base, int nonlin, int rosenbrock, int fmt,
                         double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = csr_blocks(op.n);
  EI_DISPATCH_FMT(fmt, (k_csr_F<F_><<<nb, EI_TPB, 0, stm>>>(op, u, F, qc_out, c_base, nonlin, rosenbrock, partials, ctl)));
  return cudaGetLastError();
}

cudaError_t launch_csr_gershgorin(const CsrDev& op, int prec, const void* val_user,
                                  const void* diag_user, double* lo, double* hi,
                                  double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = ew_blocks(op.n);
  if (prec == 0)
    k_csr_gershgorin<double><<<nb, EI_TPB, 0, stm>>>(op.n, op.rowptr, op.col,
        static_cast<const double*>(val_user), static_cast<const double*>(diag_user), lo, hi, partials, ctl);
  else
    k_csr_gershgorin<float><<<nb, EI_TPB, 0, stm>>>(op.n, op.rowptr, op.col,
        static_cast<const float*>(val_user), static_cast<const float*>(diag_user), lo, hi, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_stencil_gershgorin(const StencilDev& u, int prec, const double dx[3],
                                      const void* D, double Dc, const void* const b[3],
                                      const double bc[3], const void* c, double cc, double* lo,
                                      double* hi, double* partials, DevCtl* ctl,
                                      cudaStream_t stm) {
  const int64_t n = (int64_t)u.nx * u.ny * u.nz;
  const int nb = ew_blocks(n);
  if (prec == 0)
    k_stencil_gershgorin<double><<<nb, EI_TPB, 0, stm>>>(
        u.dim, u.nx, u.ny, u.nz, u.bc[0], u.bc[1], u.bc[2], u.bc[3], u.bc[4], u.bc[5], dx[0],
        dx[1], dx[2], D, Dc, b[0], b[1], b[2], bc[0], bc[1], bc[2], c, cc, lo, hi, partials, ctl);
  else
    k_stencil_gershgorin<float><<<nb, EI_TPB, 0, stm>>>(
        u.dim, u.nx, u.ny, u.nz, u.bc[0], u.bc[1], u.bc[2], u.bc[3], u.bc[4], u.bc[5], dx[0],
        dx[1], dx[2], D, Dc, b[0], b[1], b[2], bc[0], bc[1], bc[2], c, cc, lo, hi, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_shifted_minmax(int64_t n, const double* lo, const double* hi, const void* u,
                                  int prec, int nonlin, double* partials, DevCtl* ctl,
                                  cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (prec == 0)
    k_shifted_minmax<double><<<nb, EI_TPB, 0, stm>>>(n, lo, hi, static_cast<const double*>(u),
                                                      nonlin, partials, ctl);
  else
    k_shifted_minmax<float><<<nb, EI_TPB, 0, stm>>>(n, lo, hi, static_cast<const float*>(u),
                                                     nonlin, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_fill_coef(void* dst, int fmt, int64_t n, const void* src, int src_prec,
                             double cst, double scale, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (src_prec == 0) {
    EI_DISPATCH_FMT(fmt, (k_fill_coef<F_, double><<<nb, EI_TPB, 0, stm>>>(dst, n, static_cast<const double*>(src), cst, scale)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_fill_coef<F_, float><<<nb, EI_TPB, 0, stm>>>(dst, n, static_cast<const float*>(src), cst, scale)));
  }
  return cudaGetLastError();
}

cudaError_t launch_import(void* dst, int fmt, const void* src, int src_prec, int64_t n,
                          double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (src_prec == 0) {
    EI_DISPATCH_FMT(fmt, (k_import<F_, double><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const double*>(src), n, partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_import<F_, float><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const float*>(src), n, partials, ctl)));
  }
  return cudaGetLastError();
}

template <class U>
static void export_dispatch(U* dst, const void* src, int fmt, int src_is_p, int64_t n,
                            double scale, bool add, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  // element type of the source: df for the float-float format and for every
  // Newton sum except the double format's
  if (fmt == VF_F64) {
    const double* s = static_cast<const double*>(src);
    if (add) k_add_export<double, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
    else k_export<double, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
  } else if (fmt == VF_DF || src_is_p) {
    const df* s = static_cast<const df*>(src);
    if (add) k_add_export<df, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
    else k_export<df, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
  } else {
    const float* s = static_cast<const float*>(src);
    if (add) k_add_export<float, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
    else k_export<float, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, scale);
  }
}

cudaError_t launch_export(void* dst, int dst_prec, const void* src, int fmt, int src_is_p,
                          int64_t n, double scale, cudaStream_t stm) {
  if (dst_prec == 0)
    export_dispatch(static_cast<double*>(dst), src, fmt, src_is_p, n, scale, false, stm);
  else
    export_dispatch(static_cast<float*>(dst), src, fmt, src_is_p, n, scale, false, stm);
  return cudaGetLastError();
}

cudaError_t launch_add_export(void* u, int prec, const void* y, int fmt, int src_is_p, int64_t n,
                              double scale, cudaStream_t stm) {
  if (prec == 0)
    export_dispatch(static_cast<double*>(u), y, fmt, src_is_p, n, scale, true, stm);
  else
    export_dispatch(static_cast<float*>(u), y, fmt, src_is_p, n, scale, true, stm);
  return cudaGetLastError();
}

cudaError_t launch_p_to_vec(void* dst, const void* p, int fmt, int64_t n, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  EI_DISPATCH_FMT(fmt, (k_p_to_vec<F_><<<nb, EI_TPB, 0, stm>>>(dst, p, n)));
  return cudaGetLastError();
}

cudaError_t launch_axpy(void* y, const void* p, int fmt, int64_t n, double tau,
                        cudaStream_t stm) {
  const int nb = ew_blocks(n);
  EI_DISPATCH_FMT(fmt, (k_axpy<F_><<<nb, EI_TPB, 0, stm>>>(y, p, n, tau)));
  return cudaGetLastError();
}

cudaError_t launch_zero(void* x, int fmt, int64_t n, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  EI_DISPATCH_FMT(fmt, (k_zero<F_><<<nb, EI_TPB, 0, stm>>>(x, n)));
  return cudaGetLastError();
}

}  // namespace ei
