// CUDA kernels of the Leja exponential-integrator path other than the
// TMA-staged stencil Newton iteration (ei_newton_tma.cu): operator setup
// (coefficients, Gershgorin rows), the per-step F = A u + g(u) evaluation, the
// substep residual, the CSR Newton iteration, and the elementwise moves
// between the caller's contiguous vectors and the library's padded formats.
//
// A is a matrix-free stencil with the boundary conditions folded in (Sec.
// III-A of the paper) and position-dependent coefficients (Sec. III-B), or a
// CSR matrix (Sec. III-D).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "ei.h"
#include "ei_device.cuh"

namespace ei {

// logical point i (x fastest, contiguous) -> padded index
__device__ __forceinline__ int64_t pidx(int64_t i, int nx, int pitch) {
  const int64_t t = i / nx;  // z*ny + y
  return t * pitch + (i - t * nx);
}

// (x, y, z) and the row t = z*ny + y of logical point i; 32-bit division
// when the grid has fewer than 2^31 points (the usual case)
__device__ __forceinline__ void grid_coords(const StencilDev& g, int64_t n, int64_t i, int& x,
                                            int& y, int& z, int64_t& t) {
  if (n < ((int64_t)1 << 31)) {
    const unsigned ui = (unsigned)i, tt = ui / (unsigned)g.nx;
    x = (int)(ui - tt * (unsigned)g.nx);
    y = (int)(tt % (unsigned)g.ny);
    z = (int)(tt / (unsigned)g.ny);
    t = tt;
  } else {
    t = i / g.nx;
    x = (int)(i - t * g.nx);
    y = (int)(t % g.ny);
    z = (int)(t / g.ny);
  }
}

// Walk of the rows (y, z) of a grid by warps, grid-stride: a warp takes one
// row at a time and its lanes stride along x, so a point costs no division
// and the loads of a warp are contiguous.
#define EI_FOR_ROWS(nrows, row)                                                        \
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);    \
       row < (nrows); row += (int64_t)gridDim.x * (blockDim.x >> 5))
#define EI_FOR_X(nx, x) for (int x = (int)(threadIdx.x & 31); x < (nx); x += 32)
// f(i, j) for every logical point i (contiguous, x fastest) and its padded
// index j: a flat walk when there is no padding (pitch == nx, e.g. CSR
// vectors), the row walk otherwise.
template <class Fn>
__device__ __forceinline__ void for_points(int64_t n, int nx, int pitch, Fn f) {
  if (pitch == nx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      f(i, i);
  } else {
    EI_FOR_ROWS(n / nx, row) {
      EI_FOR_X(nx, x) f(row * nx + x, row * pitch + x);
    }
  }
}

// The same walk with K points per thread and pass, the K loads of a pass
// issued before any of its stores: a warp-wide load of one point per thread
// moves only 128-256 bytes, and with the grid capped at full occupancy a
// thread needs several loads in flight to cover HBM latency.  ld(i, j) loads
// what point i needs (a value or a small struct); body(i, j, v) uses it.  The
// padded index j of a logical point i is row * pitch + x.
template <int K, class Ld, class Body>
__device__ __forceinline__ void for_points_k(int64_t n, int nx, int pitch, Ld ld, Body body) {
  using V = decltype(ld(int64_t(0), int64_t(0)));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool flat = pitch == nx;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < n;
       base += K * stride) {
    V v[K];
    int64_t jj[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t i = base + k * stride;
      jj[k] = flat ? i : (i / nx) * pitch + i % nx;
      if (i < n) v[k] = ld(i, jj[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t i = base + k * stride;
      if (i < n) body(i, jj[k], v[k]);
    }
  }
}
constexpr int EW_K = 4;  // points per thread and pass of the element-wise kernels

// ---------------------------------------------------------------------------
// one row of the stencil operator in FP64 (shared by the Gershgorin bounds and
// the coefficient arrays): for each axis e and side s,
//   neighbour inside : a = D_face/dx_e^2 + s*b_e/(2 dx_e), diag -= D_face/dx_e^2
//   Dirichlet ghost  : a = 0, diag -= D_i/dx_e^2          (ghost u = 0, ghost D = D_i)
//   Neumann ghost    : a = 0, diag += s*b_e/(2 dx_e)      (ghost u = u_i: no flux)
// with D_face = (D_i + D_nb)/2, plus diag += c_i.
// ---------------------------------------------------------------------------
template <class U>
__device__ __forceinline__ double uval(const void* p, double cst, int64_t i) {
  return p ? (double)__ldg(static_cast<const U*>(p) + i) : cst;
}

struct UserCoef {
  int dim, nx, ny, nz;
  int bc[6];
  double dx[3];
  const void* D;
  double Dc;
  const void* b[3];
  double bc_[3];
  const void* c;
  double cc;
};

template <class U>
__device__ __forceinline__ void stencil_row(const UserCoef& u, int64_t i, int x, int y, int z,
                                            double a[6], double& diag, double& rad) {
  const int crd[3] = {x, y, z};
  const int ext[3] = {u.nx, u.ny, u.nz};
  const int64_t str[3] = {1, u.nx, (int64_t)u.nx * u.ny};
  const double Di = uval<U>(u.D, u.Dc, i);
  diag = uval<U>(u.c, u.cc, i);
  rad = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) a[k] = 0.0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (e >= u.dim) break;
    const double h2 = u.dx[e] * u.dx[e];
    const double be = uval<U>(u.b[e], u.bc_[e], i);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int sgn = side ? 1 : -1;
      const bool has = side ? crd[e] < ext[e] - 1 : crd[e] > 0;
      if (has) {
        const double Df = 0.5 * (Di + uval<U>(u.D, u.Dc, i + sgn * str[e]));
        a[2 * e + side] = Df / h2 + sgn * be / (2.0 * u.dx[e]);
        rad += fabs(a[2 * e + side]);
        diag -= Df / h2;
      } else if (u.bc[2 * e + side] == 1) {
        diag += sgn * be / (2.0 * u.dx[e]);
      } else {
        diag -= Di / h2;
      }
    }
  }
}

template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_gershgorin(UserCoef u, double* lo, double* hi, double* partials, DevCtl* ctl) {
  const int64_t n = (int64_t)u.nx * u.ny * u.nz;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % u.nx);
    const int y = (int)((i / u.nx) % u.ny);
    const int z = (int)(i / ((int64_t)u.nx * u.ny));
    double a[6], diag, rad;
    stencil_row<U>(u, i, x, y, z, a, diag, rad);
    lo[i] = diag - rad;
    hi[i] = diag + rad;
    minmax_row(mn, mx, diag - rad, diag + rad);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

template <int FMT, class U>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_coef(UserCoef u, int pitch, void* a0, void* a1, void* a2, void* a3, void* a4, void* a5,
               void* diag_out) {
  using T = typename VT<FMT>::T;
  T* out[6] = {static_cast<T*>(a0), static_cast<T*>(a1), static_cast<T*>(a2),
               static_cast<T*>(a3), static_cast<T*>(a4), static_cast<T*>(a5)};
  const int64_t n = (int64_t)u.nx * u.ny * u.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % u.nx);
    const int y = (int)((i / u.nx) % u.ny);
    const int z = (int)(i / ((int64_t)u.nx * u.ny));
    double a[6], diag, rad;
    stencil_row<U>(u, i, x, y, z, a, diag, rad);
    const int64_t j = pidx(i, u.nx, pitch);
#pragma unroll
    for (int k = 0; k < 6; ++k) st(out[k], j, from_d<T>(a[k]));
    st(static_cast<T*>(diag_out), j, from_d<T>(diag));
  }
}

// ---------------------------------------------------------------------------
// the stencil operator at one point, from global memory (padded arrays)
// ---------------------------------------------------------------------------
// explicit coefficients: (A w)_i = diag_i w_i + sum_nb a_nb,i w_nb
template <class T>
__device__ __forceinline__ T apply_coef7(const StencilDev& g, const T* __restrict__ w,
                                         const T* __restrict__ diag, int x, int y, int z,
                                         int64_t idx, T& wc) {
  const int64_t sy = g.pitch, sz = (int64_t)g.pitch * g.ny;
  wc = ldg(w, idx);
  T acc = mul(ldg(diag, idx), wc);
  if (x > 0) acc = mac(acc, ldg(static_cast<const T*>(g.a[0]), idx), ldg(w, idx - 1));
  if (x < g.nx - 1) acc = mac(acc, ldg(static_cast<const T*>(g.a[1]), idx), ldg(w, idx + 1));
  if (y > 0) acc = mac(acc, ldg(static_cast<const T*>(g.a[2]), idx), ldg(w, idx - sy));
  if (y < g.ny - 1) acc = mac(acc, ldg(static_cast<const T*>(g.a[3]), idx), ldg(w, idx + sy));
  if (z > 0) acc = mac(acc, ldg(static_cast<const T*>(g.a[4]), idx), ldg(w, idx - sz));
  if (z < g.nz - 1) acc = mac(acc, ldg(static_cast<const T*>(g.a[5]), idx), ldg(w, idx + sz));
  return acc;
}

// r = J y + v, ||r||^2 (J's diagonal: g.diag)
template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_stencil_residual(StencilDev g, const void* __restrict__ y_, const void* __restrict__ v_,
                   void* __restrict__ r_, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ yv = static_cast<const T*>(y_);
  const T* __restrict__ v = static_cast<const T*>(v_);
  T* __restrict__ r = static_cast<T*>(r_);
  const T* dg = static_cast<const T*>(g.diag);
  const int64_t n = (int64_t)g.nx * g.ny * g.nz;
  T ar = zero<T>();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    int64_t t;
    grid_coords(g, n, i, x, y, z, t);
    const int64_t idx = t * g.pitch + x;
    T yc;
    const T Ay = apply_coef7<T>(g, yv, dg, x, y, z, idx, yc);
    const T rv = add(Ay, ldg(v, idx));
    st(r, idx, rv);
    ar = mac(ar, rv, rv);
  }
  double a = to_d(ar), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) ctl->sum0 = a;
  }
}


// ---------------------------------------------------------------------------
// CSR operator (Sec. III-D): one thread per row.  The paper's C2075 code gave
// each row four threads; rows of the random geometric graph carry ~12
// entries, and on sm_103a one thread per row issues a row's column, value
// and gather loads in batches (eight, then four at a time; two independent
// accumulators) and keeps every lane busy in the Newton update.
// ---------------------------------------------------------------------------

// (W x)_row
template <class T>
__device__ __forceinline__ T csr_row(const CsrDev& op, const T* __restrict__ x, int64_t row) {
  const T* __restrict__ val = static_cast<const T*>(op.val);
  const int32_t* __restrict__ col = op.col;
  const int64_t b = __ldg(op.rowptr + row), e = __ldg(op.rowptr + row + 1);
  typename Acc<T>::type s1 = Acc<T>::zero(), s2 = Acc<T>::zero();
  int64_t k = b;
  // batches of 8 entries: all column and value loads of a batch, then all its
  // gathers, so a row of ~12 entries needs two dependent rounds
  for (; k + 8 <= e; k += 8) {
    int c[8];
    T v[8], xv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = __ldg(col + k + i);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = ldg(val, k + i);
#pragma unroll
    for (int i = 0; i < 8; ++i) xv[i] = ldg(x, c[i]);
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      s1 = lmac(s1, v[i], xv[i]);
      s2 = lmac(s2, v[i + 1], xv[i + 1]);
    }
  }
  for (; k + 4 <= e; k += 4) {
    const int c0 = __ldg(col + k), c1 = __ldg(col + k + 1);
    const int c2 = __ldg(col + k + 2), c3 = __ldg(col + k + 3);
    const T v0 = ldg(val, k), v1 = ldg(val, k + 1), v2 = ldg(val, k + 2), v3 = ldg(val, k + 3);
    const T x0 = ldg(x, c0), x1 = ldg(x, c1), x2 = ldg(x, c2), x3 = ldg(x, c3);
    s1 = lmac(s1, v0, x0);
    s2 = lmac(s2, v1, x1);
    s1 = lmac(s1, v2, x2);
    s2 = lmac(s2, v3, x3);
  }
  for (; k < e; ++k) s1 = lmac(s1, ldg(val, k), ldg(x, __ldg(col + k)));
  return lsum(s1, s2);
}

// Rows pipelined across a grid-stride walk: each thread keeps the row
// pointers of its next two rows in registers and the columns of its next row
// in its own shared-memory slots (cp.async, no registers held), so a row's
// value loads and gathers go out at once and the chain rowptr -> col -> x of
// a later row runs behind the current row's arithmetic.  A row's first
// CSR_PFC columns are prefetched; its entries are consumed in register batches
// of CSR_PF (value loads and gathers of a batch issued together); columns past
// CSR_PFC are read directly, four at a time.
template <class T>
__device__ __forceinline__ T csr_row_pf(const CsrDev& op, const T* __restrict__ x, int64_t b,
                                        int64_t e, const int32_t (*slot)[EI_TPB]) {
  const T* __restrict__ val = static_cast<const T*>(op.val);
  typename Acc<T>::type s1 = Acc<T>::zero(), s2 = Acc<T>::zero();
  const int m = (int)(e - b < CSR_PFC ? e - b : CSR_PFC);
  // prefetched columns, in batches of CSR_PF entries
  for (int q0 = 0; q0 < m; q0 += CSR_PF) {
    T v[CSR_PF], xv[CSR_PF];
#pragma unroll
    for (int q = 0; q < CSR_PF; ++q) {
      const bool in = q0 + q < m;
      v[q] = in ? ldg(val, b + q0 + q) : zero<T>();
      xv[q] = in ? ldg(x, slot[in ? q0 + q : 0][threadIdx.x]) : zero<T>();
    }
#pragma unroll
    for (int q = 0; q < CSR_PF; q += 2) {
      s1 = lmac(s1, v[q], xv[q]);
      s2 = lmac(s2, v[q + 1], xv[q + 1]);
    }
  }
  // the rest, four entries at a time
  for (int64_t k = b + CSR_PFC; k < e; k += 4) {
    int c[4];
    T v[4], xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = k + q < e ? __ldg(op.col + k + q) : -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = c[q] >= 0 ? ldg(val, k + q) : zero<T>();
      xv[q] = c[q] >= 0 ? ldg(x, c[q]) : zero<T>();
    }
    s1 = lmac(s1, v[0], xv[0]);
    s2 = lmac(s2, v[1], xv[1]);
    s1 = lmac(s1, v[2], xv[2]);
    s2 = lmac(s2, v[3], xv[3]);
  }
  return lsum(s1, s2);
}

template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_csr_newton(CsrDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
             void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  __shared__ int32_t slots[2][CSR_PFC][EI_TPB];
  if (*(volatile int*)&ctl->done != 0) return;
  const T* __restrict__ w_in = static_cast<const T*>(w_in_);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = op.n;
  int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;
  if (row < n) {
    b0 = __ldg(op.rowptr + row);
    e0 = __ldg(op.rowptr + row + 1);
  }
  if (row + G < n) {
    b1 = __ldg(op.rowptr + row + G);
    e1 = __ldg(op.rowptr + row + G + 1);
  }
  csr_prefetch_cols(slots[0], op.col, b0, e0);
  cp_async_commit();
  int buf = 0;
  for (; row < n; row += G) {
    int64_t b2 = 0, e2 = 0;
    if (row + 2 * G < n) {
      b2 = __ldg(op.rowptr + row + 2 * G);
      e2 = __ldg(op.rowptr + row + 2 * G + 1);
    }
    csr_prefetch_cols(slots[buf ^ 1], op.col, b1, e1);
    cp_async_commit();
    cp_async_wait<1>();  // this row's columns have landed
    const T wc = ldg(w_in, row);
    const T Aw = mac(csr_row_pf<T>(op, w_in, b0, e0, slots[buf]), ldg(qc, row), wc);
    const T wn = newton_update(Aw, invg, nshift, wc);
    const P pold = (s.j == 0) ? mul(d0, to_p(wc)) : ld(p, row);
    const P pn = mac(pold, dn, to_p(wn));
    st(w_out, row, wn);
    st(p, row, pn);
    aw = acc_sq(aw, wn);
    ap = acc_sq(ap, pn);
    b0 = b1;
    e0 = e1;
    b1 = b2;
    e1 = e2;
    buf ^= 1;
  }
  cp_async_wait<0>();
  double nw2 = acc_d(aw), np2 = acc_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      newton_verdict(ctl, s, s.j + 1, s.d_next, nw2, np2);
    }
  }
}

// The Newton step with G lanes per row (G = 2..32): the warp takes 32 rows
// in G rounds of 32/G rows, the lanes of a group reading consecutive entries
// of a row (whole sectors of the value and column arrays per warp load);
// after round t lane t of each group keeps its row's sum, so the update runs
// on all 32 lanes.  The 33 row pointers of the 32 rows come from one
// coalesced load and reach the rounds by shuffle.  A lane's entries go in
// predicated batches of U (all loads of a batch in flight together).  Five
// blocks of 256 per SM (48 registers) hold more rows in flight; the
// float-float variants of 4 or more lanes spill 8-12 bytes at that bound.
template <int FMT, int G, int U = (FMT == VF_F32 ? 8 : 4)>
__global__ void __launch_bounds__(EI_TPB, 5)
k_csr_newton_g(CsrDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
               void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  static_assert(U % 2 == 0, "batches accumulate entries in pairs");
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const T* __restrict__ w_in = static_cast<const T*>(w_in_);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T* __restrict__ val = static_cast<const T*>(op.val);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  constexpr int RPW = 32 / G;
  const int L = threadIdx.x & 31;
  const int lane = L & (G - 1);
  const int gsub = L / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = op.n;
  for (int64_t r0 = warp * 32; r0 < n; r0 += nwarp * 32) {
    const int64_t rl = r0 + L < n ? r0 + L : n;
    const int64_t rp_lo = __ldg(op.rowptr + rl);
    const int64_t rp_hi = __ldg(op.rowptr + (rl + 1 < n ? rl + 1 : n));
    T mine = zero<T>();
#pragma unroll 1
    for (int t = 0; t < G; ++t) {
      const int src = t * RPW + gsub;
      const int64_t b = __shfl_sync(0xffffffffu, rp_lo, src);
      const int64_t e = __shfl_sync(0xffffffffu, rp_hi, src);
      typename Acc<T>::type a1 = Acc<T>::zero(), a2 = Acc<T>::zero();
      int64_t k = b + lane;
      // U entries a lane per batch, loads issued together, predicated on the
      // row end; float-float and double skip the multiply-adds of empty slots
      for (; k < e; k += U * G) {
        int c[U];
        T v[U], xv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) c[q] = k + q * G < e ? __ldg(op.col + k + q * G) : -1;
#pragma unroll
        for (int q = 0; q < U; ++q) v[q] = c[q] >= 0 ? ldg(val, k + q * G) : zero<T>();
#pragma unroll
        for (int q = 0; q < U; ++q) xv[q] = c[q] >= 0 ? ldg(w_in, c[q]) : zero<T>();
#pragma unroll
        for (int q = 0; q + 1 < U; q += 2) {
          if (FMT == VF_F32 || c[q] >= 0) a1 = lmac(a1, v[q], xv[q]);
          if (FMT == VF_F32 || c[q + 1] >= 0) a2 = lmac(a2, v[q + 1], xv[q + 1]);
        }
      }
      T h = lsum(a1, a2);
#pragma unroll
      for (int m = G / 2; m > 0; m >>= 1) h = add(h, shfl_x(h, m));
      if (lane == t) mine = h;
    }
    const int64_t row = r0 + lane * RPW + gsub;  // the row whose sum this lane kept
    if (row < n) {
      const T wc = ldg(w_in, row);
      const T wn = newton_update(mac(mine, ldg(qc, row), wc), invg, nshift, wc);
      const P pold = (s.j == 0) ? mul(d0, to_p(wc)) : ld(p, row);
      const P pn = mac(pold, dn, to_p(wn));
      st(w_out, row, wn);
      st(p, row, pn);
      aw = acc_sq(aw, wn);
      ap = acc_sq(ap, pn);
    }
  }
  double nw2 = acc_d(aw), np2 = acc_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      newton_verdict(ctl, s, s.j + 1, s.d_next, nw2, np2);
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
  typename Acc<T>::type ar = Acc<T>::zero();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < op.n) {
    const T rv = add(mac(csr_row<T>(op, yv, row), ldg(qc, row), ldg(yv, row)), ldg(v, row));
    st(r, row, rv);
    ar = acc_sq(ar, rv);
  }
  double a = acc_d(ar), b = 0.0;
  if (last_block_reduce2<RED_SUM>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) ctl->sum0 = a;
  }
}

template <int FMT, bool COMB>
__global__ void __launch_bounds__(EI_TPB)
k_csr_F(CsrDev op, const void* __restrict__ u_, void* __restrict__ F_, void* __restrict__ qo_,
        const void* __restrict__ cb_, int nonlin, int rosenbrock, double* partials,
        DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  const T* __restrict__ u = static_cast<const T*>(u_);
  const T* __restrict__ cb = static_cast<const T*>(cb_);
  T* __restrict__ F = static_cast<T*>(F_);
  T* __restrict__ qo = static_cast<T*>(qo_);
  const T one = from_d<T>(1.0);
  typename Acc<T>::type af = Acc<T>::zero();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < op.n) {
    const T uc = ldg(u, row);
    T Fv = mac(csr_row<T>(op, u, row), ldg(cb, row), uc);
    T gq = zero<T>();
    if constexpr (COMB) {
      T gv;
      combustion_term(nonlin, uc, gv, gq);
      Fv = add(Fv, gv);
    } else if (nonlin == EI_NONLIN_LOGISTIC) {
      Fv = mac(Fv, uc, sub(one, uc));
      gq = mac(one, from_d<T>(-2.0), uc);
    }
    st(F, row, Fv);
    if (rosenbrock) st(qo, row, nonlin ? add(ldg(cb, row), gq) : ldg(cb, row));
    af = acc_sq(af, Fv);
  }
  double a = acc_d(af), b = 0.0;
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
    minmax_row(mn, mx, d - r, d + r);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

// g'(u) of the caller's u for the Rosenbrock interval: FP64 arrays in
// float-float (the FP64 pipes are slow), FP32 arrays in float
__device__ __forceinline__ double nonlin_slope(int nonlin, double u) {
  if (nonlin == EI_NONLIN_LOGISTIC) return 1.0 - 2.0 * u;
  if (nonlin == EI_NONLIN_NONE) return 0.0;
  df gv, dq;
  combustion_term(nonlin, df_from_double(u), gv, dq);
  return to_d(dq);
}
__device__ __forceinline__ double nonlin_slope(int nonlin, float u) {
  if (nonlin == EI_NONLIN_LOGISTIC) return 1.0 - 2.0 * (double)u;
  if (nonlin == EI_NONLIN_NONE) return 0.0;
  float gv, dq;
  combustion_term(nonlin, u, gv, dq);
  return (double)dq;
}

// min/max of (lo + q), (hi + q), q = g'(u).  The running min/max compare
// integer keys (order_key), which keeps the comparisons off the FP64 pipe;
// a NaN ends up in one of the two keys and makes the thread's interval
// (-inf, inf), as minmax_row does.
template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_shifted_minmax(int64_t n, const double* __restrict__ lo, const double* __restrict__ hi,
                 const U* __restrict__ u, int nonlin, double* partials, DevCtl* ctl) {
  long long kmn = order_key(INFINITY), kmx = order_key(-INFINITY);
  struct LHU {
    double lo, hi;
    U u;
  };
  for_points_k<EW_K>(
      n, (int)1, (int)1, [&](int64_t i, int64_t) { return LHU{lo[i], hi[i], u[i]}; },
      [&](int64_t, int64_t, LHU a) {
        const double q = nonlin_slope(nonlin, a.u);
        const long long kl = order_key(a.lo + q), kh = order_key(a.hi + q);
        kmn = kl < kmn ? kl : kmn;
        kmx = kh > kmx ? kh : kmx;
      });
  double mn = key_value(kmn), mx = key_value(kmx);
  if (isnan(mn) || isnan(mx)) {
    mn = -INFINITY;
    mx = INFINITY;
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}


// ---------------------------------------------------------------------------
// elementwise moves (caller's contiguous layout <-> padded vector formats)
// ---------------------------------------------------------------------------
template <int FMT, class U>
__global__ void k_fill_coef(void* dst_, int64_t n, int nx, int pitch, const U* src, double cst,
                            double scale) {
  using T = typename VT<FMT>::T;
  T* dst = static_cast<T*>(dst_);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (src ? (double)src[i] : cst) * scale;
    st(dst, pidx(i, nx, pitch), from_d<T>(v));
  }
}

template <int FMT, class U>
__global__ void __launch_bounds__(EI_TPB)
k_import(void* dst_, const U* __restrict__ src, int64_t n, int nx, int pitch, U* raw,
         double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  T* dst = static_cast<T*>(dst_);
  double a = 0.0;
  // max |x| from the IEEE bits with the sign cleared: for non-negative values
  // the integer order is the value order, and it keeps the FP64 pipe free
  unsigned long long mbits = 0ull;
  auto mag = [](U x) -> unsigned long long {
    if constexpr (sizeof(U) == 8)
      return (unsigned long long)__double_as_longlong((double)x) & 0x7fffffffffffffffull;
    else
      return (unsigned long long)(__float_as_uint((float)x) & 0x7fffffffu);
  };
  auto ld = [&](int64_t i, int64_t) { return src[i]; };
  if constexpr (FMT == VF_DF) {
    // the split and the squared norm on the FP32 pipes (the FP64 pipe is slow)
    dfacc acc{0.0f, 0.0f};
    for_points_k<EW_K>(n, nx, pitch, ld, [&](int64_t i, int64_t j, U x) {
      if (raw) raw[i] = x;
      mbits = max(mbits, mag(x));
      const df v = df_split_double((double)x);
      st(dst, j, v);
      acc = dfa_mac(acc, v, v);
    });
    a = acc_d(acc);
  } else {
    for_points_k<EW_K>(n, nx, pitch, ld, [&](int64_t i, int64_t j, U x) {
      if (raw) raw[i] = x;
      mbits = max(mbits, mag(x));
      const double v = (double)x;
      st(dst, j, from_d<T>(v));
      a = fma(v, v, a);
    });
  }
  double b;
  if constexpr (sizeof(U) == 8) b = __longlong_as_double((long long)mbits);
  else b = (double)__uint_as_float((unsigned)mbits);
  if (last_block_reduce2<RED_SUMMAX>(a, b, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->sum0 = a;
      ctl->sum1 = finite_d(a) ? 1.0 : 0.0;
      ctl->vmax = b;
    }
  }
}

template <class S, class U>
__global__ void k_export(U* dst, const S* __restrict__ src, int64_t n, int nx, int pitch,
                         double scale) {
  for_points_k<EW_K>(
      n, nx, pitch, [&](int64_t, int64_t j) { return ldg(src, j); },
      [&](int64_t i, int64_t, S y) { dst[i] = (U)(to_d(y) * scale); });
}

// out = u + scale * y (out may be u, or a mapped host buffer)
template <class S, class U>
struct AddExportLd {
  S y;
  U u;
};
template <class S, class U>
__global__ void k_add_export(U* out, const U* u, const S* __restrict__ y, int64_t n, int nx,
                             int pitch, double scale) {
  for_points_k<EW_K>(
      n, nx, pitch, [&](int64_t i, int64_t j) { return AddExportLd<S, U>{ldg(y, j), u[i]}; },
      [&](int64_t i, int64_t, AddExportLd<S, U> v) {
        out[i] = (U)fma(to_d(v.y), scale, (double)v.u);
      });
}

template <int FMT>
__global__ void k_p_to_vec(void* dst_, const void* p_, int64_t n) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  T* dst = static_cast<T*>(dst_);
  const P* p = static_cast<const P*>(p_);
  for_points_k<EW_K>(
      n, (int)1, (int)1, [&](int64_t i, int64_t) { return ldg(p, i); },
      [&](int64_t i, int64_t, P v) {
        if constexpr (FMT == VF_F32) {
          st(dst, i, (float)to_d(v));
        } else {
          st(dst, i, v);
        }
      });
}

// y += tau * p  (y in vector format, p in the Newton-sum format)
template <int FMT>
__global__ void k_axpy(void* y_, const void* p_, int64_t n, double tau) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  T* y = static_cast<T*>(y_);
  const P* p = static_cast<const P*>(p_);
  const P t = from_d<P>(tau);
  struct YP {
    T y;
    P p;
  };
  for_points_k<EW_K>(
      n, (int)1, (int)1, [&](int64_t i, int64_t) { return YP{ld(y, i), ldg(p, i)}; },
      [&](int64_t i, int64_t, YP a) {
        const P v = mac(to_p(a.y), t, a.p);
        if constexpr (FMT == VF_F32) {
          st(y, i, (float)to_d(v));
        } else {
          st(y, i, v);
        }
      });
}

// (A - cI)/gamma as seven native FP64 coefficient arrays.  The padding stays
// harmless: padded neighbour coefficients are 0 and stay 0; the padded
// diagonal becomes -c/gamma but multiplies a padded w = 0.
struct PrescaleArgs {
  void* s[7];
  const void* a[7];  // a[0..5], diagonal
};
template <class T>
struct Coef7T {
  T a[7];
};
// the scaled operator, in the vector format T (double or float-float)
template <class T>
__global__ void __launch_bounds__(EI_TPB)
k_prescale(const PrescaleArgs P, int64_t n, double c, double inv_gamma) {
  const T g = from_d<T>(inv_gamma), cc = from_d<T>(c);
  for_points_k<EW_K>(
      n, (int)1, (int)1,
      [&](int64_t i, int64_t) {
        Coef7T<T> v;
#pragma unroll
        for (int k = 0; k < 7; ++k) v.a[k] = ldg(static_cast<const T*>(P.a[k]), i);
        return v;
      },
      [&](int64_t i, int64_t, Coef7T<T> v) {
#pragma unroll
        for (int k = 0; k < 6; ++k) st(static_cast<T*>(P.s[k]), i, mul(v.a[k], g));
        st(static_cast<T*>(P.s[6]), i, mul(sub(v.a[6], cc), g));
      });
}

template <class T>
__global__ void __launch_bounds__(EI_TPB)
k_prescale_diag(T* __restrict__ sa6, const T* __restrict__ diag, int64_t n, double c,
                double inv_gamma) {
  const T g = from_d<T>(inv_gamma), cc = from_d<T>(c);
  for_points_k<EW_K>(
      n, (int)1, (int)1, [&](int64_t i, int64_t) { return ldg(diag, i); },
      [&](int64_t i, int64_t, T v) { st(sa6, i, mul(sub(v, cc), g)); });
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

int reduction_capacity() { return num_sms() * 8; }
int sm_count() { return num_sms(); }

int csr_blocks(int64_t n) {  // one thread per row
  int64_t b = (n + EI_TPB - 1) / EI_TPB;
  return b < 1 ? 1 : (int)b;
}

#define EI_DISPATCH_FMT(fmt, KERNEL_CALL)                           \
  switch (fmt) {                                                    \
    case VF_DF: { constexpr int F_ = VF_DF; KERNEL_CALL; } break;   \
    case VF_F64: { constexpr int F_ = VF_F64; KERNEL_CALL; } break; \
    default: { constexpr int F_ = VF_F32; KERNEL_CALL; } break;     \
  }

static UserCoef user_coef(const StencilDev& g, const double dx[3], const void* D, double Dc,
                          const void* const b[3], const double bc[3], const void* c, double cc) {
  UserCoef u;
  u.dim = g.dim;
  u.nx = g.nx;
  u.ny = g.ny;
  u.nz = g.nz;
  for (int f = 0; f < 6; ++f) u.bc[f] = g.bc[f];
  for (int e = 0; e < 3; ++e) {
    u.dx[e] = dx[e];
    u.b[e] = b[e];
    u.bc_[e] = bc[e];
  }
  u.D = D;
  u.Dc = Dc;
  u.c = c;
  u.cc = cc;
  return u;
}

cudaError_t launch_stencil_gershgorin(const StencilDev& g, int prec, const double dx[3],
                                      const void* D, double Dc, const void* const b[3],
                                      const double bc[3], const void* c, double cc, double* lo,
                                      double* hi, double* partials, DevCtl* ctl,
                                      cudaStream_t stm) {
  const UserCoef u = user_coef(g, dx, D, Dc, b, bc, c, cc);
  const int nb = ew_blocks((int64_t)g.nx * g.ny * g.nz);
  if (prec == 0)
    k_stencil_gershgorin<double><<<nb, EI_TPB, 0, stm>>>(u, lo, hi, partials, ctl);
  else
    k_stencil_gershgorin<float><<<nb, EI_TPB, 0, stm>>>(u, lo, hi, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_stencil_coef(const StencilDev& g, int prec, const double dx[3], const void* D,
                                double Dc, const void* const b[3], const double bc[3],
                                const void* c, double cc, void* const a[6], void* diag, int fmt,
                                cudaStream_t stm) {
  const UserCoef u = user_coef(g, dx, D, Dc, b, bc, c, cc);
  const int nb = ew_blocks((int64_t)g.nx * g.ny * g.nz);
  if (prec == 0) {
    EI_DISPATCH_FMT(fmt, (k_stencil_coef<F_, double><<<nb, EI_TPB, 0, stm>>>(u, g.pitch, a[0], a[1], a[2], a[3], a[4], a[5], diag)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_stencil_coef<F_, float><<<nb, EI_TPB, 0, stm>>>(u, g.pitch, a[0], a[1], a[2], a[3], a[4], a[5], diag)));
  }
  return cudaGetLastError();
}

cudaError_t launch_stencil_residual(const StencilDev& g, const void* y, const void* v, void* r,
                                    int fmt, double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = ew_blocks((int64_t)g.nx * g.ny * g.nz);
  EI_DISPATCH_FMT(fmt, (k_stencil_residual<F_><<<nb, EI_TPB, 0, stm>>>(g, y, v, r, partials, ctl)));
  return cudaGetLastError();
}


// Face term of face f (2 ax + side): at each boundary row next to the face,
// (D_i/dx^2 + sgn b_i/(2 dx)) x the prescribed ghost value (the ghost D is D_i),
// in FP64 from the caller's arrays (contiguous, x fastest) or constants.
// Face layout: faces 0/1 [z][y], 2/3 [z][x], 4/5 [y][x].
template <class U>
__global__ void __launch_bounds__(EI_TPB)
k_face_term(StencilDev g, int face, double h, const U* D, double Dc, const U* b, double bc,
            const U* vals, double* out) {
  const int ax = face / 2;
  const double sgn = (face & 1) ? 1.0 : -1.0;
  const int64_t m0 = ax == 0 ? g.ny : g.nx;           // fastest index of the face
  const int64_t m1 = ax == 2 ? g.ny : g.nz;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m0 * m1;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a0 = j % m0, a1 = j / m0;
    int64_t x, y, z;
    if (ax == 0) { x = (face & 1) ? g.nx - 1 : 0; y = a0; z = a1; }
    else if (ax == 1) { x = a0; y = (face & 1) ? g.ny - 1 : 0; z = a1; }
    else { x = a0; y = a1; z = (face & 1) ? g.nz - 1 : 0; }
    const int64_t i = (z * g.ny + y) * g.nx + x;
    const double Di = D ? (double)D[i] : Dc;
    const double bi = b ? (double)b[i] : bc;
    out[j] = (Di / (h * h) + sgn * bi / (2.0 * h)) * (double)vals[j];
  }
}

cudaError_t launch_face_term(const StencilDev& g, int face, int prec, const double dx[3],
                             const void* D, double D_const, const void* b_axis,
                             double b_const, const void* vals, double* out, cudaStream_t stm) {
  const int ax = face / 2;
  const int64_t m = (ax == 0 ? (int64_t)g.ny * g.nz : ax == 1 ? (int64_t)g.nx * g.nz
                                                               : (int64_t)g.nx * g.ny);
  const int nb = ew_blocks(m);
  if (prec == EI_PREC_F32)
    k_face_term<float><<<nb, EI_TPB, 0, stm>>>(g, face, dx[ax], static_cast<const float*>(D),
                                                D_const, static_cast<const float*>(b_axis),
                                                b_const, static_cast<const float*>(vals), out);
  else
    k_face_term<double><<<nb, EI_TPB, 0, stm>>>(g, face, dx[ax], static_cast<const double*>(D),
                                                 D_const, static_cast<const double*>(b_axis),
                                                 b_const, static_cast<const double*>(vals), out);
  return cudaGetLastError();
}
// One Newton iteration on the sliced form: a warp per slice (grid-stride over
// slices), a lane per row.  The slice's length is the same for all its lanes,
// so the entry loop has no divergence; U entries a lane go out per batch, the
// column and value loads of a batch together, then the gathers of w_in.  The
// row's own w, diagonal and p are loaded before the entries.
constexpr int kSellMinB = 4;  // resident blocks per SM the register budget targets
template <int FMT, int U>
__global__ void __launch_bounds__(EI_TPB, kSellMinB)
k_csr_newton_sell(SellDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
                  void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const T* __restrict__ w_in = static_cast<const T*>(w_in_);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T* __restrict__ val = static_cast<const T*>(op.val);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  const int L = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = warp; sl < op.nslices; sl += nwarp) {
    const int row = __ldg(op.perm + sl * 32 + L);
    const int myl = __ldg(op.rlen + sl * 32 + L);
    const int64_t b = __ldg(op.sptr + sl);
    const int len = (int)((__ldg(op.sptr + sl + 1) - b) >> 5);
    T wc = zero<T>(), q = zero<T>();
    P pold = zero<P>();
    if (row >= 0) {
      wc = ldg(w_in, row);
      q = ldg(qc, row);
      if (s.j > 0) pold = ld(p, row);
    }
    typename Acc<T>::type a1 = Acc<T>::zero(), a2 = Acc<T>::zero();
    const int32_t* __restrict__ cp = op.col + b + L;
    const T* __restrict__ vp = val + b + L;
    for (int k = 0; k < len; k += U) {
      int c[U];
      T v[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = k + u < myl;  // this lane's row only: the padding is never read
        c[u] = in ? __ldg(cp + (int64_t)(k + u) * 32) : -1;
        v[u] = in ? ldg(vp, (int64_t)(k + u) * 32) : zero<T>();
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? ldg(w_in, c[u]) : zero<T>();
      if constexpr (FMT == VF_F64) {
        // native FP64: the FP64 pipe bounds this kernel and an issued
        // multiply-add costs the same whether its lanes are active or not, so
        // the slots past the slice's length (a warp-uniform count) are skipped
        // by a branch, not predicated (padding inside the length has value 0)
        static_assert(U == 6, "the fall-through below covers batches of 6");
        switch (len - k < U ? len - k : U) {
          case 6: a2 = lmac(a2, v[5], xv[5]); [[fallthrough]];
          case 5: a1 = lmac(a1, v[4], xv[4]); [[fallthrough]];
          case 4: a2 = lmac(a2, v[3], xv[3]); [[fallthrough]];
          case 3: a1 = lmac(a1, v[2], xv[2]); [[fallthrough]];
          case 2: a2 = lmac(a2, v[1], xv[1]); [[fallthrough]];
          default: a1 = lmac(a1, v[0], xv[0]);
        }
      } else {
#pragma unroll
        for (int u = 0; u + 1 < U; u += 2) {
          if (FMT == VF_F32 || c[u] >= 0) a1 = lmac(a1, v[u], xv[u]);
          if (FMT == VF_F32 || c[u + 1] >= 0) a2 = lmac(a2, v[u + 1], xv[u + 1]);
        }
      }
    }
    if (row >= 0) {
      const T mine = lsum(a1, a2);
      const T wn = newton_update(mac(mine, q, wc), invg, nshift, wc);
      if (s.j == 0) pold = mul(d0, to_p(wc));
      const P pn = mac(pold, dn, to_p(wn));
      st(w_out, row, wn);
      st(p, row, pn);
      aw = acc_sq(aw, wn);
      ap = acc_sq(ap, pn);
    }
  }
  double nw2 = acc_d(aw), np2 = acc_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      newton_verdict(ctl, s, s.j + 1, s.d_next, nw2, np2);
    }
  }
}

template <class U, int FMT>
__global__ void k_sell_gather(int64_t e, const int64_t* __restrict__ src,
                              const int32_t* __restrict__ col, int32_t* col_out,
                              const U* __restrict__ val, void* val_out_) {
  using T = typename VT<FMT>::T;
  T* val_out = static_cast<T*>(val_out_);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = src[i];
    if (col_out) col_out[i] = k >= 0 ? col[k] : -1;
    if (val_out) st(val_out, i, k >= 0 ? from_d<T>((double)val[k]) : zero<T>());
  }
}

template <int FMT, int U>
static int csr_sell_grid(int64_t nslices) {
  static const int per = [] {
    int b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_csr_newton_sell<FMT, U>, EI_TPB, 0);
    return b < 1 ? 1 : (b > 8 ? 8 : b);  // the partials hold 8 blocks per SM
  }();
  int64_t nb = (nslices + EI_TPB / 32 - 1) / (EI_TPB / 32);
  if (nb > (int64_t)num_sms() * per) nb = (int64_t)num_sms() * per;
  return nb < 1 ? 1 : (int)nb;
}

template <int FMT, int G>
static int csr_g_grid(int64_t n) {
  // resident blocks per SM, once per variant (capped at 8: the partials' capacity)
  static const int per = [] {
    int b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_csr_newton_g<FMT, G>, EI_TPB, 0);
    return b < 1 ? 1 : (b > 8 ? 8 : b);
  }();
  int64_t nb = (n + EI_TPB - 1) / EI_TPB;  // 32 rows a warp and pass
  if (nb > (int64_t)num_sms() * per) nb = (int64_t)num_sms() * per;
  return nb < 1 ? 1 : (int)nb;
}

template <int FMT>
static void csr_newton_g_fmt(int G, const CsrDev& op, const void* w_in, void* w_out, void* p,
                             const NewtonScalars& s, double* partials, DevCtl* ctl,
                             cudaStream_t stm) {
  switch (G) {
    case 2: k_csr_newton_g<FMT, 2><<<csr_g_grid<FMT, 2>(op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl); break;
    case 4: k_csr_newton_g<FMT, 4><<<csr_g_grid<FMT, 4>(op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl); break;
    case 8: k_csr_newton_g<FMT, 8><<<csr_g_grid<FMT, 8>(op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl); break;
    case 16: k_csr_newton_g<FMT, 16><<<csr_g_grid<FMT, 16>(op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl); break;
    default: k_csr_newton_g<FMT, 32><<<csr_g_grid<FMT, 32>(op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl); break;
  }
}

int csr_lanes_for(int64_t n, int64_t nnz, int lanes) {
  if (lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32)
    return lanes;
  const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
  return mean < 8.0 ? 1 : mean < 64.0 ? 2 : mean < 128.0 ? 4 : 8;
}

cudaError_t launch_csr_newton(const CsrDev& op, int64_t nnz, int lanes, const void* w_in,
                              void* w_out, void* p, const NewtonScalars& s, int fmt,
                              double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int G = csr_lanes_for(op.n, nnz, lanes);
  if (G > 1) {
    EI_DISPATCH_FMT(fmt, (csr_newton_g_fmt<F_>(G, op, w_in, w_out, p, s, partials, ctl, stm)));
    return cudaGetLastError();
  }
  // one thread a row: a grid of resident blocks walking the rows (at most csr_blocks(n))
  static int per_sm[3] = {0, 0, 0};
  if (!per_sm[fmt]) {
    int per = 1;
    EI_DISPATCH_FMT(fmt, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_csr_newton<F_>,
                                                                       EI_TPB, 0));
    per_sm[fmt] = per < 1 ? 1 : per;
  }
  int nb = csr_blocks(op.n);
  if (nb > num_sms() * per_sm[fmt]) nb = num_sms() * per_sm[fmt];
  EI_DISPATCH_FMT(fmt, (k_csr_newton<F_><<<nb, EI_TPB, 0, stm>>>(op, w_in, w_out, p, s, partials, ctl)));
  return cudaGetLastError();
}

// batch sizes of the sliced kernel: entries a lane per batch
constexpr int kSellU64 = 6, kSellU32 = 8;
cudaError_t launch_csr_newton_sell(const SellDev& op, const void* w_in, void* w_out, void* p,
                                   const NewtonScalars& s, int fmt, double* partials,
                                   DevCtl* ctl, cudaStream_t stm) {
  if (fmt == VF_DF)
    k_csr_newton_sell<VF_DF, kSellU64><<<csr_sell_grid<VF_DF, kSellU64>(op.nslices), EI_TPB, 0,
                                         stm>>>(op, w_in, w_out, p, s, partials, ctl);
  else if (fmt == VF_F64)
    k_csr_newton_sell<VF_F64, kSellU64><<<csr_sell_grid<VF_F64, kSellU64>(op.nslices), EI_TPB,
                                          0, stm>>>(op, w_in, w_out, p, s, partials, ctl);
  else
    k_csr_newton_sell<VF_F32, kSellU32><<<csr_sell_grid<VF_F32, kSellU32>(op.nslices), EI_TPB,
                                          0, stm>>>(op, w_in, w_out, p, s, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_sell_gather(int64_t e, const int64_t* src, const int32_t* col,
                               int32_t* col_out, const void* val, int val_prec, void* val_out,
                               int fmt, cudaStream_t stm) {
  const int nb = ew_blocks(e);
  if (val_prec == EI_PREC_F32) {
    EI_DISPATCH_FMT(fmt, (k_sell_gather<float, F_><<<nb, EI_TPB, 0, stm>>>(
                             e, src, col, col_out, static_cast<const float*>(val), val_out)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_sell_gather<double, F_><<<nb, EI_TPB, 0, stm>>>(
                             e, src, col, col_out, static_cast<const double*>(val), val_out)));
  }
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
  if (nonlin >= EI_NONLIN_COMBUSTION) {
    EI_DISPATCH_FMT(fmt, (k_csr_F<F_, true><<<nb, EI_TPB, 0, stm>>>(op, u, F, qc_out, c_base, nonlin, rosenbrock, partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_csr_F<F_, false><<<nb, EI_TPB, 0, stm>>>(op, u, F, qc_out, c_base, nonlin, rosenbrock, partials, ctl)));
  }
  return cudaGetLastError();
}

// Pointwise g(u) and g'(u) (Sec. III-C; Table 3 times this evaluation): U is
// the array type, T the format the arithmetic runs in.
// Below this u the combustion term's exponential e^{20(1-1/u)} < 2^-100 leaves
// the float-float range (FP32 exponents): those points use native FP64.
constexpr double kDfCombustionU = 0.25;
template <class T, class U>
__global__ void __launch_bounds__(EI_TPB)
k_nonlin_eval(int nonlin, int64_t n, const U* u, U* g, U* dg) {
  const T one = from_d<T>(1.0), mtwo = from_d<T>(-2.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 8 && sizeof(U) == 8 && !std::is_same<T, double>::value) {
      // float-float: where e^{20(1-1/u)} falls below the format's range
      // (2^-100, u < 1/4) the full form is evaluated in native FP64
      const double ud = (double)u[i];
      if (nonlin == EI_NONLIN_COMBUSTION && ud < kDfCombustionU) {
        double gd, dd;
        combustion_eval(ud, gd, dd);
        g[i] = (U)gd;
        if (dg) dg[i] = (U)dd;
        continue;
      }
    }
    const T uc = from_d<T>((double)u[i]);
    T gv = zero<T>(), dq = zero<T>();
    if (nonlin == EI_NONLIN_LOGISTIC) {
      gv = mul(uc, sub(one, uc));
      dq = mac(one, mtwo, uc);
    } else if (nonlin != EI_NONLIN_NONE) {
      combustion_term(nonlin, uc, gv, dq);
    }
    g[i] = (U)to_d(gv);
    if (dg) dg[i] = (U)to_d(dq);
  }
}

cudaError_t launch_nonlinearity(int nonlin, int prec, int arith, int64_t n, const void* u,
                                void* g, void* dg, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (prec == EI_PREC_F32)
    k_nonlin_eval<float, float><<<nb, EI_TPB, 0, stm>>>(nonlin, n, static_cast<const float*>(u),
                                                        static_cast<float*>(g),
                                                        static_cast<float*>(dg));
  else if (arith == EI_ARITH_NATIVE_F64)
    k_nonlin_eval<double, double><<<nb, EI_TPB, 0, stm>>>(nonlin, n,
                                                          static_cast<const double*>(u),
                                                          static_cast<double*>(g),
                                                          static_cast<double*>(dg));
  else
    k_nonlin_eval<df, double><<<nb, EI_TPB, 0, stm>>>(nonlin, n, static_cast<const double*>(u),
                                                      static_cast<double*>(g),
                                                      static_cast<double*>(dg));
  return cudaGetLastError();
}

__global__ void k_csr_validate(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, DevCtl* ctl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    const int64_t a = __ldg(rowptr + i);
    bad |= (i == 0 && a != 0) || (i == n && a != nnz) || (i < n && __ldg(rowptr + i + 1) < a);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = __ldg(col + e);
    bad |= c < 0 || (int64_t)c >= n;
  }
  if (bad) atomicOr(&ctl->csr_bad, 1);
}

cudaError_t launch_csr_validate(int64_t n, int64_t nnz, const int64_t* rowptr,
                                const int32_t* col, DevCtl* ctl, cudaStream_t stm) {
  k_csr_validate<<<ew_blocks(n + 1 > nnz ? n + 1 : nnz), EI_TPB, 0, stm>>>(n, nnz, rowptr, col,
                                                                           ctl);
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

// Coefficient statistics (see launch_coef_stats).  Per block: the sum in a
// fixed order and the two maxima; the last block combines the blocks in
// block order.
template <class U>
__global__ void __launch_bounds__(EI_TPB)
    k_coef_stats(int64_t n, int csr, int dim, const void* D, double Dc, const void* b0,
                 const void* b1, const void* b2, double bc0, double bc1, double bc2, double dx0,
                 double dx1, double dx2, double* partials, DevCtl* ctl) {
  double sum = 0.0, mx = 0.0, pe = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double Di = uval<U>(D, Dc, i);
    if (csr) Di = fabs(Di);
    sum += Di;
    mx = fmax(mx, Di);
    if (!csr) {
      pe = fmax(pe, fabs(uval<U>(b0, bc0, i)) * dx0 / (2.0 * Di));
      if (dim > 1) pe = fmax(pe, fabs(uval<U>(b1, bc1, i)) * dx1 / (2.0 * Di));
      if (dim > 2) pe = fmax(pe, fabs(uval<U>(b2, bc2, i)) * dx2 / (2.0 * Di));
    }
  }
  double zero = 0.0, npe = -pe;
  block_reduce2<RED_SUM>(sum, zero);
  block_reduce2<RED_MINMAX>(npe, mx);
  __shared__ bool am_last;
  const unsigned nblk = gridDim.x;
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x] = sum;
    partials[4 * blockIdx.x + 1] = mx;
    partials[4 * blockIdx.x + 2] = -npe;
    __threadfence();
    am_last = (atomicAdd(&ctl->count, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!am_last || threadIdx.x != 0) return;
  __threadfence();
  double s = 0.0, m = 0.0, p = 0.0;
  for (unsigned k = 0; k < nblk; ++k) {
    s += __ldcg(partials + 4 * k);
    m = fmax(m, __ldcg(partials + 4 * k + 1));
    p = fmax(p, __ldcg(partials + 4 * k + 2));
  }
  ctl->cs_sum = s;
  ctl->cs_max = m;
  ctl->cs_pe = p;
  ctl->count = 0;
}

cudaError_t launch_coef_stats(int64_t n, int csr, int prec, int dim, const void* D, double Dc,
                              const void* const b[3], const double bcst[3], const double dx[3],
                              double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (prec == 0)
    k_coef_stats<double><<<nb, EI_TPB, 0, stm>>>(n, csr, dim, D, Dc, b[0], b[1], b[2], bcst[0],
                                                  bcst[1], bcst[2], dx[0], dx[1], dx[2],
                                                  partials, ctl);
  else
    k_coef_stats<float><<<nb, EI_TPB, 0, stm>>>(n, csr, dim, D, Dc, b[0], b[1], b[2], bcst[0],
                                                 bcst[1], bcst[2], dx[0], dx[1], dx[2],
                                                 partials, ctl);
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


cudaError_t launch_fill_coef(void* dst, int fmt, int64_t n, int nx, int ny, int pitch,
                             const void* src, int src_prec, double cst, double scale,
                             cudaStream_t stm) {
  (void)ny;
  const int nb = ew_blocks(n);
  if (src_prec == 0) {
    EI_DISPATCH_FMT(fmt, (k_fill_coef<F_, double><<<nb, EI_TPB, 0, stm>>>(dst, n, nx, pitch, static_cast<const double*>(src), cst, scale)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_fill_coef<F_, float><<<nb, EI_TPB, 0, stm>>>(dst, n, nx, pitch, static_cast<const float*>(src), cst, scale)));
  }
  return cudaGetLastError();
}

cudaError_t launch_import(void* dst, int fmt, const void* src, int src_prec, int64_t n, int nx,
                          int ny, int pitch, double* partials, DevCtl* ctl, cudaStream_t stm,
                          void* raw) {
  (void)ny;
  const int nb = ew_blocks(n);
  if (src_prec == 0) {
    EI_DISPATCH_FMT(fmt, (k_import<F_, double><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const double*>(src), n, nx, pitch, static_cast<double*>(raw), partials, ctl)));
  } else {
    EI_DISPATCH_FMT(fmt, (k_import<F_, float><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const float*>(src), n, nx, pitch, static_cast<float*>(raw), partials, ctl)));
  }
  return cudaGetLastError();
}

template <class U>
static void export_dispatch(U* dst, const void* src, int fmt, int src_is_p, int64_t n, int nx,
                            int pitch, double scale, bool add, cudaStream_t stm,
                            U* add_out = nullptr) {
  U* out = add_out ? add_out : dst;
  const int nb = ew_blocks(n);
  // source element type: df for the float-float format and for the Newton
  // sum of every format but the double one
  if (fmt == VF_F64) {
    const double* s = static_cast<const double*>(src);
    if (add) k_add_export<double, U><<<nb, EI_TPB, 0, stm>>>(out, dst, s, n, nx, pitch, scale);
    else k_export<double, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, nx, pitch, scale);
  } else if (fmt == VF_DF || src_is_p) {
    const df* s = static_cast<const df*>(src);
    if (add) k_add_export<df, U><<<nb, EI_TPB, 0, stm>>>(out, dst, s, n, nx, pitch, scale);
    else k_export<df, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, nx, pitch, scale);
  } else {
    const float* s = static_cast<const float*>(src);
    if (add) k_add_export<float, U><<<nb, EI_TPB, 0, stm>>>(out, dst, s, n, nx, pitch, scale);
    else k_export<float, U><<<nb, EI_TPB, 0, stm>>>(dst, s, n, nx, pitch, scale);
  }
}

cudaError_t launch_export(void* dst, int dst_prec, const void* src, int fmt, int src_is_p,
                          int64_t n, int nx, int ny, int pitch, double scale, cudaStream_t stm) {
  (void)ny;
  if (dst_prec == 0)
    export_dispatch(static_cast<double*>(dst), src, fmt, src_is_p, n, nx, pitch, scale, false, stm);
  else
    export_dispatch(static_cast<float*>(dst), src, fmt, src_is_p, n, nx, pitch, scale, false, stm);
  return cudaGetLastError();
}

cudaError_t launch_add_export(void* u, int prec, const void* y, int fmt, int src_is_p, int64_t n,
                              int nx, int ny, int pitch, double scale, cudaStream_t stm,
                              void* out) {
  (void)ny;
  if (prec == 0)
    export_dispatch(static_cast<double*>(u), y, fmt, src_is_p, n, nx, pitch, scale, true, stm,
                    static_cast<double*>(out));
  else
    export_dispatch(static_cast<float*>(u), y, fmt, src_is_p, n, nx, pitch, scale, true, stm,
                    static_cast<float*>(out));
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

cudaError_t launch_prescale(void* const sa[7], const void* const a[6], const void* diag,
                            int64_t n_alloc, double c, double inv_gamma, int fmt,
                            cudaStream_t stm) {
  PrescaleArgs P{};
  for (int i = 0; i < 7; ++i) P.s[i] = sa[i];
  for (int i = 0; i < 6; ++i) P.a[i] = a[i];
  P.a[6] = diag;
  if (fmt == VF_DF)
    k_prescale<df><<<ew_blocks(n_alloc), EI_TPB, 0, stm>>>(P, n_alloc, c, inv_gamma);
  else
    k_prescale<double><<<ew_blocks(n_alloc), EI_TPB, 0, stm>>>(P, n_alloc, c, inv_gamma);
  return cudaGetLastError();
}

cudaError_t launch_prescale_diag(void* sa6, const void* diag, int64_t n_alloc, double c,
                                 double inv_gamma, int fmt, cudaStream_t stm) {
  if (fmt == VF_DF)
    k_prescale_diag<df><<<ew_blocks(n_alloc), EI_TPB, 0, stm>>>(
        static_cast<df*>(sa6), static_cast<const df*>(diag), n_alloc, c, inv_gamma);
  else
    k_prescale_diag<double><<<ew_blocks(n_alloc), EI_TPB, 0, stm>>>(
        static_cast<double*>(sa6), static_cast<const double*>(diag), n_alloc, c, inv_gamma);
  return cudaGetLastError();
}

template <class P>
__global__ void __launch_bounds__(EI_TPB)
k_p_sqnorm(const P* __restrict__ x, int64_t n, double* partials, DevCtl* ctl) {
  typename Acc<P>::type a = Acc<P>::zero();
  for_points_k<EW_K>(
      n, (int)1, (int)1, [&](int64_t i, int64_t) { return ldg(x, i); },
      [&](int64_t, int64_t, P v) { a = acc_sq(a, v); });
  double s0 = acc_d(a), s1 = 0.0;
  if (last_block_reduce2<RED_SUM>(s0, s1, partials, ctl)) {
    if (threadIdx.x == 0) ctl->sum0 = s0;
  }
}

cudaError_t launch_p_sqnorm(const void* x, int fmt, int64_t n, double* partials, DevCtl* ctl,
                            cudaStream_t stm) {
  const int nb = ew_blocks(n);
  if (fmt == VF_F64)
    k_p_sqnorm<double><<<nb, EI_TPB, 0, stm>>>(static_cast<const double*>(x), n, partials, ctl);
  else
    k_p_sqnorm<df><<<nb, EI_TPB, 0, stm>>>(static_cast<const df*>(x), n, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* x, int fmt, int64_t n, cudaStream_t stm) {
  const int nb = ew_blocks(n);
  EI_DISPATCH_FMT(fmt, (k_zero<F_><<<nb, EI_TPB, 0, stm>>>(x, n)));
  return cudaGetLastError();
}

}  // namespace ei

// ===========================================================================
// Spectral interval without device allocation
// ===========================================================================
// Some callers may not allocate device memory at all: real-time loops and
// device-memory budgets in which every byte is reserved up front (a
// cudaMalloc there can fail, or stall while the driver synchronises the
// device), and hosts whose framework owns all of the GPU's memory through its
// own pool allocator (memory from cudaMalloc is invisible to that pool and can
// push it past its limit).  ei_estimate_spectrum_stencil_noalloc serves them:
// it computes the Gershgorin interval of a stencil operator straight from the
// caller's coefficient arrays, with its reduction scratch (the arrival counter
// and one pair of doubles per block) in the fixed array below instead of
// memory from cudaMalloc.  The array exists once per GPU that loads the
// library and stays there until the process exits.
namespace ei {

static constexpr int kNoallocChunk = 8192;       // grid points per block (256 threads x 32)
static constexpr int kNoallocMaxBlocks = 16384;  // so at most 2^27 = 512^3 points
static constexpr int kNoallocMaxDevices = 64;
static constexpr size_t kNoallocBytes = 256 + sizeof(double) * 2 * kNoallocMaxBlocks;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];
// the control block occupies the first 256 bytes, the block partials follow
static_assert(sizeof(DevCtl) <= 256, "DevCtl must fit the scratch header");

// The Gershgorin row kernel with a fixed chunk of points per block; the
// control block sits at the start of the scratch, the block partials after it.
template <class U>
__global__ void __launch_bounds__(EI_TPB) k_stencil_gershgorin_chunk(UserCoef u, unsigned char* scratch) {
  DevCtl* ctl = reinterpret_cast<DevCtl*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + 256);
  const int64_t n = (int64_t)u.nx * u.ny * u.nz;
  const int64_t i0 = (int64_t)blockIdx.x * kNoallocChunk;
  const int64_t i1 = i0 + kNoallocChunk < n ? i0 + kNoallocChunk : n;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int x = (int)(i % u.nx);
    const int y = (int)((i / u.nx) % u.ny);
    const int z = (int)(i / ((int64_t)u.nx * u.ny));
    double a[6], diag, rad;
    stencil_row<U>(u, i, x, y, z, a, diag, rad);
    minmax_row(mn, mx, diag - rad, diag + rad);
  }
  if (last_block_reduce2<RED_MINMAX>(mn, mx, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->mn = mn;
      ctl->mx = mx;
    }
  }
}

// Device address of the scratch array, looked up once per device (with that
// device current, by the first call on it) and cached for the life of the
// process.  The cache is not invalidated: after cudaDeviceReset the address
// may no longer be valid, so a process that resets a device must not call the
// entry point on that device again.
static void* noalloc_scratch(int device, cudaError_t* err) {
  static std::mutex mu;
  static void* addr[kNoallocMaxDevices] = {nullptr};
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = p;
  }
  *err = cudaSuccess;
  return addr[device];
}

}  // namespace ei

extern "C" ei_status ei_estimate_spectrum_stencil_noalloc(
    int device, void* cuda_stream, int dim, const int64_t n[3], const double dx[3], const void* D,
    double D_const, const void* const b[3], const double b_const[3], const void* c,
    double c_const, const int bc[6], int prec, double* alpha, double* beta) {
  using namespace ei;
  if (!n || !dx || !bc || !alpha || !beta || (dim != 2 && dim != 3) ||
      (prec != EI_PREC_F64 && prec != EI_PREC_F32) || device < 0 || device >= kNoallocMaxDevices)
    return EI_ERR_INVALID_ARG;
  const int64_t ext[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  for (int e = 0; e < 3; ++e)
    if (ext[e] < 1 || ext[e] > ((int64_t)1 << 30)) return EI_ERR_INVALID_ARG;
  for (int e = 0; e < dim; ++e)
    if (!(dx[e] > 0) || !isfinite(dx[e])) return EI_ERR_INVALID_ARG;
  for (int f = 0; f < 2 * dim; ++f)
    if (bc[f] != EI_BC_DIRICHLET0 && bc[f] != EI_BC_NEUMANN0) return EI_ERR_INVALID_ARG;
  const int64_t npts = ext[0] * ext[1] * ext[2];
  if ((double)ext[0] * ext[1] * ext[2] > (double)kNoallocMaxBlocks * kNoallocChunk)
    return EI_ERR_INVALID_ARG;  // more points than the fixed scratch can reduce
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return EI_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return EI_ERR_CUDA;
  }
  ei_status rc = EI_OK;
  cudaError_t e = cudaSuccess;
  unsigned char* scratch = static_cast<unsigned char*>(noalloc_scratch(device, &e));
  if (!scratch) {
    rc = EI_ERR_CUDA;
  } else {
    UserCoef u;
    u.dim = dim;
    u.nx = (int)ext[0];
    u.ny = (int)ext[1];
    u.nz = (int)ext[2];
    for (int f = 0; f < 6; ++f) u.bc[f] = (f < 2 * dim) ? bc[f] : EI_BC_NEUMANN0;
    for (int k = 0; k < 3; ++k) {
      u.dx[k] = k < dim ? dx[k] : 1.0;
      u.b[k] = (b && k < dim) ? b[k] : nullptr;
      u.bc_[k] = (b_const && k < dim) ? b_const[k] : 0.0;
    }
    u.D = D;
    u.Dc = D_const;
    u.c = c;
    u.cc = c_const;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = (int)((npts + kNoallocChunk - 1) / kNoallocChunk);
    double out[2] = {0.0, 0.0};
    // the arrival counter must start at zero; the rest is written before it is read
    e = cudaMemsetAsync(scratch, 0, sizeof(DevCtl), st);
    if (e == cudaSuccess) {
      if (prec == EI_PREC_F64)
        k_stencil_gershgorin_chunk<double><<<blocks, EI_TPB, 0, st>>>(u, scratch);
      else
        k_stencil_gershgorin_chunk<float><<<blocks, EI_TPB, 0, st>>>(u, scratch);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, scratch + offsetof(DevCtl, mn), sizeof(out),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = EI_ERR_CUDA;
    } else if (!isfinite(out[0]) || !isfinite(out[1])) {
      rc = EI_ERR_NONFINITE;
    } else {
      *alpha = out[0];
      *beta = out[1];
    }
  }
  cudaSetDevice(prev);
  return rc;
}
