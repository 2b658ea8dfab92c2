// Complex Newton iteration for phi_k(-i h H) v with H real symmetric: the
// products (alpha A + beta I) x of Eq. (3) with K = C (Sec. II-C), on the CSR
// operator of Sec. III-D (the spin-system problem psi' = -i H psi).
//
// The Newton basis of H on its real interval is the real recurrence
//     w_{j+1} = (H w_j) / gamma - (c/gamma + xi_j) w_j,
// complex only through v, and the divided differences d_j of
// f(xi) = phi_k(-i tau (c + gamma xi)) are complex, so one step updates
//     p_{j+1} = p_j + d_{j+1} w_{j+1}
// with a complex product.  Vectors are interleaved (re, im): one gather of
// x[col] brings both parts of a neighbour (16 bytes for the float-float and
// double formats, 8 for float), and the column and value loads of a row
// serve both parts.
#include "ei_device.cuh"

namespace ei {

template <class T> struct Cx {
  T re, im;
};

__device__ __forceinline__ Cx<df> ldgc(const Cx<df>* p, int64_t i) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
  return Cx<df>{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ Cx<double> ldgc(const Cx<double>* p, int64_t i) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
  return Cx<double>{v.x, v.y};
}
__device__ __forceinline__ Cx<float> ldgc(const Cx<float>* p, int64_t i) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
  return Cx<float>{v.x, v.y};
}
// the Newton sum is read and written by the same kernel: plain loads
__device__ __forceinline__ Cx<df> ldc(const Cx<df>* p, int64_t i) {
  const float4 v = reinterpret_cast<const float4*>(p)[i];
  return Cx<df>{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ Cx<double> ldc(const Cx<double>* p, int64_t i) {
  const double2 v = reinterpret_cast<const double2*>(p)[i];
  return Cx<double>{v.x, v.y};
}
__device__ __forceinline__ void stc(Cx<df>* p, int64_t i, Cx<df> v) {
  reinterpret_cast<float4*>(p)[i] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
}
__device__ __forceinline__ void stc(Cx<double>* p, int64_t i, Cx<double> v) {
  reinterpret_cast<double2*>(p)[i] = make_double2(v.re, v.im);
}
__device__ __forceinline__ void stc(Cx<float>* p, int64_t i, Cx<float> v) {
  reinterpret_cast<float2*>(p)[i] = make_float2(v.re, v.im);
}

// (H x)_row for complex x over entries [b, e): the first CSR_PFC columns
// from this thread's prefetch slots, in batches of CPF, the rest four at a
// time.  Two accumulators per part.
constexpr int CPF = 10;
template <class T>
__device__ __forceinline__ Cx<T> csr_row_c(const CsrDev& op, const Cx<T>* __restrict__ x,
                                           int64_t b, int64_t e,
                                           const int32_t (*slot)[EI_TPB]) {
  const T* __restrict__ val = static_cast<const T*>(op.val);
  typename Acc<T>::type r1 = Acc<T>::zero(), r2 = Acc<T>::zero();
  typename Acc<T>::type i1 = Acc<T>::zero(), i2 = Acc<T>::zero();
  const int m = (int)(e - b < CSR_PFC ? e - b : CSR_PFC);
  for (int q0 = 0; q0 < m; q0 += CPF) {
    T v[CPF];
    Cx<T> xv[CPF];
#pragma unroll
    for (int q = 0; q < CPF; ++q) {
      const bool in = q0 + q < m;
      v[q] = in ? ldg(val, b + q0 + q) : zero<T>();
      xv[q] = in ? ldgc(x, slot[in ? q0 + q : 0][threadIdx.x]) : Cx<T>{zero<T>(), zero<T>()};
    }
#pragma unroll
    for (int q = 0; q < CPF; q += 2) {
      r1 = lmac(r1, v[q], xv[q].re);
      i1 = lmac(i1, v[q], xv[q].im);
      r2 = lmac(r2, v[q + 1], xv[q + 1].re);
      i2 = lmac(i2, v[q + 1], xv[q + 1].im);
    }
  }
  for (int64_t k = b + CSR_PFC; k < e; k += 4) {
    int c[4];
    T v[4];
    Cx<T> xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = k + q < e ? __ldg(op.col + k + q) : -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = c[q] >= 0 ? ldg(val, k + q) : zero<T>();
      xv[q] = c[q] >= 0 ? ldgc(x, c[q]) : Cx<T>{zero<T>(), zero<T>()};
    }
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      r1 = lmac(r1, v[q], xv[q].re);
      i1 = lmac(i1, v[q], xv[q].im);
      r2 = lmac(r2, v[q + 1], xv[q + 1].re);
      i2 = lmac(i2, v[q + 1], xv[q + 1].im);
    }
  }
  return Cx<T>{lsum(r1, r2), lsum(i1, i2)};
}

// One Newton step on complex w, the rows walked as in k_csr_newton (grid of
// resident blocks, the next rows' pointers in registers, their first columns
// in shared memory).  qc is the operator's diagonal (real).
template <int FMT>
__global__ void __launch_bounds__(EI_TPB)
k_csr_newton_c(CsrDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
               void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  __shared__ int32_t slots[2][CSR_PFC][EI_TPB];
  if (*(volatile int*)&ctl->done != 0) return;
  const Cx<T>* __restrict__ w_in = static_cast<const Cx<T>*>(w_in_);
  Cx<T>* __restrict__ w_out = static_cast<Cx<T>*>(w_out_);
  Cx<P>* __restrict__ p = static_cast<Cx<P>*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dnr = from_d<P>(s.d_next), dni = from_d<P>(s.d_next_im);
  const P ndni = from_d<P>(-s.d_next_im);
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
    cp_async_wait<1>();
    const Cx<T> wc = ldgc(w_in, row);
    const Cx<T> hx = csr_row_c<T>(op, w_in, b0, e0, slots[buf]);
    const T q = ldg(qc, row);
    Cx<T> wn;
    wn.re = newton_update(mac(hx.re, q, wc.re), invg, nshift, wc.re);
    wn.im = newton_update(mac(hx.im, q, wc.im), invg, nshift, wc.im);
    Cx<P> pold;
    if (s.j == 0) {  // p_0 = d_0 w_0
      const P d0r = from_d<P>(s.d0), d0i = from_d<P>(s.d0_im), nd0i = from_d<P>(-s.d0_im);
      const P xr = to_p(wc.re), xi = to_p(wc.im);
      pold.re = mac(mul(d0r, xr), nd0i, xi);
      pold.im = mac(mul(d0r, xi), d0i, xr);
    } else {
      pold = ldc(p, row);
    }
    const P nr = to_p(wn.re), ni = to_p(wn.im);
    Cx<P> pn;
    pn.re = mac(mac(pold.re, dnr, nr), ndni, ni);
    pn.im = mac(mac(pold.im, dnr, ni), dni, nr);
    stc(w_out, row, wn);
    stc(p, row, pn);
    aw = acc_sq(acc_sq(aw, wn.re), wn.im);
    ap = acc_sq(acc_sq(ap, pn.re), pn.im);
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
      newton_verdict(ctl, s, s.j + 1, hypot(s.d_next, s.d_next_im), nw2, np2);
    }
  }
}

// The same step with G lanes per row (G = 2..32, a power of two), for long
// rows: the lanes of a group read consecutive entries of the row, so a
// warp's column and value loads cover whole sectors instead of one entry per
// 32-byte sector and row, and the row sum is finished by a butterfly over
// the group.  A warp takes 32 rows at a time in G rounds of 32/G rows; after
// round t lane t of each group keeps its row's sum, so that every lane ends
// with one of the 32 rows and the Newton update (the heavier part for the
// float-float format) runs on all lanes at once.  The warp walks its rows
// together (a warp-uniform loop bound), so the shuffles see all 32 lanes.

template <int FMT, int G, int U = (FMT == VF_F32 ? 8 : 4)>
__global__ void __launch_bounds__(EI_TPB)
k_csr_newton_cg(CsrDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
                void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  static_assert(U % 2 == 0, "batches accumulate entries in pairs");
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const Cx<T>* __restrict__ w_in = static_cast<const Cx<T>*>(w_in_);
  Cx<T>* __restrict__ w_out = static_cast<Cx<T>*>(w_out_);
  Cx<P>* __restrict__ p = static_cast<Cx<P>*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T* __restrict__ val = static_cast<const T*>(op.val);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dnr = from_d<P>(s.d_next), dni = from_d<P>(s.d_next_im);
  const P ndni = from_d<P>(-s.d_next_im);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  constexpr int RPW = 32 / G;  // rows of a round
  const int lane = threadIdx.x & (G - 1);
  const int gsub = (threadIdx.x & 31) / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = op.n;
  for (int64_t r0 = warp * 32; r0 < n; r0 += nwarp * 32) {
    // the 33 row pointers of this block of 32 rows, one coalesced load;
    // round t reads its row's pair by shuffle (no dependent load per round)
    const int L = threadIdx.x & 31;
    const int64_t rl = r0 + L < n ? r0 + L : n;
    const int64_t rp_lo = __ldg(op.rowptr + rl);
    const int64_t rp_hi = __ldg(op.rowptr + (rl + 1 < n ? rl + 1 : n));
    T myr = zero<T>(), myi = zero<T>();
#pragma unroll 1
    for (int t = 0; t < G; ++t) {
      const int src = t * RPW + gsub;
      const int64_t b = __shfl_sync(0xffffffffu, rp_lo, src);
      const int64_t e = __shfl_sync(0xffffffffu, rp_hi, src);
      typename Acc<T>::type r1 = Acc<T>::zero(), r2 = Acc<T>::zero();
      typename Acc<T>::type i1 = Acc<T>::zero(), i2 = Acc<T>::zero();
      int64_t k = b + lane;
      // U entries a lane per batch, loads issued together, predicated on the
      // row end; float-float and double skip the multiply-adds of empty slots
      for (; k < e; k += U * G) {
        int c[U];
        T v[U];
        Cx<T> xv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) c[q] = k + q * G < e ? __ldg(op.col + k + q * G) : -1;
#pragma unroll
        for (int q = 0; q < U; ++q) v[q] = c[q] >= 0 ? ldg(val, k + q * G) : zero<T>();
#pragma unroll
        for (int q = 0; q < U; ++q)
          xv[q] = c[q] >= 0 ? ldgc(w_in, c[q]) : Cx<T>{zero<T>(), zero<T>()};
#pragma unroll
        for (int q = 0; q + 1 < U; q += 2) {
          if (FMT == VF_F32 || c[q] >= 0) {
            r1 = lmac(r1, v[q], xv[q].re);
            i1 = lmac(i1, v[q], xv[q].im);
          }
          if (FMT == VF_F32 || c[q + 1] >= 0) {
            r2 = lmac(r2, v[q + 1], xv[q + 1].re);
            i2 = lmac(i2, v[q + 1], xv[q + 1].im);
          }
        }
      }
      T hr = lsum(r1, r2), hi = lsum(i1, i2);
#pragma unroll
      for (int m = G / 2; m > 0; m >>= 1) {
        hr = add(hr, shfl_x(hr, m));
        hi = add(hi, shfl_x(hi, m));
      }
      if (lane == t) {
        myr = hr;
        myi = hi;
      }
    }
    const int64_t row = r0 + lane * RPW + gsub;  // the row whose sum this lane kept
    if (row < n) {
      const Cx<T> wc = ldgc(w_in, row);
      const T q = ldg(qc, row);
      Cx<T> wn;
      wn.re = newton_update(mac(myr, q, wc.re), invg, nshift, wc.re);
      wn.im = newton_update(mac(myi, q, wc.im), invg, nshift, wc.im);
      Cx<P> pold;
      if (s.j == 0) {
        const P d0r = from_d<P>(s.d0), d0i = from_d<P>(s.d0_im), nd0i = from_d<P>(-s.d0_im);
        const P xr = to_p(wc.re), xi = to_p(wc.im);
        pold.re = mac(mul(d0r, xr), nd0i, xi);
        pold.im = mac(mul(d0r, xi), d0i, xr);
      } else {
        pold = ldc(p, row);
      }
      const P nr = to_p(wn.re), ni = to_p(wn.im);
      Cx<P> pn;
      pn.re = mac(mac(pold.re, dnr, nr), ndni, ni);
      pn.im = mac(mac(pold.im, dnr, ni), dni, nr);
      stc(w_out, row, wn);
      stc(p, row, pn);
      aw = acc_sq(acc_sq(aw, wn.re), wn.im);
      ap = acc_sq(acc_sq(ap, pn.re), pn.im);
    }
  }
  double nw2 = acc_d(aw), np2 = acc_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      newton_verdict(ctl, s, s.j + 1, hypot(s.d_next, s.d_next_im), nw2, np2);
    }
  }
}

// dst = (sr + i si) src for interleaved complex arrays (U the user's part type)
template <class S, class U>
__global__ void __launch_bounds__(EI_TPB)
k_cexport(U* __restrict__ dst, const Cx<S>* __restrict__ src, int64_t n, double sr, double si) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Cx<S> x = ldgc(src, i);
    const double a = to_d(x.re), b = to_d(x.im);
    dst[2 * i] = (U)(sr * a - si * b);
    dst[2 * i + 1] = (U)(sr * b + si * a);
  }
}


// resident blocks per SM of a kernel variant, from the occupancy calculator
// once per variant (capped at 8, the reduction partials' capacity per SM)
template <class K>
static int blocks_per_sm(K kernel) {
  int per = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, EI_TPB, 0);
  return per < 1 ? 1 : (per > 8 ? 8 : per);
}

// a grid of resident blocks walking the rows: at most one block per 256 rows
static int grid_of(int per_sm, int64_t n) {
  int64_t nb = (n + EI_TPB - 1) / EI_TPB;
  if (nb > (int64_t)sm_count() * per_sm) nb = (int64_t)sm_count() * per_sm;
  return nb < 1 ? 1 : (int)nb;
}

template <int FMT, int G>
static void launch_cg(const CsrDev& op, const void* w_in, void* w_out, void* p,
                      const NewtonScalars& s, double* partials, DevCtl* ctl, cudaStream_t stm) {
  static const int per = blocks_per_sm(k_csr_newton_cg<FMT, G>);
  k_csr_newton_cg<FMT, G><<<grid_of(per, op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s,
                                                                 partials, ctl);
}

template <int FMT>
static cudaError_t csr_newton_c_fmt(const CsrDev& op, int lanes, const void* w_in, void* w_out,
                                    void* p, const NewtonScalars& s, double* partials,
                                    DevCtl* ctl, cudaStream_t stm) {
  switch (lanes) {
    case 1: {
      static const int per = blocks_per_sm(k_csr_newton_c<FMT>);
      k_csr_newton_c<FMT><<<grid_of(per, op.n), EI_TPB, 0, stm>>>(op, w_in, w_out, p, s,
                                                                  partials, ctl);
      break;
    }
    case 2: launch_cg<FMT, 2>(op, w_in, w_out, p, s, partials, ctl, stm); break;
    case 4: launch_cg<FMT, 4>(op, w_in, w_out, p, s, partials, ctl, stm); break;
    case 8: launch_cg<FMT, 8>(op, w_in, w_out, p, s, partials, ctl, stm); break;
    case 16: launch_cg<FMT, 16>(op, w_in, w_out, p, s, partials, ctl, stm); break;
    default: launch_cg<FMT, 32>(op, w_in, w_out, p, s, partials, ctl, stm); break;
  }
  return cudaGetLastError();
}

// The complex step on the sliced form (SellDev): a warp a slice of 32 rows, a
// lane a row, the column and value loads of entry k one coalesced access.  On
// operators whose rows share a structure (the spin-bath Hamiltonian: column q
// of row i is i XOR mask_q) the gathers of a slice's entry k fall in one
// aligned block of 32 rows: whole lines.
// (a register cap for four blocks a SM measured slower: 263.7 against 255.8
// us float-float, 155.5 against 145.4 FP32, on the 21-spin bath)
template <int FMT, int U = (FMT == VF_F32 ? 8 : 4)>
__global__ void __launch_bounds__(EI_TPB)
k_csr_newton_sell_c(SellDev op, const void* __restrict__ w_in_, void* __restrict__ w_out_,
                    void* __restrict__ p_, NewtonScalars s, double* partials, DevCtl* ctl) {
  static_assert(U % 2 == 0, "batches accumulate entries in pairs");
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile int*)&ctl->done != 0) return;
  const Cx<T>* __restrict__ w_in = static_cast<const Cx<T>*>(w_in_);
  Cx<T>* __restrict__ w_out = static_cast<Cx<T>*>(w_out_);
  Cx<P>* __restrict__ p = static_cast<Cx<P>*>(p_);
  const T* __restrict__ qc = static_cast<const T*>(op.qc);
  const T* __restrict__ val = static_cast<const T*>(op.val);
  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(-s.shift);
  const P dnr = from_d<P>(s.d_next), dni = from_d<P>(s.d_next_im);
  const P ndni = from_d<P>(-s.d_next_im);
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
    Cx<T> wc{zero<T>(), zero<T>()};
    T q = zero<T>();
    Cx<P> pold{zero<P>(), zero<P>()};
    if (row >= 0) {
      wc = ldgc(w_in, row);
      q = ldg(qc, row);
      if (s.j > 0) pold = ldc(p, row);
    }
    typename Acc<T>::type r1 = Acc<T>::zero(), r2 = Acc<T>::zero();
    typename Acc<T>::type i1 = Acc<T>::zero(), i2 = Acc<T>::zero();
    const int32_t* __restrict__ cp = op.col + b + L;
    const T* __restrict__ vp = val + b + L;
    for (int k = 0; k < len; k += U) {
      int c[U];
      T v[U];
      Cx<T> xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = k + u < myl;
        c[u] = in ? __ldg(cp + (int64_t)(k + u) * 32) : -1;
        v[u] = in ? ldg(vp, (int64_t)(k + u) * 32) : zero<T>();
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        xv[u] = c[u] >= 0 ? ldgc(w_in, c[u]) : Cx<T>{zero<T>(), zero<T>()};
#pragma unroll
      for (int u = 0; u + 1 < U; u += 2) {
        if (FMT == VF_F32 || c[u] >= 0) {
          r1 = lmac(r1, v[u], xv[u].re);
          i1 = lmac(i1, v[u], xv[u].im);
        }
        if (FMT == VF_F32 || c[u + 1] >= 0) {
          r2 = lmac(r2, v[u + 1], xv[u + 1].re);
          i2 = lmac(i2, v[u + 1], xv[u + 1].im);
        }
      }
    }
    if (row >= 0) {
      const T myr = lsum(r1, r2), myi = lsum(i1, i2);
      Cx<T> wn;
      wn.re = newton_update(mac(myr, q, wc.re), invg, nshift, wc.re);
      wn.im = newton_update(mac(myi, q, wc.im), invg, nshift, wc.im);
      if (s.j == 0) {
        const P d0r = from_d<P>(s.d0), d0i = from_d<P>(s.d0_im), nd0i = from_d<P>(-s.d0_im);
        const P xr = to_p(wc.re), xi = to_p(wc.im);
        pold.re = mac(mul(d0r, xr), nd0i, xi);
        pold.im = mac(mul(d0r, xi), d0i, xr);
      }
      const P nr = to_p(wn.re), ni = to_p(wn.im);
      Cx<P> pn;
      pn.re = mac(mac(pold.re, dnr, nr), ndni, ni);
      pn.im = mac(mac(pold.im, dnr, ni), dni, nr);
      stc(w_out, row, wn);
      stc(p, row, pn);
      aw = acc_sq(acc_sq(aw, wn.re), wn.im);
      ap = acc_sq(acc_sq(ap, pn.re), pn.im);
    }
  }
  double nw2 = acc_d(aw), np2 = acc_d(ap);
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (threadIdx.x == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      newton_verdict(ctl, s, s.j + 1, hypot(s.d_next, s.d_next_im), nw2, np2);
    }
  }
}

template <int FMT>
static int csr_sell_c_grid(int64_t nslices) {
  static const int per = [] {
    int b = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_csr_newton_sell_c<FMT>, EI_TPB, 0);
    return b < 1 ? 1 : (b > 8 ? 8 : b);  // the partials hold 8 blocks per SM
  }();
  int64_t nb = (nslices + EI_TPB / 32 - 1) / (EI_TPB / 32);
  if (nb > (int64_t)sm_count() * per) nb = (int64_t)sm_count() * per;
  return nb < 1 ? 1 : (int)nb;
}

cudaError_t launch_csr_newton_sell_c(const SellDev& op, const void* w_in, void* w_out, void* p,
                                     const NewtonScalars& s, int fmt, double* partials,
                                     DevCtl* ctl, cudaStream_t stm) {
  if (fmt == VF_DF)
    k_csr_newton_sell_c<VF_DF><<<csr_sell_c_grid<VF_DF>(op.nslices), EI_TPB, 0, stm>>>(
        op, w_in, w_out, p, s, partials, ctl);
  else if (fmt == VF_F64)
    k_csr_newton_sell_c<VF_F64><<<csr_sell_c_grid<VF_F64>(op.nslices), EI_TPB, 0, stm>>>(
        op, w_in, w_out, p, s, partials, ctl);
  else
    k_csr_newton_sell_c<VF_F32><<<csr_sell_c_grid<VF_F32>(op.nslices), EI_TPB, 0, stm>>>(
        op, w_in, w_out, p, s, partials, ctl);
  return cudaGetLastError();
}

cudaError_t launch_csr_newton_c(const CsrDev& op, int64_t nnz, int lanes, const void* w_in,
                                void* w_out, void* p, const NewtonScalars& s, int fmt,
                                double* partials, DevCtl* ctl, cudaStream_t stm) {
  const int g = csr_lanes_for(op.n, nnz, lanes);
  switch (fmt) {
    case VF_DF: return csr_newton_c_fmt<VF_DF>(op, g, w_in, w_out, p, s, partials, ctl, stm);
    case VF_F64: return csr_newton_c_fmt<VF_F64>(op, g, w_in, w_out, p, s, partials, ctl, stm);
    default: return csr_newton_c_fmt<VF_F32>(op, g, w_in, w_out, p, s, partials, ctl, stm);
  }
}

template <class U>
static void cexport_u(U* dst, const void* src, int fmt, int src_is_p, int64_t n, double sr,
                      double si, int nb, cudaStream_t stm) {
  if (fmt == VF_F64)
    k_cexport<double, U><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const Cx<double>*>(src), n, sr, si);
  else if (fmt == VF_DF || src_is_p)
    k_cexport<df, U><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const Cx<df>*>(src), n, sr, si);
  else
    k_cexport<float, U><<<nb, EI_TPB, 0, stm>>>(dst, static_cast<const Cx<float>*>(src), n, sr, si);
}

cudaError_t launch_cexport(void* dst, int prec, const void* src, int fmt, int src_is_p,
                           int64_t n, double sr, double si, cudaStream_t stm) {
  int64_t nb = (n + EI_TPB - 1) / EI_TPB;
  if (nb > (int64_t)sm_count() * 8) nb = (int64_t)sm_count() * 8;
  if (nb < 1) nb = 1;
  if (prec == EI_PREC_F32)
    cexport_u(static_cast<float*>(dst), src, fmt, src_is_p, n, sr, si, (int)nb, stm);
  else
    cexport_u(static_cast<double*>(dst), src, fmt, src_is_p, n, sr, si, (int)nb, stm);
  return cudaGetLastError();
}

}  // namespace ei
