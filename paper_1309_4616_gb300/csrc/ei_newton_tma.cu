// The fused Newton iteration of the stencil path, staged through shared
// memory by TMA (sm_103a).
//
// One iteration is one product of Eq. (3) of the paper, (alpha*A + beta*I)w
// with alpha = 1/gamma and beta = -(c/gamma + xi_j), fused with the Newton sum
// p += d_{j+1} w_{j+1}, the squared norms of w_{j+1} and p (block partials and
// a fixed-order last-block reduction) and the stop test of the a-posteriori
// estimate |d_{j+1}| ||w_{j+1}|| <= tol ||p||.
//
// Tiling: a block marches along z through 32 x 8 columns of the grid (Sec.
// III-A of the paper keeps a 2D slice on chip and iterates over the third
// index; here the slice is fed by TMA).  The one-iteration kernel runs one
// wave of resident blocks, each taking an equal run of the column-planes
// (one or more z-runs); the two-iteration kernel gives each block one
// column's chunk of planes.  Per plane, one thread
// issues cp.async.bulk.tensor loads of the w tile with its x/y halo (x start
// rounded down to a 16-byte boundary), the coefficient tiles and the p tile
// into two rings: the w tiles (planes z-1, z, z+1 are read while plane z is
// computed) and the coefficient and p tiles (plane z only).  Four planes (two
// for native FP64) are in flight ahead of the one being computed; an mbarrier
// per plane carries the transaction bytes of all its copies.  Halo columns and planes outside the grid arrive as zeros (TMA
// out-of-bounds fill); with the explicit-coefficient layout every coefficient
// that would touch them is zero, so no boundary branches are needed.
//
// Every mbarrier wait is bounded (0.5 s of %globaltimer); a block that gives up
// records it in ctl->err, waits (bounded) for its own copies in flight and
// still takes part in the reduction, whose last block reports status 5.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "ei_device.cuh"

namespace ei {

template <int FMT>
struct TmaCfg {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  static constexpr int TX = 32, TY = 8;
  // planes in flight ahead of the one computed.  Native FP64 is bound by its
  // arithmetic rather than by HBM: a shallower ring lets more blocks share an
  // SM and keep its FP64 pipe busy across the per-plane barriers.
  static constexpr int PF = FMT == VF_F64 ? 2 : 4;
  static constexpr int MINB = FMT == VF_F64 ? 3 : 2;  // resident blocks per SM
  // planes per block barrier: a ring one slot deeper per extra plane lets a
  // thread lag the issuing thread by that many planes
  static constexpr int SYNC = 1;
  static constexpr int NW = PF + 1 + SYNC;  // w ring: planes z-1, z, z+1 + PF in flight
  static constexpr int NC = PF + SYNC;      // coefficient/p ring: plane z + PF in flight
  static constexpr int NBAR = 8;        // one mbarrier per plane, reused every 8 planes
  static constexpr int HX = 16 / (int)sizeof(T);  // x halo, rounded to 16 bytes
  static constexpr int WX = TX + 2 * HX, WY = TY + 2;
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int W_BYTES = WX * WY * (int)sizeof(T);
  static constexpr int C_BYTES = TX * TY * (int)sizeof(T);
  static constexpr int P_BYTES = TX * TY * (int)sizeof(P);
  static constexpr int N_CT = 7;        // interior coefficient tiles: a[0..5], diagonal
  // w-ring slot: the w halo tile
  static constexpr int OFF_W = 0;
  static constexpr int WSTAGE = al(W_BYTES);
  // coefficient-ring slot: interior coefficient tiles, then the p tile
  static constexpr int OFF_CT = 0;
  static constexpr int OFF_P = N_CT * C_BYTES;
  static constexpr int CSTAGE = al(OFF_P + P_BYTES);
  static constexpr int CRING = NW * WSTAGE;
  static constexpr int BARS = CRING + NC * CSTAGE;
  static constexpr int SMEM = BARS + 8 * NBAR + 128;  // + alignment slack
};

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the given phase parity; false when limit_ns of wall time passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

static constexpr uint64_t kWaitLimitNs = 500000000ull;  // 0.5 s; a plane lands in microseconds

// One-iteration Newton launches go out with programmatic stream serialization
// (launch_pdl): a launch may be scheduled while the previous Newton step
// drains (15.584 -> 15.466 ms a native 256^3 step; the two-iteration kernel's
// many-wave grid gained nothing and launches plainly).  Before reading anything that step wrote (w, p, the control block)
// it waits for that grid to complete and its writes to be visible; then it
// lets the next launch be scheduled early in turn.  Both are no-ops for a
// launch without the attribute.
__device__ __forceinline__ void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// PRE: the coefficient tiles hold the scaled operator (A - cI)/gamma (native
// FP64 and float-float), so w_{j+1} = (A w_j - c w_j)/gamma - xi_j w_j is the
// 7-point sum and one multiply-add with -xi_j: the scaling saves a multiply
// per point.
// PN: form both squared norms in FP64 (false only with s.bracket, native
// FP64: both are bracketed in FP32, which saves the FP64-bound kernel two FMAs
// a point)
// FSTEP (native FP64 or float-float, with PRE false): the step's F pass
// instead of a Newton iteration (launch_f_tma): u in M.w, A's raw coefficients
// in M.c, F to w_out, J's diagonal to p_; it runs whatever ctl->done says.
// 1: g none or logistic; 2: also the combustion terms (a separate
// instantiation: their exponential and reciprocal take many registers).
// FACES: the Dirichlet data's face terms are compiled in (a separate
// instantiation: the compiler predicates their FP64 adds onto every point,
// which the FP64-bound pass cannot afford).
template <int FMT, bool PRE, bool PN = true, int FSTEP = 0, bool FACES = false>
__global__ void __launch_bounds__(256, TmaCfg<FMT>::MINB)
k_newton_tma(const __grid_constant__ NewtonMaps M, const StencilDev g, const NewtonScalars s,
             void* __restrict__ w_out_, void* __restrict__ p_, double* partials, DevCtl* ctl,
             const FStepArgs fa) {
  using C = TmaCfg<FMT>;
  using T = typename C::T;
  using P = typename C::P;
  static_assert(!FSTEP || !PRE, "the F pass runs on A");
  if constexpr (!FSTEP) pdl_wait_and_release();
  if (!FSTEP && *(volatile int*)&ctl->done != 0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // stage tiles start on 128-byte boundaries whatever the static shared memory
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  unsigned char* smem = smem_raw + (sbase - raw);
  const uint32_t bar0 = sbase + C::BARS;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * C::TX + tx;
  // this block's equal share [ub, ue) of the column-planes u = column * nz + z
  // (columns of 32 x 8 points, x fastest): one or more z-runs (segments)
  const int bxc = (g.nx + C::TX - 1) / C::TX;
  const int64_t units = (int64_t)bxc * ((g.ny + C::TY - 1) / C::TY) * g.nz;
  const int64_t ub = units * blockIdx.x / gridDim.x;
  const int64_t ue = units * (blockIdx.x + 1) / gridDim.x;
  const bool needp = !FSTEP && s.j > 0;
  const uint32_t tx_halo = C::W_BYTES;
  const uint32_t tx_full = tx_halo + C::N_CT * C::C_BYTES + (needp ? C::P_BYTES : 0);

  if (tid == 0) {
    for (int i = 0; i < C::NBAR; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncthreads();

  const T invg = from_d<T>(s.inv_gamma);
  const T nshift = from_d<T>(PRE ? -s.xi : -s.shift);
  const P dn = from_d<P>(s.d_next);
  const P d0 = from_d<P>(s.d0);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  // bracket steps (!PN, native FP64): ||w_{j+1}||^2 and ||p_{j+1}||^2 are only
  // bracketed, in FP32 off the FP64 pipe (NormBrackets)
  NormBrackets br;
  if constexpr (!PN) br.init(ctl, (double)g.nx * g.ny * g.nz);
  // F pass: ||F||^2 and the interval keys of J's Gershgorin rows
  T af = zero<T>();
  long long kmn = order_key(INFINITY), kmx = order_key(-INFINITY);
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  const int wi = (ty + 1) * C::WX + tx + C::HX;
  const int ci = ty * C::TX + tx;
  constexpr int TT = C::TX * C::TY;
  bool bad = false;
  // The mbarriers count planes over all segments (qb: planes of the earlier
  // ones), so their phases run on; the ring slots restart with each segment.
  int qb = 0;
  int last_issued = -1;  // last plane issued (thread 0)
  int waited_ok = -1;    // last plane whose copies this thread saw complete

  for (int64_t us = ub; us < ue && !bad;) {
    const int col = (int)(us / g.nz);
    const int z0 = (int)(us - (int64_t)col * g.nz);
    const int z1 = (int)min((int64_t)g.nz, z0 + (ue - us));
    us += z1 - z0;
    const int x0 = (col % bxc) * C::TX, y0 = (col / bxc) * C::TY;
    const int nplanes = z1 - z0 + 2;  // z0-1 .. z1
    auto issue = [&](int q) {
      const uint32_t wb = sbase + (q % C::NW) * C::WSTAGE;
      const uint32_t cb = sbase + C::CRING + (q % C::NC) * C::CSTAGE;
      const uint32_t bar = bar0 + 8 * ((qb + q) % C::NBAR);
      const int z = z0 - 1 + q;
      const bool halo = (q == 0) || (q == nplanes - 1);
      mbar_expect_tx(bar, halo ? tx_halo : tx_full);
      tma_load_3d(wb + C::OFF_W, &M.w, x0 - C::HX, y0 - 1, z, bar);
      if (!halo) {
#pragma unroll
        for (int k = 0; k < C::N_CT; ++k)
          tma_load_3d(cb + C::OFF_CT + k * C::C_BYTES, &M.c[k], x0, y0, z, bar);
        if (needp) tma_load_3d(cb + C::OFF_P, &M.p, x0, y0, z, bar);
      }
      last_issued = qb + q;
    };
    auto wait = [&](int q) {
      const int qg = qb + q;
      const bool ok =
          mbar_wait_bounded(bar0 + 8 * (qg % C::NBAR), (qg / C::NBAR) & 1, kWaitLimitNs);
      if (ok) waited_ok = qg;
      return ok;
    };

    if (tid == 0) {
      // the previous segment's reads of these slots ended at its last barrier
      fence_proxy_async();
      for (int q = 0; q <= C::PF && q < nplanes; ++q) issue(q);
    }
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = (x < g.nx) && (y < g.ny);

    for (int q = 1; q <= nplanes - 2; ++q) {
      if (tid == 0 && q + C::PF < nplanes) {
        fence_proxy_async();
        issue(q + C::PF);  // into the slots of planes q+PF-NW (w) and q+PF-NC (coefficients)
      }
      if (q == 1) {
        if (!bad) bad = !wait(0);
        if (!bad) bad = !wait(1);
      }
      if (!bad) bad = !wait(q + 1);
      if (!bad && inside) {
        const int z = z0 - 1 + q;
        const unsigned char* sm = smem + (q % C::NW) * C::WSTAGE;
        const unsigned char* smm = smem + ((q - 1) % C::NW) * C::WSTAGE;
        const unsigned char* smp = smem + ((q + 1) % C::NW) * C::WSTAGE;
        const unsigned char* scq = smem + C::CRING + (q % C::NC) * C::CSTAGE;
        const T* Wc = reinterpret_cast<const T*>(sm + C::OFF_W);
        const T* Wm = reinterpret_cast<const T*>(smm + C::OFF_W);
        const T* Wp = reinterpret_cast<const T*>(smp + C::OFF_W);
        const T* Ct = reinterpret_cast<const T*>(scq + C::OFF_CT);
        const T wc = Wc[wi];
        const T acc = stencil7(Ct[6 * TT + ci], wc, Ct[0 * TT + ci], Wc[wi - 1], Ct[1 * TT + ci],
                               Wc[wi + 1], Ct[2 * TT + ci], Wc[wi - C::WX], Ct[3 * TT + ci],
                               Wc[wi + C::WX], Ct[4 * TT + ci], Wm[wi], Ct[5 * TT + ci], Wp[wi]);
        const int64_t idx = ((int64_t)z * g.ny + y) * g.pitch + x;
        if constexpr (FSTEP) {
          // F = A u + g(u), g(u) = u(1 - u), g'(u) = 1 - 2u (logistic)
          const T one = from_d<T>(1.0), mtwo = from_d<T>(-2.0);
          T Fv = acc, gq = zero<T>();
          if (FACES &&
              (x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1)) {
            // b_D: the Dirichlet data's face terms at the rows next to a face
            double bd = 0.0;
            if (x == 0 && fa.face[0]) bd += fa.face[0][(int64_t)z * g.ny + y];
            if (x == g.nx - 1 && fa.face[1]) bd += fa.face[1][(int64_t)z * g.ny + y];
            if (y == 0 && fa.face[2]) bd += fa.face[2][(int64_t)z * g.nx + x];
            if (y == g.ny - 1 && fa.face[3]) bd += fa.face[3][(int64_t)z * g.nx + x];
            if (z == 0 && fa.face[4]) bd += fa.face[4][(int64_t)y * g.nx + x];
            if (z == g.nz - 1 && fa.face[5]) bd += fa.face[5][(int64_t)y * g.nx + x];
            if (bd != 0.0) Fv = add(Fv, from_d<T>(bd));
          }
          if (fa.nonlin == EI_NONLIN_LOGISTIC) {
            Fv = mac(Fv, wc, sub(one, wc));
            gq = mac(one, mtwo, wc);
          } else if constexpr (FSTEP == 2) {
            if (fa.nonlin != EI_NONLIN_NONE) {
              T gv;
              combustion_term(fa.nonlin, wc, gv, gq);
              Fv = add(Fv, gv);
            }
          }
          st(w_out, idx, Fv);
          if (fa.rosen) {
            st(static_cast<T*>(p_), idx, add(Ct[6 * TT + ci], gq));  // J's diagonal
            const int64_t ic = ((int64_t)z * g.ny + y) * g.nx + x;
            // g'(u) of the interval in FP64: the other formats take the
            // logistic slope of the caller's u (as the separate interval pass
            // does) and the combustion slope in their own format from u as
            // imported (the separate pass converts the caller's u itself; both
            // conversions keep the format's 48 bits, so the slopes agree to
            // its precision)
            double q;
            if constexpr (FMT == VF_F64) {
              q = gq;
            } else if (fa.nonlin == EI_NONLIN_LOGISTIC) {
              const double ud = FMT == VF_F32
                                    ? (double)__ldg(static_cast<const float*>(fa.u) + ic)
                                    : __ldg(static_cast<const double*>(fa.u) + ic);
              q = 1.0 - 2.0 * ud;
            } else {
              q = to_d(gq);
            }
            const long long kl = order_key(__ldg(fa.lo + ic) + q);
            const long long kh = order_key(__ldg(fa.hi + ic) + q);
            kmn = kl < kmn ? kl : kmn;
            kmx = kh > kmx ? kh : kmx;
          }
          af = mac(af, Fv, Fv);
        } else {
          const T wn = PRE ? mac(acc, nshift, wc) : newton_update(acc, invg, nshift, wc);
          const P* Pt = reinterpret_cast<const P*>(scq + C::OFF_P);
          const P pold = needp ? Pt[ci] : mul(d0, to_p(wc));
          const P pn = mac(pold, dn, to_p(wn));
          st(w_out, idx, wn);
          st(p, idx, pn);
          if constexpr (PN) {
            aw = acc_sq(aw, wn);
            ap = acc_sq(ap, pn);
          } else {
            br.add(wn, pn);
          }
        }
      }
      // every plane: the slots read here are reissued only after this barrier
      // (the segment's last plane included, which frees all slots for the next)
      if ((q % C::SYNC == 0 || q == nplanes - 2) && __syncthreads_or(bad)) {
        bad = true;
        break;
      }
    }
    qb += nplanes;
  }
  if (bad && tid == 0) {
    atomicOr(&ctl->err, 1);
    // let this block's copies in flight land before its shared memory goes away
    for (int q = waited_ok + 1; q <= last_issued; ++q)
      mbar_wait_bounded(bar0 + 8 * (q % C::NBAR), (q / C::NBAR) & 1, kWaitLimitNs / 8);
  }

  if constexpr (FSTEP) {
    double v[4] = {to_d(af), 0.0, key_value(kmn), key_value(kmx)};
    if (isnan(v[2]) || isnan(v[3])) {
      v[2] = -INFINITY;
      v[3] = INFINITY;
    }
    if (last_block_reduce4<RED_SUM, RED_MINMAX>(v, partials, ctl)) {
      if (tid == 0) {
        ctl->sum0 = v[0];
        ctl->sum1 = finite_d(v[0]) ? 1.0 : 0.0;
        if (fa.rosen) {
          ctl->mn = v[2];
          ctl->mx = v[3];
        }
      }
    }
    return;
  }
  double nw2 = PN ? acc_d(aw) : br.sum_w(), np2 = PN ? acc_d(ap) : br.sum_p();
  if (last_block_reduce2<RED_SUM>(nw2, np2, partials, ctl)) {
    if (tid == 0) {
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      if constexpr (PN)
        newton_verdict(ctl, s, s.j + 1, s.d_next, nw2, np2);
      else
        br.verdict(ctl, s, nw2, np2, (double)((units + gridDim.x - 1) / gridDim.x));
    }
  }
}


// ===========================================================================
// Two Newton iterations per pass (temporal blocking), explicit coefficients.
//
// The pass reads w_j with a two-point halo, the coefficient and p tiles of
// each plane once, forms w_{j+1} on chip over the tile plus a one-point halo
// (the halo points' coefficients come from global memory, where they are the
// neighbouring tiles' interior), and writes only w_{j+2} and p_{j+2}:
// 88 bytes per point for two iterations instead of 176.  w_{j+1} and p_{j+1}
// are bit-identical to the one-iteration kernel's, so the stop test is taken
// at both degrees; when it already holds at j+1 the host subtracts
// d_{j+2} w_{j+2} from p.
//
// z-march step m computes w_{j+1} on plane zc = z0-1+m and, from m = 2 on,
// w_{j+2} on plane zc-1.  It reads w_j planes zc-1..zc+1 and the coefficients
// of planes zc (w_{j+1}) and zc-1 (w_{j+2}).  Only the x/y neighbours of
// w_{j+1} cross threads: they come from the plane finished in the previous
// step (a ring of 2 in shared memory); the centre and z neighbours are the
// thread's own values in registers, so a step needs a single barrier.
// ===========================================================================
// CONST: the operator's coefficients come from a 70-entry table (kConstTab)
// instead of seven tiles a plane, so a coefficient-ring slot holds the p tile
// alone and the table follows the mbarriers.
template <int FMT, bool CONST = false>
struct TmaCfg2 {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  static constexpr int TX = 32, TY = 8;
  static constexpr int PF = 2;                 // planes in flight ahead
  static constexpr int NW = PF + 3, NC = PF + 3, NBAR = 8;
  // w_j box: two-point halo in y; in x the halo is widened to 16 bytes (2
  // elements of 8 bytes, 4 of 4 bytes) so the box starts on a TMA boundary
  static constexpr int XH = 16 / (int)sizeof(T);
  static constexpr int WJX = TX + 2 * XH, WJY = TY + 4;
  static constexpr int W1X = TX + 2, W1Y = TY + 2;   // w_{j+1} region, one-point halo
  static constexpr int NHALO = W1X * W1Y - TX * TY;  // 84
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int WJ_BYTES = WJX * WJY * (int)sizeof(T);
  static constexpr int C_BYTES = TX * TY * (int)sizeof(T);
  static constexpr int P_BYTES = TX * TY * (int)sizeof(P);
  static constexpr int WSTAGE = al(WJ_BYTES);
  static constexpr int OFF_P = CONST ? 0 : 7 * C_BYTES;
  static constexpr int CSTAGE = al(OFF_P + P_BYTES);
  static constexpr int W1STAGE = al(W1X * W1Y * (int)sizeof(T));
  static constexpr int CRING = NW * WSTAGE;
  static constexpr int W1RING = CRING + NC * CSTAGE;
  static constexpr int BARS = W1RING + 2 * W1STAGE;
  static constexpr int TAB = BARS + 8 * NBAR;
  static constexpr int SMEM = TAB + (CONST ? kConstTab * (int)sizeof(T) : 0) + 128;
};

// The boundary class of a coordinate: bit 0 on the low face, bit 1 on the
// high one (both when the extent is 1).  A point's class is cx + 4 cy + 16 cz.
__device__ __forceinline__ int face_class(int x, int n) {
  return (x == 0 ? 1 : 0) | (x == n - 1 ? 2 : 0);
}

template <int FMT, bool PRE = false, bool CONST = false>
__global__ void __launch_bounds__(256, CONST ? 3 : 2)
k_newton2_tma(const __grid_constant__ NewtonMaps M, const StencilDev g, const NewtonScalars s,
              void* __restrict__ w_out_, void* __restrict__ p_, double* partials, DevCtl* ctl,
              int zc_len, const void* __restrict__ ctab) {
  using C = TmaCfg2<FMT, CONST>;
  using T = typename C::T;
  using P = typename C::P;
  if (*(volatile int*)&ctl->done != 0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  unsigned char* smem = smem_raw + (sbase - raw);
  const uint32_t bar0 = sbase + C::BARS;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * C::TX + tx;
  const int x0 = blockIdx.x * C::TX, y0 = blockIdx.y * C::TY;
  const int z0 = blockIdx.z * zc_len;
  const int z1 = min(z0 + zc_len, g.nz);
  const int nzc = z1 - z0;
  const int nq = nzc + 4;  // w_j planes z0-2 .. z1+1
  const bool needp = s.j > 0;
  // CONST: the six off-diagonals, then the diagonal of each boundary class
  T* ktab = reinterpret_cast<T*>(smem + C::TAB);
  if constexpr (CONST) {
    if (tid < kConstTab) ktab[tid] = ldg(static_cast<const T*>(ctab), tid);
  }

  if (tid == 0) {
    for (int i = 0; i < C::NBAR; ++i) mbar_init(bar0 + 8 * i, 1);
    fence_mbar_init();
  }
  __syncthreads();

  int last_issued = -1;
  auto issue = [&](int q) {
    const uint32_t wb = sbase + (q % C::NW) * C::WSTAGE;
    const uint32_t cb = sbase + C::CRING + (q % C::NC) * C::CSTAGE;
    const uint32_t bar = bar0 + 8 * (q % C::NBAR);
    const int z = z0 - 2 + q;
    // coefficient planes z0-1 .. z1
    const bool hasc = !CONST && (q >= 1) && (q <= nzc + 2);
    const bool hasp = needp && (q >= 2) && (q <= nzc + 1);
    mbar_expect_tx(bar, C::WJ_BYTES + (hasc ? 7 * C::C_BYTES : 0) + (hasp ? C::P_BYTES : 0));
    tma_load_3d(wb, &M.w, x0 - C::XH, y0 - 2, z, bar);
    if (hasc) {
#pragma unroll
      for (int k = 0; k < 7; ++k) tma_load_3d(cb + k * C::C_BYTES, &M.c[k], x0, y0, z, bar);
    }
    if (hasp) tma_load_3d(cb + C::OFF_P, &M.p, x0, y0, z, bar);
    last_issued = q;
  };
  int waited_ok = -1;
  auto wait = [&](int q) {
    const bool ok = mbar_wait_bounded(bar0 + 8 * (q % C::NBAR), (q / C::NBAR) & 1, kWaitLimitNs);
    if (ok) waited_ok = q;
    return ok;
  };
  if (tid == 0) {
    for (int q = 0; q <= 2 + C::PF && q < nq; ++q) issue(q);
  }

  // PRE: the coefficient tiles and halo coefficients hold the scaled operator
  // (the update is the 7-point sum and one multiply-add with the shift)
  const T invg = from_d<T>(s.inv_gamma);
  const T nsh1 = from_d<T>(PRE ? -s.xi : -s.shift);
  const T nsh2 = from_d<T>(PRE ? -s.xi2 : -s.shift2);
  const P d1 = from_d<P>(s.d_next);
  const P d2 = from_d<P>(s.d_next2);
  const P d0 = from_d<P>(s.d0);
  double acc4[4] = {0.0, 0.0, 0.0, 0.0};
  typename Acc<T>::type aw1 = Acc<T>::zero(), aw2 = Acc<T>::zero();
  typename Acc<P>::type ap1 = Acc<P>::zero(), ap2 = Acc<P>::zero();
  T* __restrict__ w_out = static_cast<T*>(w_out_);
  P* __restrict__ p = static_cast<P*>(p_);
  constexpr int TT = C::TX * C::TY;
  // every thread owns one of the 32 x 8 interior points; threads 0-83 (the
  // first three warps) also one of the 84 halo points of the 34 x 10 region
  const bool interior = true;
  int hlx = -1, hly = -1;
  if (tid < C::NHALO) {
    const int h = tid;
    if (h < C::W1X) { hlx = h; hly = 0; }
    else if (h < 2 * C::W1X) { hlx = h - C::W1X; hly = C::W1Y - 1; }
    else if (h < 2 * C::W1X + C::TY) { hlx = 0; hly = 1 + h - 2 * C::W1X; }
    else { hlx = C::W1X - 1; hly = 1 + h - 2 * C::W1X - C::TY; }
  }
  const int hx = x0 - 1 + hlx, hy = y0 - 1 + hly;
  const bool hxy = hlx >= 0 && hx >= 0 && hx < g.nx && hy >= 0 && hy < g.ny;
  const int hcls = CONST && hxy ? face_class(hx, g.nx) + 4 * face_class(hy, g.ny) : 0;
  // halo coefficients come from global memory one step ahead of their use
  // (CONST: from the table where they are used; an off-diagonal towards a
  // neighbour outside the grid multiplies the zero that the w box holds there)
  auto load_halo = [&](int zz, T* a) {
    if (hxy && zz >= 0 && zz < g.nz) {
      const int64_t gi = ((int64_t)zz * g.ny + hy) * g.pitch + hx;
#pragma unroll
      for (int k = 0; k < 6; ++k) a[k] = ldg(static_cast<const T*>(g.a[k]), gi);
      a[6] = ldg(static_cast<const T*>(g.diag), gi);
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) a[k] = zero<T>();
    }
  };
  T hcur[CONST ? 1 : 7], hnxt[CONST ? 1 : 7];
  if constexpr (!CONST) load_halo(z0 - 1, hcur);
  bool bad = false;

  // this thread's own w_{j+1} values on planes zc-2 and zc-1 (registers)
  T w1_m2 = zero<T>(), w1_m1 = zero<T>();
  const int xi_ = x0 + tx, yi_ = y0 + ty;
  const bool own_xy = interior && (xi_ < g.nx) && (yi_ < g.ny);
  const int ocls = CONST ? face_class(xi_, g.nx) + 4 * face_class(yi_, g.ny) : 0;
  const int wi_own = (ty + 2) * C::WJX + tx + C::XH;  // own point in the w_j box
  const int vi_own = (ty + 1) * C::W1X + tx + 1;   // own point in the w_{j+1} region
  const int ci = ty * C::TX + tx;
  int sw = 0, sc = 0;  // ring slots of plane m (w_j ring, coefficient ring)

  for (int m = 0; m <= nzc + 1; ++m) {
    if (tid == 0 && m >= 1 && m + 2 + C::PF < nq) {
      fence_proxy_async();
      issue(m + 2 + C::PF);  // into the slots of plane m-1
    }
    if (m == 0) {
      if (!bad) bad = !wait(0);
      if (!bad) bad = !wait(1);
    }
    if (!bad) bad = !wait(m + 2);
    const int zc = z0 - 1 + m;
    if constexpr (!CONST) {
      if (hlx >= 0) load_halo(zc + 1, hnxt);  // in flight while this step computes
    }
    const int sw1 = (sw + 1 == C::NW) ? 0 : sw + 1, sw2 = (sw1 + 1 == C::NW) ? 0 : sw1 + 1;
    const int sc1 = (sc + 1 == C::NC) ? 0 : sc + 1;
    T w1own = zero<T>();
    if (!bad) {
      const T* Wm = reinterpret_cast<const T*>(smem + sw * C::WSTAGE);
      const T* Wc = reinterpret_cast<const T*>(smem + sw1 * C::WSTAGE);
      const T* Wp = reinterpret_cast<const T*>(smem + sw2 * C::WSTAGE);
      T* W1 = reinterpret_cast<T*>(smem + C::W1RING + (m & 1) * C::W1STAGE);
      const bool zin = (zc >= 0) && (zc < g.nz);
      // ---- w_{j+1}(zc) at the own point
      if (interior && zin && own_xy) {
        const T* Ct = reinterpret_cast<const T*>(smem + C::CRING + sc1 * C::CSTAGE);
        const T wc = Wc[wi_own];
        T acc;
        if constexpr (CONST)
          acc = stencil7(ktab[6 + ocls + 16 * face_class(zc, g.nz)], wc, ktab[0],
                         Wc[wi_own - 1], ktab[1], Wc[wi_own + 1], ktab[2], Wc[wi_own - C::WJX],
                         ktab[3], Wc[wi_own + C::WJX], ktab[4], Wm[wi_own], ktab[5], Wp[wi_own]);
        else
          acc = stencil7(Ct[6 * TT + ci], wc, Ct[0 * TT + ci], Wc[wi_own - 1], Ct[1 * TT + ci],
                         Wc[wi_own + 1], Ct[2 * TT + ci], Wc[wi_own - C::WJX], Ct[3 * TT + ci],
                         Wc[wi_own + C::WJX], Ct[4 * TT + ci], Wm[wi_own], Ct[5 * TT + ci],
                         Wp[wi_own]);
        w1own = PRE ? mac(acc, nsh1, wc) : newton_update(acc, invg, nsh1, wc);
      }
      if (interior) W1[vi_own] = w1own;
      // ---- w_{j+1}(zc) at this thread's halo point (first three warps)
      if (hlx >= 0) {
        T w1 = zero<T>();
        if (zin && hxy) {
          const int wi = (hly + 1) * C::WJX + hlx + C::XH - 1;
          const T wc = Wc[wi];
          T acc;
          if constexpr (CONST)
            acc = stencil7(ktab[6 + hcls + 16 * face_class(zc, g.nz)], wc, ktab[0], Wc[wi - 1],
                           ktab[1], Wc[wi + 1], ktab[2], Wc[wi - C::WJX], ktab[3],
                           Wc[wi + C::WJX], ktab[4], Wm[wi], ktab[5], Wp[wi]);
          else
            acc = stencil7(hcur[6], wc, hcur[0], Wc[wi - 1], hcur[1], Wc[wi + 1], hcur[2],
                           Wc[wi - C::WJX], hcur[3], Wc[wi + C::WJX], hcur[4], Wm[wi], hcur[5],
                           Wp[wi]);
          w1 = PRE ? mac(acc, nsh1, wc) : newton_update(acc, invg, nsh1, wc);
        }
        W1[hly * C::W1X + hlx] = w1;
      }
      // ---- w_{j+2}(zc - 1) at the own point: its x/y neighbours come from the
      // w_{j+1} plane finished in the previous step, its z neighbours and centre
      // are this thread's own values
      if (m >= 2 && own_xy) {
        const int z = zc - 1;
        const T* V1 = reinterpret_cast<const T*>(smem + C::W1RING + ((m - 1) & 1) * C::W1STAGE);
        const unsigned char* cs = smem + C::CRING + sc * C::CSTAGE;
        const T* Ct = reinterpret_cast<const T*>(cs);
        const P* Pt = reinterpret_cast<const P*>(cs + C::OFF_P);
        const T w1c = w1_m1;
        T acc;
        if constexpr (CONST)
          acc = stencil7(ktab[6 + ocls + 16 * face_class(z, g.nz)], w1c, ktab[0],
                         V1[vi_own - 1], ktab[1], V1[vi_own + 1], ktab[2], V1[vi_own - C::W1X],
                         ktab[3], V1[vi_own + C::W1X], ktab[4], w1_m2, ktab[5], w1own);
        else
          acc = stencil7(Ct[6 * TT + ci], w1c, Ct[0 * TT + ci], V1[vi_own - 1], Ct[1 * TT + ci],
                         V1[vi_own + 1], Ct[2 * TT + ci], V1[vi_own - C::W1X], Ct[3 * TT + ci],
                         V1[vi_own + C::W1X], Ct[4 * TT + ci], w1_m2, Ct[5 * TT + ci], w1own);
        const T w2 = PRE ? mac(acc, nsh2, w1c) : newton_update(acc, invg, nsh2, w1c);
        const P pj = needp ? Pt[ci] : mul(d0, to_p(Wm[wi_own]));
        const P p1 = mac(pj, d1, to_p(w1c));
        const P p2 = mac(p1, d2, to_p(w2));
        const int64_t idx = ((int64_t)z * g.ny + yi_) * g.pitch + xi_;
        st(w_out, idx, w2);
        st(p, idx, p2);
        aw1 = acc_sq(aw1, w1c);
        ap1 = acc_sq(ap1, p1);
        aw2 = acc_sq(aw2, w2);
        ap2 = acc_sq(ap2, p2);
      }
    }
    w1_m2 = w1_m1;
    w1_m1 = w1own;
    if (!CONST && hlx >= 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) hcur[k] = hnxt[k];
    }
    sw = sw1;
    sc = sc1;
    if (__syncthreads_or(bad)) {
      bad = true;
      break;
    }
  }
  if (bad && tid == 0) {
    atomicOr(&ctl->err, 1);
    for (int q = waited_ok + 1; q <= last_issued; ++q)
      mbar_wait_bounded(bar0 + 8 * (q % C::NBAR), (q / C::NBAR) & 1, kWaitLimitNs / 8);
  }
  acc4[0] = acc_d(aw1);
  acc4[1] = acc_d(ap1);
  acc4[2] = acc_d(aw2);
  acc4[3] = acc_d(ap2);
  if (last_block_reduce4(acc4, partials, ctl)) {
    if (tid == 0) {
      const double nw1 = acc4[0], np1 = acc4[1], nw2 = acc4[2], np2 = acc4[3];
      ctl->nw2 = nw2;
      ctl->np2 = np2;
      if (!finite_d(nw2) || !finite_d(np2)) {
        newton_verdict(ctl, s, s.j + 1, s.d_next, nw2, np2);  // stops: non-finite
      } else if (newton_verdict(ctl, s, s.j + 1, s.d_next, nw1, np1)) {
        // stopped at j+1 (not at degree 0): p holds p_{j+2}; the host fixes it
        if (ctl->done <= 2 && ctl->degree == s.j + 1) ctl->fixup = 1;
      } else {
        newton_verdict(ctl, s, s.j + 2, s.d_next2, nw2, np2);
      }
    }
  }
}

template <int FMT>
__global__ void k_p_fixup(void* p_, const void* w_, int64_t n, double d) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  P* p = static_cast<P*>(p_);
  const T* w = static_cast<const T*>(w_);
  const P nd = from_d<P>(-d);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    st(p, i, mac(ld(p, i), nd, to_p(ldg(w, i))));
}

// ---- host side ----------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool encode_map(CUtensorMap* m, const void* base, int elem_bytes, const StencilDev& g, int halo) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int hx = 16 / elem_bytes;
  cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  cuuint64_t strides[2] = {(cuuint64_t)g.pitch * elem_bytes,
                           (cuuint64_t)g.pitch * g.ny * elem_bytes};
  cuuint32_t box[3] = {(cuuint32_t)(32 + (halo ? 2 * hx : 0)), (cuuint32_t)(8 + 2 * halo), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Planes per block (the z-chunk).  Blocks run in waves of `slots` (SMs x
// resident blocks per SM) and the last, partial wave takes as long as a full
// one, so the chunk is the candidate whose waves finish soonest: the time is
// modelled as waves x (zc + halo), `halo` being a block's fixed cost in planes
// (its extra halo planes and pipeline start).  Ties go to the larger chunk.
static constexpr int kZChunks[5] = {64, 32, 16, 8, 4};
static int tma_zchunk(const StencilDev& g, int slots, double halo) {
  const int64_t bxy = (int64_t)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
  int best = 1;
  double best_t = INFINITY;
  for (int zc : kZChunks) {
    const int z = zc < g.nz ? zc : g.nz;
    const int64_t nzb = (g.nz + z - 1) / z;
    if (nzb > 65535) continue;
    const int64_t waves = (bxy * nzb + slots - 1) / slots;
    const double t = (double)waves * (z + halo);
    if (t < best_t - 1e-9) {
      best_t = t;
      best = z;
    }
  }
  return best;
}

int newton_tma_blocks(const StencilDev& g) {
  const int64_t bxy = (int64_t)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
  const int zmin = kZChunks[4] < g.nz ? kZChunks[4] : g.nz;
  return (int)(bxy * ((g.nz + zmin - 1) / zmin));
}

// The two-iteration kernel's fixed cost of a block in plane-equivalents: two
// more w planes, two more coefficient planes and w_{j+1} on two more planes.
static constexpr double kHaloPair = 2.3;

// The one-iteration kernel's grid: one wave of resident blocks (SMs x blocks
// an SM holds), each an equal share of the column-planes, so that every SM
// runs the same work and all finish together.  (Sweeps of 6, 4, 3 and 2 waves
// of smaller shares on 256^3 were slower: each block start costs two halo
// planes and a pipeline fill, and a wave boundary leaves SMs waiting.)  No
// block takes fewer than kMinPlanes column-planes.
static constexpr int kMinPlanes = 4;
static int64_t tma_balanced_blocks(const StencilDev& g, int slots) {
  const int64_t units = (int64_t)((g.nx + 31) / 32) * ((g.ny + 7) / 8) * g.nz;
  const int64_t cap = (units + kMinPlanes - 1) / kMinPlanes;
  const int64_t nb = slots < cap ? slots : cap;
  return nb < 1 ? 1 : nb;
}

// a kernel launch with programmatic stream serialization allowed
template <class... KArgs, class... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int FMT, bool PRE, bool PN = true, int FSTEP = 0, bool FACES = false>
static cudaError_t launch_one(const StencilDev& g, const NewtonMaps& M, void* w_out, void* p,
                              const NewtonScalars& s, double* partials, DevCtl* ctl,
                              cudaStream_t st, const FStepArgs& fa = FStepArgs{}) {
  using C = TmaCfg<FMT>;
  static int slots = 0;
  if (slots == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_newton_tma<FMT, PRE, PN, FSTEP, FACES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_newton_tma<FMT, PRE, PN, FSTEP, FACES>, 256, C::SMEM);
    if (e != cudaSuccess) return e;
    slots = (per_sm > 0 ? per_sm : 1) * sm_count();
  }
  const int64_t nb = tma_balanced_blocks(g, slots);
  if constexpr (FSTEP == 0)
    return launch_pdl(k_newton_tma<FMT, PRE, PN, FSTEP>, dim3((unsigned)nb), dim3(32, 8, 1),
                      C::SMEM, st, M, g, s, w_out, p, partials, ctl, fa);
  k_newton_tma<FMT, PRE, PN, FSTEP, FACES><<<(unsigned)nb, dim3(32, 8, 1), C::SMEM, st>>>(
      M, g, s, w_out, p, partials, ctl, fa);
  return cudaGetLastError();
}

template <int FMT, int FSTEP>
static cudaError_t launch_f_faces(const StencilDev& g, const NewtonMaps& M, void* F, void* dout,
                                  const FStepArgs& fa, double* partials, DevCtl* ctl,
                                  cudaStream_t st) {
  bool faces = false;
  for (int f = 0; f < 6; ++f) faces = faces || fa.face[f] != nullptr;
  const NewtonScalars none{};
  if (faces)
    return launch_one<FMT, false, true, FSTEP, true>(g, M, F, dout, none, partials, ctl, st, fa);
  return launch_one<FMT, false, true, FSTEP, false>(g, M, F, dout, none, partials, ctl, st, fa);
}

cudaError_t launch_f_tma(const StencilDev& g, const NewtonMaps& M, void* F, void* dout,
                         const FStepArgs& fa, int fmt, double* partials, DevCtl* ctl,
                         cudaStream_t st) {
  const bool comb = fa.nonlin != EI_NONLIN_NONE && fa.nonlin != EI_NONLIN_LOGISTIC;
  if (fmt == VF_DF)
    return comb ? launch_f_faces<VF_DF, 2>(g, M, F, dout, fa, partials, ctl, st)
                : launch_f_faces<VF_DF, 1>(g, M, F, dout, fa, partials, ctl, st);
  if (fmt == VF_F64)
    return comb ? launch_f_faces<VF_F64, 2>(g, M, F, dout, fa, partials, ctl, st)
                : launch_f_faces<VF_F64, 1>(g, M, F, dout, fa, partials, ctl, st);
  return comb ? launch_f_faces<VF_F32, 2>(g, M, F, dout, fa, partials, ctl, st)
              : launch_f_faces<VF_F32, 1>(g, M, F, dout, fa, partials, ctl, st);
}

cudaError_t launch_newton_tma(const StencilDev& g, const NewtonMaps& M, void* w_out, void* p,
                              const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                              cudaStream_t st, bool prescaled) {
  if (fmt == VF_DF && prescaled) return launch_one<VF_DF, true>(g, M, w_out, p, s, partials, ctl, st);
  if (fmt == VF_DF) return launch_one<VF_DF, false>(g, M, w_out, p, s, partials, ctl, st);
  if (fmt == VF_F64) {
    if (prescaled && s.bracket)
      return launch_one<VF_F64, true, false>(g, M, w_out, p, s, partials, ctl, st);
    if (prescaled) return launch_one<VF_F64, true>(g, M, w_out, p, s, partials, ctl, st);
    return launch_one<VF_F64, false>(g, M, w_out, p, s, partials, ctl, st);
  }
  return launch_one<VF_F32, false>(g, M, w_out, p, s, partials, ctl, st);
}

template <int FMT, bool PRE, bool CONST = false>
static cudaError_t launch_pair(const StencilDev& g, const NewtonMaps& M, void* w_out, void* p,
                               const NewtonScalars& s, double* partials, DevCtl* ctl,
                               cudaStream_t st, const void* ctab = nullptr) {
  using C = TmaCfg2<FMT, CONST>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_newton2_tma<FMT, PRE, CONST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // blocks per SM: two (shared memory for the coefficient tiles); the table
  // form three (its registers)
  const int zc = tma_zchunk(g, sm_count() * (CONST ? 3 : 2), kHaloPair);
  dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + zc - 1) / zc), block(32, 8, 1);
  k_newton2_tma<FMT, PRE, CONST><<<grid, block, C::SMEM, st>>>(M, g, s, w_out, p, partials, ctl,
                                                               zc, ctab);
  return cudaGetLastError();
}

cudaError_t launch_newton2_tma(const StencilDev& g, const NewtonMaps& M, void* w_out, void* p,
                               const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                               cudaStream_t st, bool prescaled, const void* ctab) {
  if (fmt == VF_DF && prescaled && ctab)
    return launch_pair<VF_DF, true, true>(g, M, w_out, p, s, partials, ctl, st, ctab);
  if (fmt == VF_DF && prescaled)
    return launch_pair<VF_DF, true>(g, M, w_out, p, s, partials, ctl, st);
  if (fmt == VF_DF) return launch_pair<VF_DF, false>(g, M, w_out, p, s, partials, ctl, st);
  if (fmt == VF_F64 && prescaled)
    return launch_pair<VF_F64, true>(g, M, w_out, p, s, partials, ctl, st);
  if (fmt == VF_F64) return launch_pair<VF_F64, false>(g, M, w_out, p, s, partials, ctl, st);
  return launch_pair<VF_F32, false>(g, M, w_out, p, s, partials, ctl, st);
}

// the constant operator's table: one thread an entry
template <class T>
__global__ void k_const_table(const __grid_constant__ ConstTabIdx ix, const T* a0, const T* a1,
                              const T* a2, const T* a3, const T* a4, const T* a5, const T* dg,
                              T* tab) {
  const int t = threadIdx.x;
  if (t >= kConstTab) return;
  const T* src = t == 0 ? a0 : t == 1 ? a1 : t == 2 ? a2 : t == 3 ? a3 : t == 4 ? a4
               : t == 5 ? a5 : dg;
  st(tab, t, ix.idx[t] >= 0 ? ldg(src, ix.idx[t]) : zero<T>());
}

cudaError_t launch_const_table(const void* const sa[7], const ConstTabIdx& ix, void* ctab,
                               int fmt, cudaStream_t st) {
  if (fmt == VF_DF) {
    k_const_table<df><<<1, 96, 0, st>>>(
        ix, static_cast<const df*>(sa[0]), static_cast<const df*>(sa[1]),
        static_cast<const df*>(sa[2]), static_cast<const df*>(sa[3]),
        static_cast<const df*>(sa[4]), static_cast<const df*>(sa[5]),
        static_cast<const df*>(sa[6]), static_cast<df*>(ctab));
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;  // the table form runs in float-float only
}

cudaError_t launch_p_fixup(void* p, const void* w, int fmt, int64_t n, double d,
                           cudaStream_t st) {
  const int nb = 152 * 8;
  if (fmt == VF_DF) k_p_fixup<VF_DF><<<nb, 256, 0, st>>>(p, w, n, d);
  else if (fmt == VF_F64) k_p_fixup<VF_F64><<<nb, 256, 0, st>>>(p, w, n, d);
  else k_p_fixup<VF_F32><<<nb, 256, 0, st>>>(p, w, n, d);
  return cudaGetLastError();
}

}  // namespace ei
