// Batched form: phi_1(h_i A_i) v_i for many independent 2D stencil problems
// of uneven size in one persistent kernel launch (sm_103a).
//
// Each problem i runs the same method as the single-problem path (Gershgorin
// interval, a-priori substeps s_i, Newton form at Leja points with the stop
// test |d_{j+1}| ||w_{j+1}|| <= tol ||p_{j+1}||; Sec. II-C, Eq. (3), Sec. III-C
// of the paper) and proceeds through phases, each a sweep over its tiles:
//   NEWTON(j): w_{j+1} = (A w_j)/gamma - (c/gamma + xi_j) w_j, p += d_{j+1} w_{j+1}
//   AXPY:      y += tau p          (substeps s > 1)
//   RES:       r = A y + v         (start of substeps 2..s)
// Work distribution: the unit of work is a strip, 32 columns x `rows` rows of
// one problem, processed by one warp; no block-level synchronisation.
// - Claim queue: one 64-bit word per problem, descriptor << 32 | next strip,
//   where the descriptor names the current epoch (phase, Newton index j,
//   substep).  Queue order puts the longest expected chains of epochs first
//   (critical path first; then the bigger problem).
// - Availability bitmap: a bit per queue position whose epoch has unclaimed
//   strips, set when an epoch is published and cleared by the claimer of its
//   last strip.  A warp looking for work reads it (one L2 round trip per 1024
//   problems) and claims from the front of the queue, so the long chains start
//   at once instead of forming a tail.
// - Claims: one atomicAdd returns the strip and its epoch at once.  Outside
//   the first 32 queue positions the next strip of the same epoch is claimed
//   before the current one's arithmetic (the epoch cannot close while the warp
//   holds an unfinished strip), so the claim's latency hides behind the strip;
//   at the front, where the chains of epochs are longest, a held-back strip
//   would delay its epoch by a whole strip, so each strip goes to a free warp.
// - Epochs: after a strip the warp writes its norm partials and counts it
//   done; the warp that completes the last strip of an epoch sums the partials
//   in strip order (deterministic), takes the phase's decision and publishes
//   the next epoch.
// No warp waits for another; a warp that finds nothing to claim sleeps
// briefly, and gives up after 5 s (ei_batch_set_wait_limit) without global
// progress (status EI_ERR_TIMEOUT; the export then writes nothing).  Data written by other warps in earlier epochs is read
// through L2 (ld.global.cg).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ei.h"
#include "ei_device.cuh"

namespace ei {
const double* leja_table();
void divided_differences(int k, double tau, double c, double gamma, int m, double* out);
int schedule(int k, double h, double c, double gamma, double tol, int m_max, int* s_out,
             int* m_out, double* d_out);
double phi_scalar(int k, double z);

enum { PH_NEWTON = 0, PH_AXPY = 1, PH_RES = 2 };
enum { ST_RUN = 0, ST_DONE = 1, ST_FAIL = 2, ST_NONFINITE = 3, ST_SCALAR = 4, ST_SKIP = 5 };

struct BInst {
  int nx, ny, tiles_x, tiles, rows;  // tiles: strips of 32 columns x rows rows
  int bc[4];
  int s;
  int pos;                           // position in the claim queue
  double d0, axm, axp, aym, ayp;     // interior coefficients (ghost form)
  double inv_gamma, c_over_gamma, tau, h;
  int64_t off;                       // element offset of the problem's block of vectors
  int64_t npts;
  int64_t poff;                      // offset of the tile partials
  int dd_off;                        // offset of the divided differences
};

struct BState {
  unsigned int done;        // tiles completed in the current epoch
  int status, degree_sum, pad;
};

// Epoch descriptor (high half of a claim word): Newton index j in bits 0-6
// (j < m_max <= 100), phase in bits 7-8, substep in bits 9-30 (s <= 2^20).
__host__ __device__ __forceinline__ unsigned make_desc(int phase, int j, int sub) {
  return (unsigned)j | ((unsigned)phase << 7) | ((unsigned)sub << 9);
}
__device__ __forceinline__ int desc_j(unsigned d) { return (int)(d & 127u); }
__device__ __forceinline__ int desc_phase(unsigned d) { return (int)((d >> 7) & 3u); }
__device__ __forceinline__ int desc_sub(unsigned d) { return (int)(d >> 9); }
// low half of the word of a problem that is not running: above any tile count
constexpr unsigned long long IDLE_WORD = 0x40000000ull;

struct BatchDev {
  int count;
  int m_max;
  double tol;
  const BInst* inst;
  BState* state;
  unsigned long long* qword;  // claim word per queue position
  const int* qtiles;          // tile count per queue position
  unsigned* avail;            // bit k: position k's epoch has unclaimed strips
  int nwords;                 // words of the bitmap
  const int* order;           // problem at each queue position
  const double* dd;
  const double* xi;
  double* partials;
  void* pool;                // 5 vectors per problem: v, w0, w1, y, r
  void* ppool;               // Newton sum per problem
  unsigned int* finished;
  unsigned long long* progress;
  int* error;
  unsigned long long idle_limit_ns;  // an idle warp's no-progress limit
};

template <class T>
__device__ __forceinline__ T ldcg_(const T* p, int64_t i);
template <> __device__ __forceinline__ df ldcg_<df>(const df* p, int64_t i) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p) + i);
  return df{v.x, v.y};
}
template <> __device__ __forceinline__ double ldcg_<double>(const double* p, int64_t i) {
  return __ldcg(p + i);
}
template <> __device__ __forceinline__ float ldcg_<float>(const float* p, int64_t i) {
  return __ldcg(p + i);
}

// 5-point sum dg*uc + sum_k a_k*u_k.  Float-float: two lazily normalised
// accumulators (independent chains); double/float: two FMA chains.
__device__ __forceinline__ df stencil5(df dg, df uc, df a0, df u0, df a1, df u1, df a2, df u2,
                                       df a3, df u3) {
  dfacc s1 = dfa_mul(dg, uc);
  dfacc s2 = dfa_mul(a2, u2);
  s1 = dfa_mac(s1, a0, u0);
  s2 = dfa_mac(s2, a3, u3);
  s1 = dfa_mac(s1, a1, u1);
  return dfa_norm(dfa_add(s1, s2));
}
template <class R>
__device__ __forceinline__ R stencil5(R dg, R uc, R a0, R u0, R a1, R u1, R a2, R u2, R a3,
                                      R u3) {
  R s1 = dg * uc, s2 = a2 * u2;
  s1 = fma(a0, u0, s1);
  s2 = fma(a3, u3, s2);
  s1 = fma(a1, u1, s1);
  return s1 + s2;
}

// a lane's value from the lane below / above (lane 0 / 31 get their own)
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_down1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_down1(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ df shfl_up1(df v) {
  return df{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}
__device__ __forceinline__ df shfl_down1(df v) {
  return df{__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1)};
}
// a vector value carried in the Newton sum's type, back to the vector type
__device__ __forceinline__ float narrow_to(df a, float) { return a.hi; }
__device__ __forceinline__ df narrow_to(df a, df) { return a; }
__device__ __forceinline__ double narrow_to(double a, double) { return a; }

// One strip: 32 columns x `rows` rows.  Lane = column; the warp marches down
// the strip keeping u(y-1), u(y), u(y+1) of its column in registers and takes
// u(x-1), u(x+1) from the adjacent lanes, so a point costs one load of u plus
// its Newton sum (and the two edge lanes one halo value); the loads of a row
// are issued three rows ahead of its arithmetic.  A ghost value is 0 behind a Dirichlet face and u itself behind
// a Neumann face.
template <int FMT>
__device__ void batch_tile(const BatchDev& B, int i, int t, int phase, int j, int sub,
                           double& o0, double& o1) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  const BInst& I = B.inst[i];
  T* __restrict__ base = static_cast<T*>(B.pool) + I.off;
  const T* V = base;
  T* W0 = base + I.npts;
  T* W1 = base + 2 * I.npts;
  T* Y = base + 3 * I.npts;
  T* R = base + 4 * I.npts;
  P* __restrict__ Pp = static_cast<P*>(B.ppool) + I.off / 5;
  const int x = (t % I.tiles_x) * 32 + (int)(threadIdx.x & 31);
  const int y0 = (t / I.tiles_x) * I.rows;
  const int y1 = min(y0 + I.rows, I.ny);
  typename Acc<T>::type aw = Acc<T>::zero();
  typename Acc<P>::type ap = Acc<P>::zero();
  if (phase == PH_AXPY) {
    const P tau = from_d<P>(I.tau);
    if (x < I.nx)
      for (int y = y0; y < y1; ++y) {
        const int64_t k = (int64_t)y * I.nx + x;
        const P yo = (sub == 0) ? zero<P>() : to_p(ldcg_(Y, k));
        const P yn = mac(yo, tau, ldcg_(Pp, k));
        if constexpr (FMT == VF_F32) {
          st(Y, k, (float)to_d(yn));
        } else {
          st(Y, k, yn);
        }
      }
    o0 = 0.0;
    o1 = 0.0;
    return;
  }
  const T* __restrict__ u = (phase == PH_RES) ? Y : ((j == 0) ? (sub == 0 ? V : R) : ((j - 1) & 1 ? W1 : W0));
  T* wout = (j & 1) ? W1 : W0;
  // NEWTON: w' = (A u)/gamma - (c/gamma + xi_j) u as one 5-point sum with
  // coefficients a/gamma and centre d0/gamma - c/gamma - xi_j (formed in
  // double); RES: A y with the plain coefficients
  const bool newton = (phase == PH_NEWTON);
  const double sg = newton ? I.inv_gamma : 1.0;
  const T cdg = from_d<T>(newton ? I.d0 * sg - I.c_over_gamma - B.xi[j] : I.d0);
  const T axm = from_d<T>(I.axm * sg), axp = from_d<T>(I.axp * sg);
  const T aym = from_d<T>(I.aym * sg), ayp = from_d<T>(I.ayp * sg);
  const P dn = from_d<P>(phase == PH_NEWTON ? B.dd[I.dd_off + j + 1] : 0.0);
  const P dz = from_d<P>(phase == PH_NEWTON ? B.dd[I.dd_off] : 0.0);
  const T zro = zero<T>();
  if (y0 < y1) {  // the whole warp takes part (lane shuffles)
    const int lane = (int)(threadIdx.x & 31);
    const int nx = I.nx, ny = I.ny;
    const bool g0 = I.bc[0], g1 = I.bc[1], g2 = I.bc[2], g3 = I.bc[3];
    const bool xin = x < nx;
    const bool needp = newton && j > 0;
    const bool needa = needp || !newton;
    // lane 0 holds u(x0-1) and lane 31 u(x0+32) of each row (the strip's halo);
    // the other horizontal neighbours come from the adjacent lanes
    const int hx = lane == 0 ? x - 1 : x + 1;
    const bool hld = (lane == 0 && x > 0) || (lane == 31 && x + 1 < nx);
    // raw loads of a row: the centre u, the halo value, and the row's Newton
    // sum (NEWTON, j > 0) or v (RES) widened to the sum's type.  `ok`: the row
    // lies in the grid.  `ro` is the element offset of row y, advanced by nx.
    int64_t ro = (int64_t)y0 * nx;
    const int ylast = ny - 1;
    auto ldrow = [&](int yy, int64_t off, T& c, T& h, P& a) {
      const bool in = yy <= ylast;
      const int64_t kk = ro + off;
      c = (in && xin) ? ldcg_(u, kk + x) : zro;
      h = (in && hld) ? ldcg_(u, kk + hx) : zro;
      a = zero<P>();
      if (in && xin && needa) a = needp ? ldcg_(Pp, kk + x) : to_p(ldcg_(V, kk + x));
    };
    // queue: row y (uc, hc, ac), rows y+1 and y+2 in flight; the loads of row
    // y+3 are issued before row y's arithmetic (the centre of a row is used one
    // row early, as the point above)
    T uc, hc, c1, h1, c2, h2;
    P ac, a1, a2;
    ldrow(y0, 0, uc, hc, ac);
    T um = (y0 > 0 && xin) ? ldcg_(u, ro - nx + x) : zro;
    ldrow(y0 + 1, nx, c1, h1, a1);
    ldrow(y0 + 2, 2 * (int64_t)nx, c2, h2, a2);
    if (y0 == 0) um = g2 ? uc : zro;
    const int64_t off3 = 3 * (int64_t)nx;
    for (int y = y0; y < y1; ++y) {
      T c3 = zro, h3 = zro;
      P a3 = zero<P>();
      if (y + 3 <= y1) ldrow(y + 3, off3, c3, h3, a3);
      const T up = (y < ylast) ? c1 : (g3 ? uc : zro);
      const T sl = shfl_up1(uc), sr = shfl_down1(uc);
      const T ul = x > 0 ? (lane == 0 ? hc : sl) : (g0 ? uc : zro);
      const T ur = x < nx - 1 ? (lane == 31 ? hc : sr) : (g1 ? uc : zro);
      const T acc = stencil5(cdg, uc, axm, ul, axp, ur, aym, um, ayp, up);
      if (xin) {
        if (newton) {
          const T wn = acc;
          const P pold = (j == 0) ? mul(dz, to_p(uc)) : ac;
          const P pn = mac(pold, dn, to_p(wn));
          st(wout, ro + x, wn);
          st(Pp, ro + x, pn);
          aw = acc_sq(aw, wn);
          ap = acc_sq(ap, pn);
        } else {
          st(R, ro + x, add(acc, narrow_to(ac, zro)));
        }
      }
      ro += nx;
      um = uc;
      uc = c1;
      hc = h1;
      ac = a1;
      c1 = c2;
      h1 = h2;
      a1 = a2;
      c2 = c3;
      h2 = h3;
      a2 = a3;
    }
  }
  o0 = acc_d(aw);
  o1 = acc_d(ap);
}

// Atomic adds with acquire / acquire-release semantics at GPU scope: a claim
// must see the data of the epoch it claims (acquire only: the warp's own
// earlier stores need not drain first); counting a strip done releases the
// strip's stores and, for the warp that completes the epoch, acquires the
// other warps' partials.
__device__ __forceinline__ unsigned long long atom_add_acquire(unsigned long long* p,
                                                               unsigned long long v) {
  unsigned long long r;
  asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned r;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}

// After a claim that returned strip t of position k: the claimer of the last
// strip clears the position's bit (it holds an unfinished strip of the epoch,
// so the epoch cannot be closed and republished before the clear).
__device__ __forceinline__ void claimed_strip(const BatchDev& B, int k, unsigned t,
                                              unsigned tiles) {
  if (t == tiles - 1) atomicAnd(B.avail + (k >> 5), ~(1u << (k & 31)));
}

// A claim at position k found its epoch exhausted while the bit was set: clear
// the bit, then look at the word again and set the bit back if an epoch with
// unclaimed strips was published meanwhile.  The publisher writes the word,
// fences and sets the bit; this side clears, fences and reads the word; with
// both fences either the read sees the new word or the set follows the clear,
// so a published epoch never loses its bit.
__device__ __forceinline__ void stale_bit(const BatchDev& B, int k, unsigned tiles) {
  atomicAnd(B.avail + (k >> 5), ~(1u << (k & 31)));
  __threadfence();
  const unsigned long long w = *(volatile const unsigned long long*)(B.qword + k);
  if ((unsigned)(w & 0xffffffffull) < tiles) atomicOr(B.avail + (k >> 5), 1u << (k & 31));
}

// Claim one strip: the lanes read 32 bitmap words (1024 positions) at a time;
// the first word with set bits holds the front-most problems with unclaimed
// strips.  The warp tries its set bits with one atomicAdd each, starting at a
// bit chosen by the warp index to spread warps over those problems.  Returns
// the queue position (-1: nothing claimable) in every lane, with the strip and
// the epoch descriptor.
__device__ int warp_claim(const BatchDev& B, unsigned gw, int& t_out, unsigned& desc_out) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < B.nwords; base += 32) {
    const int wi = base + lane;
    const unsigned m = wi < B.nwords ? *(volatile const unsigned*)(B.avail + wi) : 0u;
    unsigned lanes = __ballot_sync(0xffffffffu, m != 0u);
    while (lanes) {
      const int l = __ffs(lanes) - 1;
      lanes &= lanes - 1;
      const unsigned bits = __shfl_sync(0xffffffffu, m, l);
      const int nb = __popc(bits);
      for (int r = 0; r < nb; ++r) {
        // the ((gw + r) mod nb)-th set bit
        unsigned rest = bits;
        for (int q = (int)((gw + (unsigned)r) % (unsigned)nb); q > 0; --q) rest &= rest - 1;
        const int k = (base + l) * 32 + __ffs(rest) - 1;
        unsigned long long w = 0;
        if (lane == 0) w = atom_add_acquire(B.qword + k, 1ull);
        w = __shfl_sync(0xffffffffu, w, 0);
        const unsigned t = (unsigned)(w & 0xffffffffull);
        const unsigned tiles = (unsigned)__ldg(B.qtiles + k);
        if (t < tiles) {
          if (lane == 0) claimed_strip(B, k, t, tiles);
          __syncwarp();  // the lanes read the epoch's data after lane 0's acquire
          t_out = (int)t;
          desc_out = (unsigned)(w >> 32);
          return k;
        }
        if (lane == 0) stale_bit(B, k, tiles);
      }
    }
  }
  return -1;
}

// Count a strip of problem i (epoch descriptor d) done; called by the whole
// warp after its stores of the strip.  The warp that completes the epoch sums
// the strip partials (lane-strided, then a fixed shuffle tree), decides and
// publishes the next epoch.
__device__ void account_strip(const BatchDev& B, int i, unsigned d) {
  const int lane = threadIdx.x & 31;
  const BInst& I = B.inst[i];
  BState* S = &B.state[i];
  int last = 0;
  __syncwarp();  // the lanes' stores of the strip precede lane 0's release
  if (lane == 0) {
    const unsigned dn = atom_add_acq_rel(&S->done, 1u);
    last = (dn == (unsigned)I.tiles - 1);
    atomicAdd(B.progress, 1ull);
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __syncwarp();  // the lanes read the partials after lane 0's acquire
  const int phase0 = desc_phase(d), j0 = desc_j(d), sub0 = desc_sub(d);
  double nw2 = 0.0, np2 = 0.0;
  if (phase0 == PH_NEWTON) {
    for (int t = lane; t < I.tiles; t += 32) {
      nw2 += __ldcg(B.partials + I.poff + 2 * t);
      np2 += __ldcg(B.partials + I.poff + 2 * t + 1);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      nw2 += __shfl_xor_sync(0xffffffffu, nw2, off);
      np2 += __shfl_xor_sync(0xffffffffu, np2, off);
    }
  }
  if (lane != 0) return;
  int phase = phase0, j = j0, sub = sub0, status = ST_RUN;
  if (phase0 == PH_NEWTON) {
    const double dn = B.dd[I.dd_off + j + 1];
    int deg = -1;
    if (!isfinite(nw2) || !isfinite(np2)) status = ST_NONFINITE;
    else if (j == 0 && np2 == 0.0) deg = 0;
    else if (fabs(dn) * sqrt(nw2) <= B.tol * sqrt(np2)) deg = j + 1;
    else if (j + 1 >= B.m_max) status = ST_FAIL;
    else j = j + 1;
    if (deg >= 0) {
      volatile int* ds = &S->degree_sum;
      *ds = *ds + deg;
      if (I.s == 1) status = ST_DONE;
      else phase = PH_AXPY;
    }
  } else if (phase0 == PH_AXPY) {
    sub = sub + 1;
    if (sub >= I.s) status = ST_DONE;
    else phase = PH_RES;
  } else {
    phase = PH_NEWTON;
    j = 0;
  }
  *(volatile unsigned*)&S->done = 0u;
  if (status != ST_RUN) {
    *(volatile int*)&S->status = status;
    __threadfence();
    atomicExch(B.qword + I.pos, IDLE_WORD);
    atomicAdd(B.finished, 1u);
  } else {
    __threadfence();
    atomicExch(B.qword + I.pos, (unsigned long long)make_desc(phase, j, sub) << 32);
    __threadfence();
    atomicOr(B.avail + (I.pos >> 5), 1u << (I.pos & 31));
  }
}

// Every warp is an independent worker: claim a strip, process it, count it
// done.  Up to 7 blocks of 4 warps per SM for FP32, 5 for the 8-byte formats
// (register budget).
constexpr int BATCH_THREADS = 128;
template <int FMT>
__global__ void __launch_bounds__(BATCH_THREADS, FMT == VF_F32 ? 7 : 5) k_batch(BatchDev B) {
  const int lane = threadIdx.x & 31;
  const unsigned gw = blockIdx.x * (BATCH_THREADS / 32) + (threadIdx.x >> 5);
  unsigned long long seen = 0;
  uint64_t idle_t0 = 0;
  int k = -1, t = 0;
  unsigned d = 0;
  while (true) {
    if (k < 0) k = warp_claim(B, gw, t, d);
    if (k < 0) {
      // nothing claimable: finished, failed, or waiting for another warp's
      // epoch; give up after B.idle_limit_ns without progress anywhere
      int ex = 0;
      if (lane == 0) {
        if (*(volatile unsigned*)B.finished >= (unsigned)B.count || *(volatile int*)B.error) {
          ex = 1;
        } else {
          const unsigned long long pr = *(volatile unsigned long long*)B.progress;
          uint64_t now;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
          if (pr != seen || idle_t0 == 0) {
            seen = pr;
            idle_t0 = now;
          } else if (now - idle_t0 > B.idle_limit_ns) {
            atomicExch(B.error, 1);
          }
          __nanosleep(256);
        }
      }
      if (__shfl_sync(0xffffffffu, ex, 0)) break;
      continue;
    }
    idle_t0 = 0;
    const int i = __ldg(B.order + k);
    // the next strip of this epoch, claimed ahead; not for the front of the
    // queue (the longest chains), whose epochs end sooner when each of their
    // strips goes to a warp that is free now
    const bool ahead = k >= 32;
    unsigned long long wn = IDLE_WORD;
    if (lane == 0 && ahead) wn = atomicAdd(B.qword + k, 1ull);
    const int phase = desc_phase(d);
    double a = 0.0, b = 0.0;
    batch_tile<FMT>(B, i, t, phase, desc_j(d), desc_sub(d), a, b);
    if (phase == PH_NEWTON) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
      }
      if (lane == 0) {
        B.partials[B.inst[i].poff + 2 * t] = a;
        B.partials[B.inst[i].poff + 2 * t + 1] = b;
      }
    }
    account_strip(B, i, d);
    wn = __shfl_sync(0xffffffffu, wn, 0);
    const unsigned tn = (unsigned)(wn & 0xffffffffull);
    const unsigned tiles = (unsigned)__ldg(B.qtiles + k);
    if (tn < tiles) {
      if (lane == 0) claimed_strip(B, k, tn, tiles);
      t = (int)tn;
      d = (unsigned)(wn >> 32);
    } else {
      k = -1;
    }
  }
}

// ---- set-up, import/export ---------------------------------------------------
__global__ void k_batch_init(const int* order, BState* state, unsigned long long* qword,
                             unsigned* avail, const int* init_status, int count,
                             unsigned int* finished, unsigned long long* progress, int* error) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // a warp covers one bitmap word
  if (k == 0) {
    *finished = 0;
    *progress = 0;
    *error = 0;
  }
  bool run = false;
  if (k < count) {
    const int i = order[k];
    BState s;
    s.done = 0;
    s.status = init_status[i];
    s.degree_sum = 0;
    s.pad = 0;
    state[i] = s;
    run = s.status == ST_RUN;
    // the first epoch of a running problem: Newton, j = 0, substep 0
    qword[k] = run ? ((unsigned long long)make_desc(PH_NEWTON, 0, 0) << 32) : IDLE_WORD;
  }
  const unsigned bits = __ballot_sync(0xffffffffu, run);
  if ((threadIdx.x & 31) == 0 && k < count) avail[k >> 5] = bits;
}

// count the problems that start finished (inactive / scalar)
__global__ void k_batch_count_idle(const BState* state, int count, unsigned int* finished) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && state[i].status != ST_RUN) atomicAdd(finished, 1u);
}

template <int FMT, class U>
__global__ void k_batch_import(const BInst* inst, const int64_t* uoff, const U* v, void* pool) {
  using T = typename VT<FMT>::T;
  const BInst& I = inst[blockIdx.y];
  T* V = static_cast<T*>(pool) + I.off;
  const U* src = v + uoff[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < I.npts;
       k += (int64_t)gridDim.x * blockDim.x)
    st(V, k, from_d<T>((double)src[k]));
}

// out = phi_1(hA) v: p (s = 1), y/h (s > 1), or scale * v (scalar problems);
// nothing when the pass gave up (error set)
template <int FMT, class U>
__global__ void k_batch_export(const BInst* inst, const BState* state, const int64_t* uoff,
                               const double* scal, const void* pool, const void* ppool,
                               U* out, const int* error) {
  using T = typename VT<FMT>::T;
  using P = typename VT<FMT>::P;
  if (*(volatile const int*)error) return;
  const int i = blockIdx.y;
  const BInst& I = inst[i];
  const T* base = static_cast<const T*>(pool) + I.off;
  const P* Pp = static_cast<const P*>(ppool) + I.off / 5;
  U* dst = out + uoff[i];
  const int st_ = state[i].status;
  if (st_ == ST_SKIP || st_ == ST_FAIL || st_ == ST_NONFINITE) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < I.npts;
       k += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (st_ == ST_SCALAR) v = scal[i] * to_d(base[k]);
    else if (I.s == 1) v = to_d(Pp[k]);
    else v = to_d(base[3 * I.npts + k]) / I.h;
    dst[k] = (U)v;
  }
}

}  // namespace ei

// ===========================================================================
// host side
// ===========================================================================
using namespace ei;

struct ei_batch {
  int device = 0, prec = 0, fmt = 0, count = 0, m_max = 100;
  double tol = 0;
  cudaStream_t stream = nullptr;  // library stream the graph is captured on
  std::vector<ei_batch_problem> prob;
  std::vector<BInst> hinst;
  std::vector<int64_t> uoff;      // packed caller layout offsets (count + 1)
  std::vector<int> active;        // 0: scalar problem (A = cI)
  std::vector<int> init;          // initial status of each problem in the next run
  std::vector<int> final_deg;     // degree sum of the accepted attempt
  std::vector<double> scal;       // phi_1(h c) for scalar problems
  std::vector<double> alpha, beta, c, gamma;
  std::vector<int> restarts;
  std::vector<double> hdd;
  // device
  BInst* inst = nullptr;
  BState* state = nullptr;
  unsigned long long* qword = nullptr;
  int* qtiles = nullptr;
  unsigned* avail = nullptr;
  int* order = nullptr;
  int* dinit = nullptr;
  int64_t* duoff = nullptr;
  double* dscal = nullptr;
  double* dd = nullptr;
  double* xi = nullptr;
  double* partials = nullptr;
  void* pool = nullptr;
  void* ppool = nullptr;
  unsigned int* finished = nullptr;
  unsigned long long* progress = nullptr;
  int* error = nullptr;
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  unsigned long long idle_limit_ns = 5000000000ull;  // ei_batch_set_wait_limit
  const void* graph_v = nullptr;
  void* graph_out = nullptr;
  int64_t parts_cap = 0;           // partials allocated (doubles)
  // learned schedule
  const ei_mlp* model = nullptr;
  bool deferred = false;           // plain plans not made yet (created with learned = 1)
  std::vector<int> dd_s;           // the s whose divided differences hdd holds (0: none)
  std::vector<int> plain_s;        // the a-priori rule's s (0: not computed)
  std::vector<int> plain_m;        // and its degree estimate
  std::vector<int> est_m;          // expected degree per substep of the current plan
  std::vector<int> learned;        // 0 plain plan, 1 learned proposal kept, 2 fell back
  double* vn2 = nullptr;           // device: ||v_i||^2
  std::vector<double> hvn2;
};

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;  // (device, format, size class) -> rows

static int size_class(int64_t npts) {
  if (npts < 64 * 64) return 0;
  if (npts < 128 * 128) return 1;
  if (npts < 256 * 256) return 2;
  return 3;
}

// Gershgorin row of the constant-coefficient 2D operator at a point class:
// the same rule as the stencil rows (neighbour inside: a = D/dx^2 +- b/(2dx),
// diag -= D/dx^2; Dirichlet face: diag -= D/dx^2; Neumann face: diag += +-b/(2dx))
static void batch_row(const ei_batch_problem& P, bool xl, bool xh, bool yl, bool yh, double* dg,
                      double* rad) {
  double d = P.c, r = 0.0;
  const bool has[4] = {!xl, !xh, !yl, !yh};
  const double h2[2] = {P.dx * P.dx, P.dy * P.dy};
  const double hh[2] = {P.dx, P.dy};
  const double b[2] = {P.bx, P.by};
  for (int e = 0; e < 2; ++e)
    for (int side = 0; side < 2; ++side) {
      const int sgn = side ? 1 : -1;
      const int f = 2 * e + side;
      if (has[f]) {
        const double a = P.D / h2[e] + sgn * b[e] / (2.0 * hh[e]);
        r += fabs(a);
        d -= P.D / h2[e];
      } else if (P.bc[f] == EI_BC_NEUMANN0) {
        d += sgn * b[e] / (2.0 * hh[e]);
      } else {
        d -= P.D / h2[e];
      }
    }
  *dg = d;
  *rad = r;
}

static void batch_interval(const ei_batch_problem& P, double* alpha, double* beta) {
  double lo = INFINITY, hi = -INFINITY;
  // classes along x: x=0 (lo), interior, x=nx-1 (hi); nx == 1: both faces
  for (int cx = 0; cx < 3; ++cx)
    for (int cy = 0; cy < 3; ++cy) {
      bool xl, xh, yl, yh;
      if (P.nx == 1) { xl = xh = true; if (cx) continue; }
      else if (P.nx == 2) { if (cx == 1) continue; xl = cx == 0; xh = cx == 2; }
      else { xl = cx == 0; xh = cx == 2; }
      if (P.ny == 1) { yl = yh = true; if (cy) continue; }
      else if (P.ny == 2) { if (cy == 1) continue; yl = cy == 0; yh = cy == 2; }
      else { yl = cy == 0; yh = cy == 2; }
      double d, r;
      batch_row(P, xl, xh, yl, yh, &d, &r);
      lo = std::min(lo, d - r);
      hi = std::max(hi, d + r);
    }
  *alpha = lo;
  *beta = hi;
}

// schedule and divided differences of problem i for its current s (s <= 0:
// a-priori rule); m_hint > 0 is the degree the plan expects per substep (the
// a-priori rule gives its own), used to order the claim queue
static bool batch_plan(ei_batch* B, int i, int s_force, int m_hint = 0) {
  const double cc = B->c[i], gm = B->gamma[i];
  const double h = B->prob[i].h;
  int s = s_force, m = 0;
  double* d = &B->hdd[(size_t)i * (B->m_max + 1)];
  if (s <= 0) {
    if (schedule(1, h, cc, gm, B->tol, B->m_max, &s, &m, d) != 0) return false;
    B->plain_s[i] = s;
    B->plain_m[i] = m;
    B->est_m[i] = m;
  } else {
    if (B->dd_s[i] != s) divided_differences(1, h / s, cc, gm, B->m_max, d);
    B->est_m[i] = m_hint > 0 ? m_hint
                             : (s == B->plain_s[i] && B->plain_m[i] > 0 ? B->plain_m[i] : B->m_max / 2);
  }
  B->dd_s[i] = s;
  B->hinst[i].s = s;
  B->hinst[i].tau = h / s;
  return true;
}

static void parallel_for(int n, const std::function<void(int)>& f) {
  int nt = (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  if (nt > n) nt = n;
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

static void batch_free(ei_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  void* ptrs[] = {B->inst, B->state, B->qword, B->qtiles, B->avail, B->order, B->dinit, B->duoff, B->dscal, B->dd, B->xi,
                  B->partials, B->pool, B->ppool, B->finished, B->progress, B->error, B->vn2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (B->stream) cudaStreamDestroy(B->stream);
}

#define BTRY(x)                        \
  do {                                 \
    if ((x) != cudaSuccess) {          \
      cudaGetLastError();              \
      return EI_ERR_CUDA;              \
    }                                  \
  } while (0)

template <int FMT>
static cudaError_t batch_launch_body(ei_batch* B) {
  const int count = B->count;
  BatchDev D;
  D.count = count;
  D.m_max = B->m_max;
  D.tol = B->tol;
  D.inst = B->inst;
  D.state = B->state;
  D.qword = B->qword;
  D.qtiles = B->qtiles;
  D.avail = B->avail;
  D.nwords = (count + 31) / 32;
  D.order = B->order;
  D.dd = B->dd;
  D.xi = B->xi;
  D.partials = B->partials;
  D.pool = B->pool;
  D.ppool = B->ppool;
  D.finished = B->finished;
  D.progress = B->progress;
  D.error = B->error;
  D.idle_limit_ns = B->idle_limit_ns;
  k_batch_init<<<(count + 255) / 256, 256, 0, B->stream>>>(B->order, B->state, B->qword,
                                                           B->avail, B->dinit, count,
                                                           B->finished, B->progress, B->error);
  k_batch_count_idle<<<(count + 255) / 256, 256, 0, B->stream>>>(B->state, count, B->finished);
  k_batch<FMT><<<B->grid, BATCH_THREADS, 0, B->stream>>>(D);
  return cudaGetLastError();
}

template <int FMT, class U>
static cudaError_t batch_io(ei_batch* B, const void* v, void* out, bool import) {
  dim3 g(64, B->count);
  if (import)
    k_batch_import<FMT, U><<<g, 256, 0, B->stream>>>(B->inst, B->duoff, static_cast<const U*>(v),
                                                     B->pool);
  else
    k_batch_export<FMT, U><<<g, 256, 0, B->stream>>>(B->inst, B->state, B->duoff, B->dscal,
                                                     B->pool, B->ppool, static_cast<U*>(out),
                                                     B->error);
  return cudaGetLastError();
}

static cudaError_t batch_sequence(ei_batch* B, const void* v, void* out) {
  cudaError_t e;
  if (B->fmt == VF_DF) {
    if ((e = batch_io<VF_DF, double>(B, v, out, true)) != cudaSuccess) return e;
    if ((e = batch_launch_body<VF_DF>(B)) != cudaSuccess) return e;
    return batch_io<VF_DF, double>(B, v, out, false);
  }
  if (B->fmt == VF_F64) {
    if ((e = batch_io<VF_F64, double>(B, v, out, true)) != cudaSuccess) return e;
    if ((e = batch_launch_body<VF_F64>(B)) != cudaSuccess) return e;
    return batch_io<VF_F64, double>(B, v, out, false);
  }
  if ((e = batch_io<VF_F32, float>(B, v, out, true)) != cudaSuccess) return e;
  if ((e = batch_launch_body<VF_F32>(B)) != cudaSuccess) return e;
  return batch_io<VF_F32, float>(B, v, out, false);
}

static int persistent_grid(int fmt) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (fmt == VF_DF) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<VF_DF>, BATCH_THREADS, 0);
  else if (fmt == VF_F64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<VF_F64>, BATCH_THREADS, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<VF_F32>, BATCH_THREADS, 0);
  if (per < 1) per = 1;
  return sms * per;
}

// upload per-problem tables that depend on the tile choice and the schedule
static ei_status batch_upload(ei_batch* B) {
  const int count = B->count;
  int64_t poff = 0;
  for (int i = 0; i < count; ++i) {
    BInst& I = B->hinst[i];
    I.tiles_x = (I.nx + 31) / 32;
    const int64_t th = I.rows;
    const int64_t tiles = (int64_t)I.tiles_x * ((I.ny + th - 1) / th);
    if (tiles >= (int64_t)IDLE_WORD) return EI_ERR_INVALID_ARG;  // the claim word's range
    I.tiles = (int)tiles;
    I.poff = poff;
    poff += 2 * (int64_t)I.tiles;
  }
  const int64_t need = poff > 0 ? poff : 2;
  if (need > B->parts_cap) {  // the captured graph holds the old pointer
    if (B->partials) cudaFree(B->partials);
    B->partials = nullptr;
    B->parts_cap = 0;
    BTRY(cudaMalloc(&B->partials, sizeof(double) * need));
    B->parts_cap = need;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  // claim queue: longest expected chain of epochs first (critical path first:
  // a problem's epochs run one after the other, its strips in parallel), then
  // the bigger problem
  std::vector<int> ord(count);
  for (int i = 0; i < count; ++i) ord[i] = i;
  std::vector<int64_t> chain(count);
  for (int i = 0; i < count; ++i) {
    const int64_t sv = B->hinst[i].s;
    chain[i] = sv * (B->est_m[i] + 1) + (sv > 1 ? 2 * sv - 1 : 0);
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return chain[a] != chain[b] ? chain[a] > chain[b] : B->hinst[a].npts > B->hinst[b].npts;
  });
  std::vector<int> qt(count);
  for (int k = 0; k < count; ++k) {
    B->hinst[ord[k]].pos = k;
    qt[k] = B->hinst[ord[k]].tiles;
  }
  BTRY(cudaMemcpy(B->inst, B->hinst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(B->dd, B->hdd.data(), sizeof(double) * B->hdd.size(), cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(B->order, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(B->qtiles, qt.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
  return EI_OK;
}

static ei_status batch_run(ei_batch* B, const void* v, void* out, bool graph) {
  if (!graph) {
    BTRY(batch_sequence(B, v, out));
  } else {
    if (!B->exec || B->graph_v != v || B->graph_out != out) {
      if (B->exec) cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
      cudaGraph_t g;
      BTRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = batch_sequence(B, v, out);
      cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return EI_ERR_CUDA;
      }
      BTRY(cudaGraphInstantiate(&B->exec, g, 0));
      cudaGraphDestroy(g);
      B->graph_v = v;
      B->graph_out = out;
    }
    BTRY(cudaGraphLaunch(B->exec, B->stream));
  }
  BTRY(cudaStreamSynchronize(B->stream));
  int err = 0;
  BTRY(cudaMemcpy(&err, B->error, sizeof(int), cudaMemcpyDeviceToHost));
  return err ? EI_ERR_TIMEOUT : EI_OK;
}

// ||v_i||^2 of every problem from the caller's packed v (one block per problem,
// fixed summation order)
template <class U>
__global__ void k_batch_vnorm(const int64_t* uoff, const U* v, int count, double* vn2) {
  const int i = blockIdx.x;
  if (i >= count) return;
  const int64_t a = uoff[i], b = uoff[i + 1];
  double acc = 0.0, zero = 0.0;
  for (int64_t k = a + threadIdx.x; k < b; k += blockDim.x) {
    const double x = (double)v[k];
    acc += x * x;
  }
  block_reduce2<RED_SUM>(acc, zero);
  if (threadIdx.x == 0) vn2[i] = acc;
}

// Plans of this call from the schedule network: per problem the features of
// s = 2^q, q = 0..q_max (constant D: coefficient ratio 1; Peclet number
// max(|b_x| dx, |b_y| dy) / (2 D)), one batched inference, the cheapest
// accepted q; a problem with no accepted q takes the a-priori rule.
static ei_status batch_learned_plan(ei_batch* B, const void* v) {
  const int count = B->count;
  if (!B->vn2) {
    BTRY(cudaMalloc(&B->vn2, sizeof(double) * count));
    B->hvn2.assign(count, 0.0);
  }
  if (B->prec == EI_PREC_F32)
    k_batch_vnorm<float><<<count, 256, 0, B->stream>>>(B->duoff, static_cast<const float*>(v),
                                                       count, B->vn2);
  else
    k_batch_vnorm<double><<<count, 256, 0, B->stream>>>(B->duoff, static_cast<const double*>(v),
                                                        count, B->vn2);
  BTRY(cudaGetLastError());
  BTRY(cudaMemcpyAsync(B->hvn2.data(), B->vn2, sizeof(double) * count, cudaMemcpyDeviceToHost,
                       B->stream));
  BTRY(cudaStreamSynchronize(B->stream));
  const ei_mlp_decision& D = mlp_decision(B->model);
  const int rows = D.q_max + 1;
  std::vector<double> feat((size_t)count * rows * EI_MLP_INPUTS, 0.0);
  for (int i = 0; i < count; ++i) {
    if (!B->active[i]) continue;
    const ei_batch_problem& P = B->prob[i];
    const double pe = std::max(fabs(P.bx) * P.dx, fabs(P.by) * P.dy) / (2.0 * P.D);
    for (int q = 0; q < rows; ++q)
      learned_features(&feat[((size_t)i * rows + q) * EI_MLP_INPUTS], (double)(1 << q), P.h,
                       B->alpha[i], B->beta[i], B->tol, 0, 2, B->hinst[i].npts, 1.0, pe,
                       sqrt(B->hvn2[i]));
  }
  std::vector<float> outs((size_t)count * rows * EI_MLP_OUTPUTS);
  ei_status st = mlp_infer_rows(B->model, feat.data(), (int64_t)count * rows, outs.data());
  if (st != EI_OK) return st;
  std::vector<int> ok(count, 1);
  parallel_for(count, [&](int i) {
    if (!B->active[i]) return;
    int s = 0, m = 0;
    if (learned_decide(&outs[(size_t)i * rows * EI_MLP_OUTPUTS], rows, D, B->m_max, &s, &m)) {
      B->learned[i] = 1;
      ok[i] = batch_plan(B, i, s, m) ? 1 : 0;
    } else {
      B->learned[i] = 0;
      ok[i] = batch_plan(B, i, B->plain_s[i] > 0 ? B->plain_s[i] : 0) ? 1 : 0;
    }
  });
  for (int i = 0; i < count; ++i)
    if (!ok[i]) return EI_ERR_NOT_CONVERGED;
  return batch_upload(B);
}

// autotuner: for each size class present, time the candidate tile heights on a
// mini-batch of copies of the class's median problem; keep the fastest
static ei_status batch_tune(ei_batch* B) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  std::vector<std::vector<int>> members(4);
  for (int i = 0; i < B->count; ++i)
    if (B->active[i]) members[size_class(B->hinst[i].npts)].push_back(i);
  const int cand[4] = {8, 16, 32, 64};
  for (int cls = 0; cls < 4; ++cls) {
    if (members[cls].empty()) continue;
    const std::string key = std::string(prop.name) + "/" + std::to_string(B->fmt) + "/" +
                            std::to_string(cls);
    int rows = 0;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) rows = it->second;
    }
    if (!rows) {
      std::vector<int>& m = members[cls];
      std::sort(m.begin(), m.end(),
                [&](int a, int b) { return B->hinst[a].npts < B->hinst[b].npts; });
      const int rep = m[m.size() / 2];
      // fixed work: copies of the median problem, one substep, 16 Newton
      // iterations each (a tolerance no iteration meets); enough copies that
      // every resident warp could hold a 64-row strip, as in a full batch
      const int64_t target = (int64_t)B->grid * (BATCH_THREADS / 32) * 64 * 32;
      int copies = (int)std::min<int64_t>(
          2048, std::max<int64_t>(4, (target + B->hinst[rep].npts - 1) / B->hinst[rep].npts));
      std::vector<ei_batch_problem> probs(copies, B->prob[rep]);
      float best = 1e30f;
      for (int c : cand) {
        ei_options o{};
        o.tile_rows = c;
        o.fixed_s = 1;
        o.m_max = 16;
        ei_batch* T = nullptr;
        if (ei_batch_create(&T, dev, copies, probs.data(), B->prec, 1e-300, &o) != EI_OK) continue;
        const int64_t total = T->uoff[copies];
        void* buf = nullptr;
        const size_t eb = B->prec == EI_PREC_F32 ? 4 : 8;
        if (cudaMalloc(&buf, 2 * total * eb) == cudaSuccess) {
          std::vector<double> ones(total, 1.0);
          std::vector<float> onesf(total, 1.0f);
          if (eb == 8) cudaMemcpy(buf, ones.data(), total * 8, cudaMemcpyHostToDevice);
          else cudaMemcpy(buf, onesf.data(), total * 4, cudaMemcpyHostToDevice);
          void* outb = static_cast<char*>(buf) + total * eb;
          batch_run(T, buf, outb, false);  // warm
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          cudaEventRecord(e0, T->stream);
          ei_status rs = batch_run(T, buf, outb, false);
          cudaEventRecord(e1, T->stream);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          if (rs == EI_OK && ms < best) {
            best = ms;
            rows = c;
          }
          cudaFree(buf);
        }
        ei_batch_destroy(T);
      }
      if (!rows) rows = 16;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = rows;
    }
    for (int i : members[cls]) B->hinst[i].rows = rows;
  }
  return EI_OK;
}

extern "C" {

ei_status ei_batch_create(ei_batch** out, int device, int count, const ei_batch_problem* problems,
                          int prec, double tol, const ei_options* opt) {
  if (!out || count < 1 || !problems || (prec != EI_PREC_F64 && prec != EI_PREC_F32) ||
      !(tol > 0) || !isfinite(tol))
    return EI_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    const ei_batch_problem& P = problems[i];
    if (P.nx < 1 || P.ny < 1 || P.nx > (1 << 20) || P.ny > (1 << 20) || !(P.dx > 0) ||
        !(P.dy > 0) || !(P.h > 0) || !isfinite(P.D) || !isfinite(P.bx) || !isfinite(P.by) ||
        !isfinite(P.c) || !isfinite(P.h))
      return EI_ERR_INVALID_ARG;
    for (int f = 0; f < 4; ++f)
      if (P.bc[f] != EI_BC_DIRICHLET0 && P.bc[f] != EI_BC_NEUMANN0) return EI_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return EI_ERR_CUDA;
  }
  ei_batch* B = new ei_batch();
  B->device = device;
  B->prec = prec;
  B->fmt = (prec == EI_PREC_F32) ? VF_F32 : ((opt && opt->arith == EI_ARITH_NATIVE_F64) ? VF_F64 : VF_DF);
  B->count = count;
  B->tol = tol;
  B->m_max = (opt && opt->m_max > 0 && opt->m_max <= 100) ? opt->m_max : 100;
  B->prob.assign(problems, problems + count);
  B->hinst.resize(count);
  B->uoff.resize(count + 1);
  B->active.assign(count, 1);
  B->scal.assign(count, 0.0);
  B->alpha.resize(count);
  B->beta.resize(count);
  B->c.resize(count);
  B->gamma.resize(count);
  B->restarts.assign(count, 0);
  B->hdd.assign((size_t)count * (B->m_max + 1), 0.0);
  B->dd_s.assign(count, 0);
  B->plain_s.assign(count, 0);
  B->plain_m.assign(count, 0);
  B->est_m.assign(count, B->m_max / 2);
  B->learned.assign(count, 0);
  B->deferred = opt && opt->learned == 1;
  int64_t uo = 0, po = 0;
  for (int i = 0; i < count; ++i) {
    const ei_batch_problem& P = problems[i];
    BInst& I = B->hinst[i];
    memset(&I, 0, sizeof(I));
    I.nx = (int)P.nx;
    I.ny = (int)P.ny;
    I.npts = P.nx * P.ny;
    for (int f = 0; f < 4; ++f) I.bc[f] = P.bc[f];
    I.axm = P.D / (P.dx * P.dx) - P.bx / (2.0 * P.dx);
    I.axp = P.D / (P.dx * P.dx) + P.bx / (2.0 * P.dx);
    I.aym = P.D / (P.dy * P.dy) - P.by / (2.0 * P.dy);
    I.ayp = P.D / (P.dy * P.dy) + P.by / (2.0 * P.dy);
    I.d0 = P.c - 2.0 * P.D / (P.dx * P.dx) - 2.0 * P.D / (P.dy * P.dy);
    I.h = P.h;
    I.rows = 16;
    B->uoff[i] = uo;
    uo += I.npts;
    I.off = po;
    po += 5 * I.npts;
    batch_interval(P, &B->alpha[i], &B->beta[i]);
    B->c[i] = 0.5 * (B->alpha[i] + B->beta[i]);
    B->gamma[i] = 0.25 * (B->beta[i] - B->alpha[i]);
    I.inv_gamma = B->gamma[i] > 0 ? 1.0 / B->gamma[i] : 0.0;
    I.c_over_gamma = B->gamma[i] > 0 ? B->c[i] / B->gamma[i] : 0.0;
    I.dd_off = i * (B->m_max + 1);
    I.s = 1;
    if (!(B->gamma[i] > 0)) {
      B->active[i] = 0;
      B->scal[i] = phi_scalar(1, P.h * B->c[i]);
    }
  }
  B->uoff[count] = uo;
  // schedules and divided differences, in parallel over problems
  std::vector<int> ok(count, 1);
  const int s_force = (opt && opt->fixed_s > 0) ? opt->fixed_s : 0;
  if (!B->deferred)
    parallel_for(count, [&](int i) {
      if (B->active[i]) ok[i] = batch_plan(B, i, s_force) ? 1 : 0;
    });
  for (int i = 0; i < count; ++i)
    if (!ok[i]) {
      delete B;
      return EI_ERR_NOT_CONVERGED;
    }
  ei_status st = EI_OK;
  auto fail = [&](ei_status s) {
    batch_free(B);
    delete B;
    return s;
  };
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(EI_ERR_CUDA);
  const size_t eb = (B->fmt == VF_F32) ? 4 : 8;
  if (cudaMalloc(&B->pool, eb * po) != cudaSuccess || cudaMalloc(&B->ppool, 8 * (po / 5)) != cudaSuccess ||
      cudaMalloc(&B->inst, sizeof(BInst) * count) != cudaSuccess ||
      cudaMalloc(&B->state, sizeof(BState) * count) != cudaSuccess ||
      cudaMalloc(&B->qword, sizeof(unsigned long long) * count) != cudaSuccess ||
      cudaMalloc(&B->qtiles, sizeof(int) * count) != cudaSuccess ||
      cudaMalloc(&B->avail, sizeof(unsigned) * ((count + 31) / 32)) != cudaSuccess ||
      cudaMalloc(&B->order, sizeof(int) * count) != cudaSuccess ||
      cudaMalloc(&B->dinit, sizeof(int) * count) != cudaSuccess ||
      cudaMalloc(&B->duoff, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&B->dscal, sizeof(double) * count) != cudaSuccess ||
      cudaMalloc(&B->dd, sizeof(double) * B->hdd.size()) != cudaSuccess ||
      cudaMalloc(&B->xi, sizeof(double) * 101) != cudaSuccess ||
      cudaMalloc(&B->finished, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&B->progress, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&B->error, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(EI_ERR_NOMEM);
  }
  cudaMemset(B->pool, 0, eb * po);
  cudaMemset(B->ppool, 0, 8 * (po / 5));
  B->init.resize(count);
  for (int i = 0; i < count; ++i) B->init[i] = B->active[i] ? ST_RUN : ST_SCALAR;
  B->final_deg.assign(count, 0);
  cudaMemcpy(B->dinit, B->init.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(B->duoff, B->uoff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(B->dscal, B->scal.data(), sizeof(double) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(B->xi, leja_table(), sizeof(double) * 101, cudaMemcpyHostToDevice);
  B->grid = persistent_grid(B->fmt);
  if (opt && opt->tile_rows > 1024) return fail(EI_ERR_INVALID_ARG);
  if (opt && opt->tile_rows > 0) {
    for (int i = 0; i < count; ++i) B->hinst[i].rows = opt->tile_rows;
  } else if ((st = batch_tune(B)) != EI_OK) {
    return fail(st);
  }
  if ((st = batch_upload(B)) != EI_OK) return fail(st);
  *out = B;
  return EI_OK;
}

ei_status ei_batch_offsets(const ei_batch* b, int64_t* offsets) {
  if (!b) return EI_ERR_INVALID_ARG;
  if (offsets)
    for (int i = 0; i <= b->count; ++i) offsets[i] = b->uoff[i];
  return EI_OK;
}

ei_status ei_batch_phi1(ei_batch* B, void* cuda_stream, const void* v, void* out,
                        ei_batch_stats* per) {
  if (!B || !v || !out) return EI_ERR_INVALID_ARG;
  if (cudaSetDevice(B->device) != cudaSuccess) return EI_ERR_CUDA;
  // order against the caller's stream: its pending work on v finishes first
  cudaStream_t us = (cudaStream_t)cuda_stream;
  cudaEvent_t ev;
  BTRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  BTRY(cudaEventRecord(ev, us));
  BTRY(cudaStreamWaitEvent(B->stream, ev, 0));
  ei_status rc = EI_OK;
  if (B->model) {
    rc = batch_learned_plan(B, v);
  } else if (B->deferred) {  // created for the learned schedule, used without a model
    std::vector<int> ok(B->count, 1);
    parallel_for(B->count, [&](int i) {
      if (B->active[i]) ok[i] = batch_plan(B, i, 0) ? 1 : 0;
    });
    for (int i = 0; i < B->count; ++i)
      if (!ok[i]) rc = EI_ERR_NOT_CONVERGED;
    if (rc == EI_OK) rc = batch_upload(B);
    B->deferred = false;
  }
  if (rc == EI_OK) rc = batch_run(B, v, out, true);
  // problems that reached m_max: double s and rerun them alone; the others keep
  // their results (status SKIP in the rerun)
  std::vector<BState> hs(B->count);
  while (rc == EI_OK) {
    BTRY(cudaMemcpy(hs.data(), B->state, sizeof(BState) * B->count, cudaMemcpyDeviceToHost));
    std::vector<int> redo;
    for (int i = 0; i < B->count; ++i) {
      if (hs[i].status == ST_NONFINITE) rc = EI_ERR_NONFINITE;
      else if (hs[i].status == ST_FAIL) redo.push_back(i);
      else if (hs[i].status == ST_DONE) B->final_deg[i] = hs[i].degree_sum;
    }
    if (rc != EI_OK || redo.empty()) break;
    std::vector<int> init(B->count, ST_SKIP);
    for (int i : redo) {
      if (B->learned[i] == 1) {  // the proposal reached m_max: the a-priori rule
        B->learned[i] = 2;
        if (!batch_plan(B, i, B->plain_s[i] > 0 ? B->plain_s[i] : 0)) {
          rc = EI_ERR_NOT_CONVERGED;
          break;
        }
      } else {
        const int s2 = 2 * B->hinst[i].s;
        if (s2 > (1 << 20)) {
          rc = EI_ERR_NOT_CONVERGED;
          break;
        }
        batch_plan(B, i, s2);
      }
      B->restarts[i] += 1;
      init[i] = ST_RUN;
    }
    if (rc != EI_OK) break;
    if ((rc = batch_upload(B)) != EI_OK) break;
    BTRY(cudaMemcpy(B->dinit, init.data(), sizeof(int) * B->count, cudaMemcpyHostToDevice));
    cudaError_t e;
    if (B->fmt == VF_DF) e = batch_launch_body<VF_DF>(B);
    else if (B->fmt == VF_F64) e = batch_launch_body<VF_F64>(B);
    else e = batch_launch_body<VF_F32>(B);
    if (e == cudaSuccess) {
      if (B->fmt == VF_DF) e = batch_io<VF_DF, double>(B, v, out, false);
      else if (B->fmt == VF_F64) e = batch_io<VF_F64, double>(B, v, out, false);
      else e = batch_io<VF_F32, float>(B, v, out, false);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    BTRY(cudaMemcpy(B->dinit, B->init.data(), sizeof(int) * B->count, cudaMemcpyHostToDevice));
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = EI_ERR_CUDA;
    } else {
      int err = 0;
      BTRY(cudaMemcpy(&err, B->error, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) rc = EI_ERR_TIMEOUT;
    }
    // the graph holds the old tables: rebuild it at the next call
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  if (per && rc == EI_OK) {
    for (int i = 0; i < B->count; ++i) {
      per[i].alpha = B->alpha[i];
      per[i].beta = B->beta[i];
      per[i].s = B->active[i] ? B->hinst[i].s : 1;
      per[i].degree_sum = B->active[i] ? B->final_deg[i] : 0;
      per[i].restarts = B->restarts[i];
      per[i].tile_rows = B->hinst[i].rows;
      per[i].learned = B->model ? B->learned[i] : 0;
    }
  }
  // the caller's stream waits for the batch
  BTRY(cudaEventRecord(ev, B->stream));
  BTRY(cudaStreamWaitEvent(us, ev, 0));
  cudaEventDestroy(ev);
  return rc;
}

ei_status ei_batch_set_wait_limit(ei_batch* B, int64_t limit_us) {
  if (!B) return EI_ERR_INVALID_ARG;
  B->idle_limit_ns = limit_us > 0 ? (unsigned long long)limit_us * 1000ull : 5000000000ull;
  if (B->exec) cudaGraphExecDestroy(B->exec);  // the graph holds the old limit
  B->exec = nullptr;
  return EI_OK;
}

ei_status ei_batch_set_schedule_model(ei_batch* B, const ei_mlp* model) {
  if (!B) return EI_ERR_INVALID_ARG;
  B->model = model;
  return EI_OK;
}

void ei_batch_destroy(ei_batch* B) {
  if (!B) return;
  cudaSetDevice(B->device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  batch_free(B);
  delete B;
}

}  // extern "C"
