// Host-side pieces of the Leja method: Leja points, divided differences of
// phi_k, and the a-priori substep rule.  FP64 throughout.
//
// Sec. II-C of the paper reduces phi-functions of A to repeated products
// (alpha*A + beta*I)x (Eq. (3)) once a bound of the field of values is known,
// and Sec. III-C names interpolation at Leja points; the details below are
// the standard real-Leja method for an interval [alpha, beta] mapped to
// [-2, 2] (capacity 1): z = c + gamma*xi, c = (alpha+beta)/2,
// gamma = (beta-alpha)/4.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <mutex>
#include <vector>

#include "ei.h"

namespace ei {

static const int kMaxM = 100;
static const double kTieLog = 1e-12;

// ---------------------------------------------------------------------------
// Leja points: xi_0 = 2, xi_j = argmax_{[-2,2]} prod_{i<j}|x - xi_i|, ties to
// the larger x.  Between two consecutive nodes the log-product is concave and
// its derivative g(x) = sum 1/(x - xi_i) decreases from +inf to -inf, so its
// one root is found by a bracketed Newton iteration; outside the outermost
// nodes the product grows towards the interval end.
// ---------------------------------------------------------------------------
static double log_prod(double x, const std::vector<double>& pts) {
  double s = 0.0;
  for (double p : pts) s += log(fabs(x - p));
  return s;
}

static double gap_root(const std::vector<double>& pts, double a, double b) {
  double lo = a, hi = b, x = 0.5 * (a + b);
  for (int it = 0; it < 200; ++it) {
    double g = 0.0, dg = 0.0;
    for (double p : pts) {
      double t = 1.0 / (x - p);
      g += t;
      dg -= t * t;
    }
    if (g > 0.0) lo = x; else hi = x;
    double xn = x - g / dg;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);  // keep inside the bracket
    if (xn == x || hi - lo <= 4e-16 * fabs(x) + 1e-300) { x = xn; break; }
    x = xn;
  }
  return x;
}

static std::vector<double> compute_leja(int m) {
  std::vector<double> pts{2.0};
  for (int j = 1; j <= m; ++j) {
    std::vector<double> srt(pts);
    std::sort(srt.begin(), srt.end());
    std::vector<double> cand;
    if (std::find(pts.begin(), pts.end(), -2.0) == pts.end()) cand.push_back(-2.0);
    for (size_t i = 0; i + 1 < srt.size(); ++i) cand.push_back(gap_root(pts, srt[i], srt[i + 1]));
    double best = -INFINITY;
    std::vector<double> val(cand.size());
    for (size_t i = 0; i < cand.size(); ++i) {
      val[i] = log_prod(cand[i], pts);
      best = std::max(best, val[i]);
    }
    double pick = -INFINITY;
    for (size_t i = 0; i < cand.size(); ++i)
      if (val[i] >= best - kTieLog) pick = std::max(pick, cand[i]);
    pts.push_back(pick);
  }
  return pts;
}

const double* leja_table() {
  static std::vector<double> tab;
  static std::once_flag once;
  std::call_once(once, [] { tab = compute_leja(kMaxM); });
  return tab.data();
}

// ---------------------------------------------------------------------------
// Divided differences by Opitz's theorem.  With the variables ordered
// (k augmentation variables, then xi_0..xi_m), phi_k of the interpolation
// matrix is the first column of exp(N) for the lower bidiagonal
//     N = bidiag(diag = [0 x k, z_0..z_m], subdiag = [1 x k, tau*gamma x m]),
// z_j = tau*c + tau*gamma*xi_j, and d_j = exp(N)[k+j][0].  N is Metzler
// (nonnegative off the diagonal), so exp(N) = e^{-sigma} exp(N + sigma I) with
// N + sigma I >= 0 entrywise: Taylor terms and squarings add only
// nonnegative numbers, which keeps every entry relatively accurate.
// Scaling: entries <= 4 after 2^-q, q >= 5; Taylor degree 64 (all terms are
// nonnegative, so the series has no cancellation; its per-factor truncation
// is negligible for the band offsets that reach the result).
// ---------------------------------------------------------------------------
static void expm_bidiag_col0(int n, const double* dg, const double* sd, double* out) {
  double sigma = 0.0, mx = 0.0;
  for (int i = 0; i < n; ++i) sigma = std::max(sigma, -dg[i]);
  for (int i = 0; i < n; ++i) mx = std::max(mx, dg[i] + sigma);
  for (int i = 0; i + 1 < n; ++i) mx = std::max(mx, sd[i]);
  int q = 5;
  while (ldexp(4.0, q) < mx) ++q;  // entries of X at most 4
  const double sc = ldexp(1.0, -q);
  std::vector<double> xd(n), xs(n > 1 ? n - 1 : 1);
  for (int i = 0; i < n; ++i) xd[i] = (dg[i] + sigma) * sc;
  for (int i = 0; i + 1 < n; ++i) xs[i] = sd[i] * sc;
  // T = sum_{i<=K} X^i/i!  (Horner), X lower bidiagonal, T dense lower triangular
  const int K = 64;
  std::vector<double> T((size_t)n * n, 0.0), U((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) T[(size_t)i * n + i] = 1.0;
  // After i Horner steps T - I has band width i (X is bidiagonal), so row r
  // only needs columns c >= r - i; the rest of the lower triangle is still 0.
  for (int it = K; it >= 1; --it) {
    const double inv = 1.0 / it;
    const int band = K - it + 1;
    // U = I + (X T)/it ;  (X T)[r][c] = xd[r] T[r][c] + xs[r-1] T[r-1][c]
    U[0] = xd[0] * T[0] * inv + 1.0;
    for (int r = 1; r < n; ++r) {
      double* __restrict__ Ur = &U[(size_t)r * n];
      const double* __restrict__ Tr = &T[(size_t)r * n];
      const double* __restrict__ Tm = &T[(size_t)(r - 1) * n];
      const double a = xd[r], b = xs[r - 1];
      const int c0 = r - band > 0 ? r - band : 0;
      for (int c = c0; c < r; ++c) Ur[c] = (a * Tr[c] + b * Tm[c]) * inv;
      Ur[r] = a * Tr[r] * inv + 1.0;
    }
    std::swap(T, U);
  }
  const double es = exp(-sigma * sc);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c <= r; ++c) T[(size_t)r * n + c] *= es;
  // exp(N) e_0 = T^(2^q) e_0.  Square T `sq` times (n^3/6 multiply-adds
  // each), then apply the result 2^(q-sq) times to e_0 as a triangular
  // matrix-vector product (n^2/2 each); sq minimises the total.  Every term
  // is nonnegative.  Row r of T*T is accumulated as sum_l T[r][l] * (row l of T).
  int sq = 0;
  {
    double best = 0.0;
    for (int j = 0; j <= q; ++j) {
      const double cost = j * (double)n * n * n / 6.0 + ldexp((double)n * n / 2.0, q - j);
      if (j == 0 || cost < best) { best = cost; sq = j; }
    }
  }
  for (int it = 0; it < sq; ++it) {
    for (int r = 0; r < n; ++r) {
      double* __restrict__ Ur = &U[(size_t)r * n];
      const double* __restrict__ Tr = &T[(size_t)r * n];
      for (int c = 0; c <= r; ++c) Ur[c] = 0.0;
      for (int l = 0; l <= r; ++l) {
        const double t = Tr[l];
        const double* __restrict__ Tl = &T[(size_t)l * n];
        for (int c = 0; c <= l; ++c) Ur[c] += t * Tl[c];
      }
    }
    std::swap(T, U);
  }
  std::vector<double> y(n), z(n);
  for (int r = 0; r < n; ++r) y[r] = T[(size_t)r * n];
  for (long rep = 1; rep < (1L << (q - sq)); ++rep) {
    for (int r = 0; r < n; ++r) {
      const double* __restrict__ Tr = &T[(size_t)r * n];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;  // four independent chains
      int l = 0;
      for (; l + 3 <= r; l += 4) {
        a0 += Tr[l] * y[l];
        a1 += Tr[l + 1] * y[l + 1];
        a2 += Tr[l + 2] * y[l + 2];
        a3 += Tr[l + 3] * y[l + 3];
      }
      for (; l <= r; ++l) a0 += Tr[l] * y[l];
      z[r] = (a0 + a1) + (a2 + a3);
    }
    std::swap(y, z);
  }
  for (int r = 0; r < n; ++r) out[r] = y[r];
}

void divided_differences(int k, double tau, double c, double gamma, int m, double* out) {
  const int n = k + m + 1;
  std::vector<double> dg(n, 0.0), sd(n > 1 ? n - 1 : 1, 0.0), col(n);
  const double* xi = leja_table();
  for (int j = 0; j <= m; ++j) dg[k + j] = tau * c + tau * gamma * xi[j];
  for (int i = 0; i < k; ++i) sd[i] = 1.0;                    // augmentation chain
  for (int i = k; i + 1 < n; ++i) sd[i] = tau * gamma;       // z_{j-1} -> z_j
  expm_bidiag_col0(n, dg.data(), sd.data(), col.data());
  for (int j = 0; j <= m; ++j) out[j] = col[k + j];
}

// ---------------------------------------------------------------------------
// scalar phi_k in FP64: series for |z| < 1, else phi_j = (phi_{j-1} - 1/(j-1)!)/z
// from phi_0 = exp (phi_1 via expm1)
// ---------------------------------------------------------------------------
double phi_scalar(int k, double z) {
  if (k == 0) return exp(z);
  if (k == 1) return z == 0.0 ? 1.0 : expm1(z) / z;
  if (fabs(z) < 1.0) {
    double fact = 1.0;
    for (int i = 2; i <= k; ++i) fact *= i;
    double term = 1.0 / fact, sum = term;
    for (int i = 0; i < 60; ++i) {
      term *= z / (i + k + 1);
      sum += term;
      if (fabs(term) < 1e-18 * fabs(sum)) break;
    }
    return sum;
  }
  double v = expm1(z) / z;  // phi_1
  double fact = 1.0;        // (j-1)!
  for (int j = 2; j <= k; ++j) {
    v = (v - 1.0 / fact) / z;
    fact *= j;
  }
  return v;
}

// ---------------------------------------------------------------------------
// a-priori rule: smallest s = 2^q such that some degree m <= m_max has
// max_G |f - p_m| <= tol max_G |f|, G = 2001 equispaced points of [-2,2]
// ---------------------------------------------------------------------------
static const int kGrid = 2001;

int schedule(int k, double h, double c, double gamma, double tol, int m_max, int* s_out,
             int* m_out, double* d_out) {
  const double* xi = leja_table();
  std::vector<double> g(kGrid), f(kGrid), p(kGrid), om(kGrid), d(m_max + 1);
  const double step = 4.0 / (kGrid - 1);  // the same points as numpy.linspace(-2, 2, 2001)
  for (int i = 0; i < kGrid; ++i) g[i] = (double)i * step + (-2.0);
  g[kGrid - 1] = 2.0;
  for (int q = 0; q <= 20; ++q) {
    const int s = 1 << q;
    const double tau = h / s;
    divided_differences(k, tau, c, gamma, m_max, d.data());
    double fmax = 0.0;
    for (int i = 0; i < kGrid; ++i) {
      f[i] = phi_scalar(k, tau * c + tau * gamma * g[i]);
      fmax = std::max(fmax, fabs(f[i]));
      p[i] = 0.0;
      om[i] = 1.0;
    }
    const double bound = tol * fmax;
    for (int j = 0; j <= m_max; ++j) {
      const double dj = d[j], xj = xi[j];
      for (int i = 0; i < kGrid; ++i) {
        p[i] += dj * om[i];
        om[i] *= (g[i] - xj);
      }
      // max_G |f - p| <= bound  <=>  no grid point exceeds the bound
      bool pass = true;
      for (int i = 0; i < kGrid; ++i)
        if (!(fabs(f[i] - p[i]) <= bound)) { pass = false; break; }
      if (pass) {
        *s_out = s;
        *m_out = j;
        if (d_out)
          for (int i = 0; i <= m_max; ++i) d_out[i] = d[i];
        return 0;
      }
    }
  }
  return 1;
}

// ---------------------------------------------------------------------------
// The skew case A = -iH, H real symmetric (products (alpha A + beta I)x with
// K = C, Sec. II-C): f(xi) = phi_k(-i tau (c + gamma xi)) on H's real interval.
// Opitz's matrix is the one above with complex entries,
//     N = bidiag(diag = [0 x k, -i tau (c + gamma xi_j)],
//                subdiag = [1 x k, -i tau gamma x m]),
// and d_j = exp(N)[k+j][0].  The Metzler shift does not apply; exp(N) is
// formed by scaling (entries of X at most 1/2), a degree-24 Taylor
// polynomial (||X||_1 <= 1, truncation below 1/25!) and squaring.  The
// entries of every power of exp(2^-q N) are divided differences of unimodular
// exponentials scaled by (tau gamma 2^-q)^j, bounded by about 1, so the
// rounding errors stay near eps in absolute terms.
// ---------------------------------------------------------------------------
typedef std::complex<double> cplx;

static void expm_bidiag_col0_c(int n, const cplx* dg, const cplx* sd, cplx* out) {
  double mx = 0.0;
  for (int i = 0; i < n; ++i) mx = std::max(mx, std::abs(dg[i]));
  for (int i = 0; i + 1 < n; ++i) mx = std::max(mx, std::abs(sd[i]));
  int q = 0;
  while (ldexp(0.5, q) < mx) ++q;
  const double sc = ldexp(1.0, -q);
  std::vector<cplx> xd(n), xs(n > 1 ? n - 1 : 1);
  for (int i = 0; i < n; ++i) xd[i] = dg[i] * sc;
  for (int i = 0; i + 1 < n; ++i) xs[i] = sd[i] * sc;
  const int K = 24;
  std::vector<cplx> T((size_t)n * n, 0.0), U((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) T[(size_t)i * n + i] = 1.0;
  for (int it = K; it >= 1; --it) {  // T <- I + X T / it (Horner), band K - it + 1
    const double inv = 1.0 / it;
    const int band = K - it + 1;
    U[0] = xd[0] * T[0] * inv + 1.0;
    for (int r = 1; r < n; ++r) {
      cplx* Ur = &U[(size_t)r * n];
      const cplx* Tr = &T[(size_t)r * n];
      const cplx* Tm = &T[(size_t)(r - 1) * n];
      const cplx a = xd[r], b = xs[r - 1];
      const int c0 = r - band > 0 ? r - band : 0;
      for (int c = c0; c < r; ++c) Ur[c] = (a * Tr[c] + b * Tm[c]) * inv;
      Ur[r] = a * Tr[r] * inv + 1.0;
    }
    std::swap(T, U);
  }
  // exp(N) e_0 = T^(2^q) e_0: `sq` squarings, then 2^(q-sq) triangular products
  int sq = 0;
  {
    double best = 0.0;
    for (int j = 0; j <= q; ++j) {
      const double cost = j * (double)n * n * n / 6.0 + ldexp((double)n * n / 2.0, q - j);
      if (j == 0 || cost < best) { best = cost; sq = j; }
    }
  }
  for (int it = 0; it < sq; ++it) {
    for (int r = 0; r < n; ++r) {
      cplx* Ur = &U[(size_t)r * n];
      const cplx* Tr = &T[(size_t)r * n];
      for (int c = 0; c <= r; ++c) Ur[c] = 0.0;
      for (int l = 0; l <= r; ++l) {
        const cplx t = Tr[l];
        const cplx* Tl = &T[(size_t)l * n];
        for (int c = 0; c <= l; ++c) Ur[c] += t * Tl[c];
      }
    }
    std::swap(T, U);
  }
  std::vector<cplx> y(n), z(n);
  for (int r = 0; r < n; ++r) y[r] = T[(size_t)r * n];
  for (long rep = 1; rep < (1L << (q - sq)); ++rep) {
    for (int r = 0; r < n; ++r) {
      const cplx* Tr = &T[(size_t)r * n];
      cplx a = 0.0;
      for (int l = 0; l <= r; ++l) a += Tr[l] * y[l];
      z[r] = a;
    }
    std::swap(y, z);
  }
  for (int r = 0; r < n; ++r) out[r] = y[r];
}

void divided_differences_imag(int k, double tau, double c, double gamma, int m, double* out) {
  const int n = k + m + 1;
  std::vector<cplx> dg(n, 0.0), sd(n > 1 ? n - 1 : 1, 0.0), col(n);
  const double* xi = leja_table();
  for (int j = 0; j <= m; ++j) dg[k + j] = cplx(0.0, -(tau * c + tau * gamma * xi[j]));
  for (int i = 0; i < k; ++i) sd[i] = 1.0;
  for (int i = k; i + 1 < n; ++i) sd[i] = cplx(0.0, -tau * gamma);
  expm_bidiag_col0_c(n, dg.data(), sd.data(), col.data());
  for (int j = 0; j <= m; ++j) {
    out[2 * j] = col[k + j].real();
    out[2 * j + 1] = col[k + j].imag();
  }
}

// phi_k(z) for complex z: series for |z| < 1, else the recurrence from e^z
static cplx phi_scalar_c(int k, cplx z) {
  if (k == 0) return std::exp(z);
  if (std::abs(z) < 1.0) {
    double fact = 1.0;
    for (int i = 2; i <= k; ++i) fact *= i;
    cplx term = 1.0 / fact, sum = term;
    for (int i = 0; i < 60; ++i) {
      term *= z / (double)(i + k + 1);
      sum += term;
      if (std::abs(term) < 1e-18 * std::abs(sum)) break;
    }
    return sum;
  }
  cplx v = (std::exp(z) - 1.0) / z;
  double fact = 1.0;
  for (int j = 2; j <= k; ++j) {
    v = (v - 1.0 / fact) / z;
    fact *= j;
  }
  return v;
}

void phi_imag(int k, double y, double* re, double* im) {
  const cplx v = phi_scalar_c(k, cplx(0.0, y));
  *re = v.real();
  *im = v.imag();
}

// The a-priori rule of `schedule` with the complex f (max over the grid of
// |f - p_m| against tol max |f|); d_out (optional) gets the interleaved
// divided differences at the chosen s.
int schedule_imag(int k, double h, double c, double gamma, double tol, int m_max, int* s_out,
                  int* m_out, double* d_out) {
  const double* xi = leja_table();
  std::vector<double> g(kGrid), om(kGrid), d(2 * (m_max + 1));
  std::vector<cplx> f(kGrid), p(kGrid);
  const double step = 4.0 / (kGrid - 1);
  for (int i = 0; i < kGrid; ++i) g[i] = (double)i * step + (-2.0);
  g[kGrid - 1] = 2.0;
  for (int q = 0; q <= 20; ++q) {
    const int s = 1 << q;
    const double tau = h / s;
    divided_differences_imag(k, tau, c, gamma, m_max, d.data());
    double fmax = 0.0;
    for (int i = 0; i < kGrid; ++i) {
      f[i] = phi_scalar_c(k, cplx(0.0, -(tau * c + tau * gamma * g[i])));
      fmax = std::max(fmax, std::abs(f[i]));
      p[i] = 0.0;
      om[i] = 1.0;
    }
    const double bound = tol * fmax;
    for (int j = 0; j <= m_max; ++j) {
      const cplx dj(d[2 * j], d[2 * j + 1]);
      const double xj = xi[j];
      for (int i = 0; i < kGrid; ++i) {
        p[i] += dj * om[i];
        om[i] *= (g[i] - xj);
      }
      bool pass = true;
      for (int i = 0; i < kGrid; ++i)
        if (!(std::abs(f[i] - p[i]) <= bound)) { pass = false; break; }
      if (pass) {
        *s_out = s;
        *m_out = j;
        if (d_out)
          for (int i = 0; i < 2 * (m_max + 1); ++i) d_out[i] = d[i];
        return 0;
      }
    }
  }
  return 1;
}

}  // namespace ei

// exported host entry points -------------------------------------------------
extern "C" ei_status ei_leja_points(int m, double* out) {
  if (m < 0 || m > ei::kMaxM || !out) return EI_ERR_INVALID_ARG;
  memcpy(out, ei::leja_table(), sizeof(double) * (m + 1));
  return EI_OK;
}

extern "C" ei_status ei_divided_differences(int k, double tau, double c, double gamma, int m,
                                            double* out) {
  if (k < 0 || k > 8 || m < 0 || m > ei::kMaxM || !out || !(tau > 0) || !(gamma >= 0) ||
      !isfinite(c) || !isfinite(gamma))
    return EI_ERR_INVALID_ARG;
  ei::divided_differences(k, tau, c, gamma, m, out);
  return EI_OK;
}

extern "C" ei_status ei_schedule(int k, double h, double c, double gamma, double tol, int m_max,
                                 int* s_out, int* m_out) {
  if (k < 0 || k > 8 || !(h > 0) || !(tol > 0) || m_max < 1 || m_max > ei::kMaxM || !s_out ||
      !m_out || !(gamma > 0) || !isfinite(c) || !isfinite(gamma))
    return EI_ERR_INVALID_ARG;
  return ei::schedule(k, h, c, gamma, tol, m_max, s_out, m_out, nullptr) ? EI_ERR_NOT_CONVERGED
                                                                          : EI_OK;
}

extern "C" ei_status ei_divided_differences_imag(int k, double tau, double c, double gamma, int m,
                                                 double* out) {
  if (k < 0 || k > 8 || m < 0 || m > ei::kMaxM || !out || !(tau > 0) || !(gamma >= 0) ||
      !isfinite(tau) || !isfinite(c) || !isfinite(gamma))
    return EI_ERR_INVALID_ARG;
  ei::divided_differences_imag(k, tau, c, gamma, m, out);
  return EI_OK;
}

extern "C" ei_status ei_schedule_imag(int k, double h, double c, double gamma, double tol,
                                      int m_max, int* s_out, int* m_out) {
  if (k < 0 || k > 8 || !(h > 0) || !isfinite(h) || !(tol > 0) || m_max < 1 ||
      m_max > ei::kMaxM || !s_out || !m_out || !(gamma > 0) || !isfinite(c) || !isfinite(gamma))
    return EI_ERR_INVALID_ARG;
  return ei::schedule_imag(k, h, c, gamma, tol, m_max, s_out, m_out, nullptr)
             ? EI_ERR_NOT_CONVERGED
             : EI_OK;
}
