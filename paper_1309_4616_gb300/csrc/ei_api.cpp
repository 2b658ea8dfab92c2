// Host orchestration of the C ABI declared in include/ei.h.
//
// phi_k(hA)v by Newton interpolation at Leja points (Sec. II-C, Eq. (3);
// Sec. III-C): the Gershgorin interval [alpha, beta] gives c and gamma; the
// a-priori rule gives the substep count s; per substep the Newton loop is a
// chain of fused kernel launches (one per degree) whose stop test runs on the
// device, so the host launches a predicted batch and synchronises once per
// substep to read the outcome.  Exponential Euler (Eq. (2)) and exponential
// Rosenbrock-Euler integrate z' = J z + F from z = 0 by the same substeps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ei.h"
#include "ei_internal.h"

namespace ei {
const double* leja_table();
void divided_differences(int k, double tau, double c, double gamma, int m, double* out);
int schedule(int k, double h, double c, double gamma, double tol, int m_max, int* s_out,
             int* m_out, double* d_out);
double phi_scalar(int k, double z);
void divided_differences_imag(int k, double tau, double c, double gamma, int m, double* out);
int schedule_imag(int k, double h, double c, double gamma, double tol, int m_max, int* s_out,
                  int* m_out, double* d_out);
void phi_imag(int k, double y, double* re, double* im);
}  // namespace ei

using namespace ei;

enum { KIND_NONE = 0, KIND_STENCIL = 1, KIND_CSR = 2 };

// Operator data and workspaces in one vector format.
struct Prepared {
  bool ready = false;
  int fmt = VF_DF;
  void* cbase = nullptr;   // the fixed diagonal c_i (stencil) / diag (CSR)
  void* qc = nullptr;      // per-step diagonal c_i + g'(u_i)
  void* w[2] = {nullptr, nullptr};
  void* p = nullptr;       // Newton sum (float-float or double)
  void* y = nullptr;       // substep accumulator
  void* r = nullptr;       // substep residual / k = 0 carry
  void* v = nullptr;       // imported right-hand side / F
  void* u = nullptr;       // imported state
  void* csr_val = nullptr; // CSR values in the matvec precision
  void* sell_val = nullptr; // the sliced form's values in this format
  void* a[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // stencil coefficients
  void* diagA = nullptr;   // stencil: diagonal of A (coefficient layout)
  bool coef7 = false;      // explicit stencil coefficients present (stencil operators)
  int64_t n_alloc = 0;     // elements per vector including row padding
  // TMA descriptors of the stencil Newton kernel
  CUtensorMap map_in[4];   // w-input candidates: v, r, w[0], w[1] (halo box)
  CUtensorMap map_in2[4];  // the same with a two-point halo (two-iteration kernel)
  CUtensorMap map_c[6];    // a[0..5]
  CUtensorMap map_diagA, map_qc, map_p;
  CUtensorMap map_u;       // the step's state u (halo box): the TMA F pass
  // native FP64 stencils: the scaled operator (J - cI)/gamma0 of the current
  // Newton loop (a[0..5]/gamma0, (diag - c)/gamma0), keyed on the diagonal
  // array, its content version and (c, gamma).  gamma0 (off_gamma) is the
  // scale the off-diagonals were written with; it is kept while the ratio
  // pre_ratio = gamma0/gamma stays near 1, so that a new interval rewrites only
  // the diagonal (the Newton loop then carries the ratio in its scalars).
  void* sa[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  CUtensorMap map_s[7];
  bool pre_valid = false;
  const void* pre_diag = nullptr;
  unsigned pre_ver = 0;
  double pre_cc = 0.0, pre_gamma = 0.0, pre_ratio = 1.0;
  bool off_valid = false;
  double off_gamma = 0.0;
  // float-float, an operator with constant D, b and c: the scaled operator as
  // a table of kConstTab coefficients (launch_const_table), current when
  // ctab_ok (sa made for the operator's own diagonal)
  void* ctab = nullptr;
  bool ctab_ok = false;
  unsigned qc_ver = 0;     // bumped whenever qc is rewritten (each Rosenbrock step)
};

struct ei_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int kind = KIND_NONE;
  int prec = EI_PREC_F64;
  int64_t n = 0;
  // stencil description (caller's arrays are referenced, not copied)
  StencilDev sd{};
  double dx[3] = {1, 1, 1};
  double* face_term[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // b_D by face
  const void* Du = nullptr;
  double Dc = 0;
  const void* bu[3] = {nullptr, nullptr, nullptr};
  double bcst[3] = {0, 0, 0};
  const void* cu = nullptr;
  double cc = 0;
  bool const_coef = false;  // D, b and c all constants (no arrays)
  // CSR description
  CsrDev cd{};
  int64_t nnz = 0;
  const void* val_u = nullptr;
  const void* diag_u = nullptr;
  // the sliced form of the CSR operator (SellDev): built at set_operator
  int64_t sell_slices = 0, sell_entries = 0;
  int32_t* sell_perm = nullptr;
  int32_t* sell_rlen = nullptr;
  int64_t* sell_ptr = nullptr;
  int32_t* sell_col = nullptr;
  int64_t* sell_src = nullptr;  // CSR entry of each sliced entry (per-format values)
  // Gershgorin rows of A (without the per-step g') and their interval
  double* ger_lo = nullptr;
  double* ger_hi = nullptr;
  double alphaA = 0, betaA = 0;
  // device control, reduction partials, pinned mirror
  DevCtl* ctl = nullptr;
  DevCtl* h_ctl = nullptr;
  double* partials = nullptr;
  int max_blocks = 0;
  Prepared prep[3];
  // staging for ei_step_host
  void* host_stage = nullptr;
  // complex workspaces of ei_phi_apply_imag (v, r, w0, w1, p), format cx_fmt
  void* cx[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int cx_fmt = -1;
  // the last complex plan: for a fixed H, repeated calls with the same
  // (k, h, tol, m_max) reuse the a-priori s, its degree estimate and the
  // divided differences at tau = h/s (keyed on the exact values)
  struct {
    bool valid = false;
    int k = 0, m_max = 0, s = 0, m_pred = 0;
    double h = 0, cc = 0, gamma = 0, tol = 0;
    std::vector<double> dd;
  } cx_plan;
  // the same for the a-priori rule of phi_1 (keyed on h, the interval, tol,
  // m_max): a fixed A called repeatedly with one h reuses it; a Rosenbrock
  // step's J moves the interval and misses
  struct {
    bool valid = false;
    int m_max = 0, s = 0, m_pred = 0;
    double h = 0, cc = 0, gamma = 0, tol = 0;
    std::vector<double> d;
  } phi1_plan;
  // launch accounting and optional per-launch timing of the Newton kernel
  int launches = 0;
  bool profile = false;
  int newton_timed = 0;
  double newton_ms = 0.0;
  int newton_fused = 1;
  int p_rechecks = 0;      // stop tests the host took with the norms formed (brackets undecided)
  // a tensor map over the caller's u of the last step that read it in place
  CUtensorMap umap;
  const void* umap_ptr = nullptr;
  int umap_fmt = -1;
  int newton_bounded = 0;  // timed Newton launches that bracketed the norms
  int coef_table = 0;      // two-iteration launches on the constant operator's table
  int fuse = 0;            // Newton iterations per stencil launch: 0 the format's
                           // default (two for float-float and float, one for native
                           // FP64), 1 one, 2 two
  int csr_lanes = 0;       // lanes per row of the CSR Newton kernels (0: by row length)
  std::vector<cudaEvent_t> ev;
  // learned schedule: the model (caller-owned), the operator's coefficient
  // statistics (computed on first use) and ||v||^2 of the current phi_1 call
  const ei_mlp* model = nullptr;
  bool cs_valid = false;
  double cs_ratio = 1.0, cs_pe = 0.0;
  double vnorm2 = 0.0;
};

#define EI_TRY_CUDA(expr)                        \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) {                     \
      ei_log_cuda(e_, #expr, __LINE__);          \
      return EI_ERR_CUDA;                        \
    }                                            \
  } while (0)

#define EI_LAUNCH(expr)                          \
  do {                                           \
    ++c->launches;                               \
    EI_TRY_CUDA(expr);                           \
  } while (0)

#define EI_TRY(expr)                             \
  do {                                           \
    ei_status s_ = (expr);                       \
    if (s_ != EI_OK) return s_;                  \
  } while (0)

static void ei_log_cuda(cudaError_t e, const char* what, int line) {
  const char* lg = getenv("EI_LOG");
  if (lg && *lg == '1') fprintf(stderr, "ei: CUDA error %s at %s (line %d)\n", cudaGetErrorString(e), what, line);
}

static bool log_on() {
  const char* lg = getenv("EI_LOG");
  return lg && *lg == '1';
}

// layout of the library's vectors: (nx, ny, pitch); CSR vectors are 1D
static int geo_nx(const ei_ctx* c) { return c->kind == KIND_STENCIL ? c->sd.nx : (int)c->n; }
static int geo_pitch(const ei_ctx* c) { return c->kind == KIND_STENCIL ? c->sd.pitch : (int)c->n; }
static int64_t n_alloc_of(const ei_ctx* c) {
  return c->kind == KIND_STENCIL ? (int64_t)c->sd.pitch * c->sd.ny * c->sd.nz : c->n;
}

static int vec_fmt_for(const ei_ctx* c, const ei_options* opt) {
  if (c->prec == EI_PREC_F32) return VF_F32;
  if (opt && opt->arith == EI_ARITH_NATIVE_F64) return VF_F64;
  return VF_DF;
}

static void free_prepared(Prepared& p) {
  void** arrs[] = {&p.cbase, &p.qc,   &p.w[0], &p.w[1], &p.p,    &p.y,    &p.r,
                   &p.v,     &p.u,    &p.csr_val, &p.sell_val, &p.a[0], &p.a[1], &p.a[2], &p.a[3],
                   &p.a[4],  &p.a[5], &p.diagA, &p.sa[0], &p.sa[1], &p.sa[2], &p.sa[3],
                   &p.sa[4], &p.sa[5], &p.sa[6], &p.ctab};
  for (void** a : arrs) {
    if (*a) cudaFree(*a);
    *a = nullptr;
  }
  p.pre_valid = false;
  p.off_valid = false;
  p.ctab_ok = false;
  p.ready = false;
  p.coef7 = false;  // a later operator of another kind must not inherit the layout
  p.n_alloc = 0;
}

static void free_faces(ei_ctx* c) {
  for (auto& f : c->face_term) {
    if (f) cudaFree(f);
    f = nullptr;
  }
}

static void free_operator(ei_ctx* c) {
  c->umap_ptr = nullptr;
  free_faces(c);
  for (auto& p : c->prep) free_prepared(p);
  if (c->ger_lo) cudaFree(c->ger_lo);
  if (c->ger_hi) cudaFree(c->ger_hi);
  if (c->partials) cudaFree(c->partials);
  if (c->host_stage) cudaFree(c->host_stage);
  c->ger_lo = c->ger_hi = nullptr;
  c->partials = nullptr;
  c->host_stage = nullptr;
  for (auto& a : c->cx) {
    if (a) cudaFree(a);
    a = nullptr;
  }
  void** sell[] = {(void**)&c->sell_perm, (void**)&c->sell_rlen, (void**)&c->sell_ptr,
                   (void**)&c->sell_col, (void**)&c->sell_src};
  for (void** a : sell) {
    if (*a) cudaFree(*a);
    *a = nullptr;
  }
  c->sell_slices = c->sell_entries = 0;
  c->cx_fmt = -1;
  c->cx_plan.valid = false;
  c->phi1_plan.valid = false;
  c->max_blocks = 0;
  c->kind = KIND_NONE;
  c->cs_valid = false;
}

static ei_status alloc(void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? EI_ERR_NOMEM : EI_ERR_CUDA;
  }
  return EI_OK;
}

// Build the operator arrays and workspaces of one vector format.  Stencils use
// explicit coefficients (7 arrays with the boundary conditions folded in): the
// Newton kernel then needs no boundary logic, little arithmetic per point, and
// can fuse two iterations per pass.
static ei_status prepare(ei_ctx* c, int fmt) {
  Prepared& P = c->prep[fmt];
  if (P.ready) return EI_OK;
  P.fmt = fmt;
  const int64_t n = c->n;
  const int64_t na = n_alloc_of(c);
  P.n_alloc = na;
  const size_t vb = vec_elem_bytes(fmt) * (size_t)na, pb = p_elem_bytes(fmt) * (size_t)na;
  const int nx = geo_nx(c), ny = c->kind == KIND_STENCIL ? c->sd.ny : 1, pitch = geo_pitch(c);
  ei_status s;
  auto take = [&](void** a, size_t bytes) {
    ei_status r = alloc(a, bytes);
    if (r == EI_OK && cudaMemsetAsync(*a, 0, bytes, c->stream) != cudaSuccess) r = EI_ERR_CUDA;
    return r;
  };
  void** vecs[] = {&P.cbase, &P.qc, &P.w[0], &P.w[1], &P.y, &P.r, &P.v, &P.u};
  for (void** a : vecs)
    if ((s = take(a, vb)) != EI_OK) { free_prepared(P); return s; }
  if ((s = take(&P.p, pb)) != EI_OK) { free_prepared(P); return s; }
  if (c->kind == KIND_STENCIL) {
    P.coef7 = true;
    for (int k = 0; k < 6; ++k)
      if ((s = take(&P.a[k], vb)) != EI_OK) { free_prepared(P); return s; }
    if ((s = take(&P.diagA, vb)) != EI_OK) { free_prepared(P); return s; }
    const void* bptr[3] = {c->bu[0], c->bu[1], c->bu[2]};
    EI_LAUNCH(launch_stencil_coef(c->sd, c->prec, c->dx, c->Du, c->Dc, bptr, c->bcst, c->cu,
                                  c->cc, P.a, P.diagA, fmt, c->stream));
    // tensor maps over the padded arrays
    const int eb = (int)vec_elem_bytes(fmt);
    const void* ins[4] = {P.v, P.r, P.w[0], P.w[1]};
    bool ok = true;
    for (int i = 0; i < 4; ++i) ok = ok && encode_map(&P.map_in[i], ins[i], eb, c->sd, 1);
    for (int i = 0; i < 4; ++i) ok = ok && encode_map(&P.map_in2[i], ins[i], eb, c->sd, 2);
    for (int k = 0; k < 6; ++k) ok = ok && encode_map(&P.map_c[k], P.a[k], eb, c->sd, 0);
    ok = ok && encode_map(&P.map_diagA, P.diagA, eb, c->sd, 0);
    if (fmt == VF_F64 || fmt == VF_DF) {  // the scaled operator of the Newton kernels
      for (int k = 0; k < 7; ++k)
        if ((s = take(&P.sa[k], vb)) != EI_OK) { free_prepared(P); return s; }
      for (int k = 0; k < 7; ++k) ok = ok && encode_map(&P.map_s[k], P.sa[k], eb, c->sd, 0);
    }
    if (fmt == VF_DF && c->const_coef)
      if ((s = alloc(&P.ctab, vec_elem_bytes(fmt) * kConstTab)) != EI_OK) { free_prepared(P); return s; }
    ok = ok && encode_map(&P.map_qc, P.qc, eb, c->sd, 0);
    ok = ok && encode_map(&P.map_p, P.p, 8, c->sd, 0);
    ok = ok && encode_map(&P.map_u, P.u, eb, c->sd, 1);
    if (!ok) { free_prepared(P); return EI_ERR_CUDA; }
  } else {
    P.coef7 = false;
    if ((s = alloc(&P.csr_val, vec_elem_bytes(fmt) * (size_t)c->nnz)) != EI_OK) { free_prepared(P); return s; }
    EI_LAUNCH(launch_fill_coef(P.csr_val, fmt, c->nnz, (int)c->nnz, 1, (int)c->nnz, c->val_u,
                               c->prec, 0.0, 1.0, c->stream));
    if (c->sell_src) {  // the sliced form's values
      if ((s = alloc(&P.sell_val, vec_elem_bytes(fmt) * (size_t)c->sell_entries)) != EI_OK) {
        free_prepared(P);
        return s;
      }
      EI_LAUNCH(launch_sell_gather(c->sell_entries, c->sell_src, nullptr, nullptr, c->val_u,
                                   c->prec, P.sell_val, fmt, c->stream));
    }
    EI_LAUNCH(launch_fill_coef(P.cbase, fmt, n, nx, ny, pitch, c->diag_u, c->prec, 0.0, 1.0,
                               c->stream));
  }
  P.ready = true;
  return EI_OK;
}

// the fixed diagonal of A in this format's layout (stencil: diagA; CSR: diag)
static void* base_diag(Prepared& P) { return P.coef7 ? P.diagA : P.cbase; }

static StencilDev stencil_view(const ei_ctx* c, const Prepared& P, const void* diag) {
  StencilDev s = c->sd;
  for (int k = 0; k < 6; ++k) s.a[k] = P.a[k];
  s.diag = diag;
  return s;
}

static StencilDev stencil_view_scaled(const ei_ctx* c, const Prepared& P) {
  StencilDev s = c->sd;
  for (int k = 0; k < 6; ++k) s.a[k] = P.sa[k];
  s.diag = P.sa[6];
  return s;
}

static CsrDev csr_view(const ei_ctx* c, const Prepared& P, const void* qc) {
  CsrDev d = c->cd;
  d.val = P.csr_val;
  d.qc = qc;
  return d;
}

static ei_status read_ctl(ei_ctx* c) {
  EI_TRY_CUDA(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return EI_OK;
}

static ei_status reset_done(ei_ctx* c) {
  EI_TRY_CUDA(cudaMemsetAsync(&c->ctl->done, 0, 4 * sizeof(int), c->stream));  // done, degree, err, fixup
  return EI_OK;
}

static cudaError_t op_residual(ei_ctx* c, Prepared& P, const void* qc, const void* y,
                               const void* v, void* r) {
  ++c->launches;
  if (c->kind == KIND_STENCIL)
    return launch_stencil_residual(stencil_view(c, P, qc), y, v, r, P.fmt, c->partials, c->ctl,
                                   c->stream);
  return launch_csr_residual(csr_view(c, P, qc), y, v, r, P.fmt, c->partials, c->ctl, c->stream);
}

// Whether the scaled operator in P.sa was made for the diagonal array qc as it
// is now (the caller also keys it on c and gamma: ensure_prescaled).
static bool prescaled_for(const Prepared& P, const void* qc) {
  return P.pre_valid && P.pre_diag == qc && (qc != P.qc || P.pre_ver == P.qc_ver);
}

// Native FP64 and float-float stencil Newton loops run on the scaled operator
// (J - cI)/gamma: one elementwise pass per interval (per step, the diagonal
// alone) saves a multiply per point in every iteration.
static bool wants_prescale(const ei_ctx* c, const Prepared& P) {
  return c->kind == KIND_STENCIL && (P.fmt == VF_F64 || P.fmt == VF_DF) && P.sa[0] != nullptr;
}

// the stencil view of the scaled operator (the two-iteration kernel's halo
// points read their coefficients through it)
static StencilDev stencil_view_scaled(const ei_ctx* c, const Prepared& P);
// d_j r^j: the divided differences of the basis w_j / r^j
static std::vector<double> rescaled_dd(const std::vector<double>& d, double r) {
  std::vector<double> out(d.size());
  double sj = 1.0;
  for (size_t j = 0; j < d.size(); ++j) {
    out[j] = d[j] * sj;
    sj *= r;
  }
  return out;
}

// One point of each entry of the constant operator's table (ConstTabIdx), as
// a padded index: for the off-diagonal towards side s of axis e, a point whose
// neighbour there is inside the grid; for the diagonal of class cx + 4 cy +
// 16 cz, a point on exactly the faces the class names.
static int class_coord(int cls, int n) {
  if (cls == 0) return n >= 3 ? 1 : -1;
  if (cls == 1) return n >= 2 ? 0 : -1;
  if (cls == 2) return n >= 2 ? n - 1 : -1;
  return n == 1 ? 0 : -1;
}
static void const_table_points(const StencilDev& g, ConstTabIdx& ix) {
  const int ext[3] = {g.nx, g.ny, g.nz};
  auto pidx = [&](const int q[3]) {
    return ((int64_t)q[2] * g.ny + q[1]) * g.pitch + q[0];
  };
  for (int k = 0; k < 6; ++k) {
    const int e = k / 2;
    int q[3] = {0, 0, 0};
    q[e] = (k & 1) ? 0 : 1;  // the x- neighbour of x = 1, the x+ neighbour of x = 0
    ix.idx[k] = ext[e] >= 2 ? pidx(q) : -1;
  }
  for (int cls = 0; cls < 64; ++cls) {
    const int q[3] = {class_coord(cls & 3, g.nx), class_coord((cls >> 2) & 3, g.ny),
                      class_coord(cls >> 4, g.nz)};
    ix.idx[6 + cls] = (q[0] < 0 || q[1] < 0 || q[2] < 0) ? -1 : pidx(q);
  }
}

// The off-diagonals keep their scale gamma0 while gamma0/gamma lies within
// 1 +- 1/8: the Newton loop's scale factors (gamma0/gamma)^j then stay within
// about 1.3e5 over 100 steps.
static constexpr double kOffRatioSlack = 0.125;
static ei_status ensure_prescaled(ei_ctx* c, Prepared& P, const void* qc, double cc,
                                  double gamma) {
  if (prescaled_for(P, qc) && P.pre_cc == cc && P.pre_gamma == gamma) return EI_OK;
  const double r = P.off_valid ? P.off_gamma / gamma : 0.0;
  if (P.off_valid && fabs(r - 1.0) <= kOffRatioSlack) {
    EI_LAUNCH(launch_prescale_diag(P.sa[6], qc, P.n_alloc, cc, 1.0 / P.off_gamma, P.fmt,
                                   c->stream));
  } else {
    EI_LAUNCH(launch_prescale(P.sa, P.a, qc, P.n_alloc, cc, 1.0 / gamma, P.fmt, c->stream));
    P.off_valid = true;
    P.off_gamma = gamma;
  }
  P.pre_ratio = P.off_gamma / gamma;
  P.pre_valid = true;
  P.pre_diag = qc;
  P.pre_ver = P.qc_ver;
  P.pre_cc = cc;
  P.pre_gamma = gamma;
  P.ctab_ok = P.ctab && qc == base_diag(P);
  if (P.ctab_ok) {
    ConstTabIdx ix;
    const_table_points(c->sd, ix);
    EI_LAUNCH(launch_const_table(P.sa, ix, P.ctab, P.fmt, c->stream));
  }
  return EI_OK;
}

// pre: run on the scaled operator that ensure_prescaled made current for this
// loop (native FP64 and float-float stencils)
static cudaError_t op_newton(ei_ctx* c, Prepared& P, const void* qc, const void* w_in,
                             void* w_out, const NewtonScalars& s, bool pre = false) {
  ++c->launches;
  if (c->kind == KIND_STENCIL) {
    NewtonMaps M;
    const void* ins[4] = {P.v, P.r, P.w[0], P.w[1]};
    int wi = -1;
    for (int i = 0; i < 4; ++i)
      if (ins[i] == w_in) wi = i;
    if (wi < 0) return cudaErrorInvalidValue;
    M.w = P.map_in[wi];
    pre = pre && prescaled_for(P, qc);
    for (int k = 0; k < 6; ++k) M.c[k] = pre ? P.map_s[k] : P.map_c[k];
    M.c[6] = pre ? P.map_s[6] : (qc == P.qc) ? P.map_qc : P.map_diagA;
    M.p = P.map_p;
    return launch_newton_tma(stencil_view(c, P, qc), M, w_out, P.p, s, P.fmt, c->partials,
                             c->ctl, c->stream, pre);
  }
  if (c->csr_lanes == 0 && P.sell_val) {
    SellDev d{c->sell_slices, c->sell_perm, c->sell_rlen, c->sell_ptr, c->sell_col, P.sell_val,
              qc};
    return launch_csr_newton_sell(d, w_in, w_out, P.p, s, P.fmt, c->partials, c->ctl, c->stream);
  }
  return launch_csr_newton(csr_view(c, P, qc), c->nnz, c->csr_lanes, w_in, w_out, P.p, s, P.fmt,
                           c->partials, c->ctl,
                           c->stream);
}

static cudaError_t op_newton2(ei_ctx* c, Prepared& P, const void* qc, const void* w_in,
                              void* w_out, const NewtonScalars& s, bool pre = false) {
  ++c->launches;
  NewtonMaps M;
  const void* ins[4] = {P.v, P.r, P.w[0], P.w[1]};
  int wi = -1;
  for (int i = 0; i < 4; ++i)
    if (ins[i] == w_in) wi = i;
  if (wi < 0) return cudaErrorInvalidValue;
  M.w = P.map_in2[wi];
  pre = pre && prescaled_for(P, qc);
  for (int k = 0; k < 6; ++k) M.c[k] = pre ? P.map_s[k] : P.map_c[k];
  M.c[6] = pre ? P.map_s[6] : (qc == P.qc) ? P.map_qc : P.map_diagA;
  M.p = P.map_p;
  const void* tab = pre && P.ctab_ok ? P.ctab : nullptr;
  if (tab) ++c->coef_table;
  return launch_newton2_tma(pre ? stencil_view_scaled(c, P) : stencil_view(c, P, qc), M, w_out,
                            P.p, s, P.fmt, c->partials, c->ctl, c->stream, pre, tab);
}

// Whether the Newton loop runs two iterations per launch: explicit-coefficient
// stencils do, except in native FP64 by default, where the FP64 pipe rather
// than HBM bounds the kernel and the fused kernel's halo recomputation only
// adds FP64 work (ei_options.single_iter overrides).
static bool use_pair(const ei_ctx* c, const Prepared& P) {
  return c->kind == KIND_STENCIL && P.coef7 &&
         (c->fuse == 2 || (c->fuse != 1 && P.fmt != VF_F64));
}

// One Newton loop on w_0 = r into P.p.  Returns the degree in *deg; *ok = 0
// when m_max was reached without meeting tol.
// With cx (complex run, CSR only): d and cx->d_im are the real and imaginary
// parts of d_j, and the complex workspaces cx->w, cx->p take the place of
// P.w, P.p.
struct CxRun {
  const double* d_im;
  void* w[2];
  void* p;
};

static ei_status newton_loop(ei_ctx* c, Prepared& P, const void* qc, const void* r,
                             const std::vector<double>& d, double cc, double gamma, double tol,
                             int m_max, int m_pred, int* deg, int* ok,
                             const CxRun* cx = nullptr) {
  const double* xi = leja_table();
  EI_TRY(reset_done(c));
  NewtonScalars s{};
  s.d0 = d[0];
  if (cx) s.d0_im = cx->d_im[0];
  void* const wbuf[2] = {cx ? cx->w[0] : P.w[0], cx ? cx->w[1] : P.w[1]};
  s.inv_gamma = 1.0 / gamma;
  s.tol = tol;
  s.m_max = m_max;
  if (c->profile && c->ev.size() < (size_t)(2 * m_max + 2)) {
    while (c->ev.size() < (size_t)(2 * m_max + 2)) {
      cudaEvent_t e;
      EI_TRY_CUDA(cudaEventCreate(&e));
      c->ev.push_back(e);
    }
  }
  const bool pair = use_pair(c, P);
  const bool pre = !cx && wants_prescale(c, P);
  if (pre) EI_TRY(ensure_prescaled(c, P, qc, cc, gamma));
  // on the operator scaled by 1/gamma0 = r/gamma the loop runs in the basis
  // w_j / r^j: shifts xi_j / r, coefficients d_j r^j (the same p and tests)
  std::vector<double> d_r;
  const double rr = pre ? P.pre_ratio : 1.0;
  if (rr != 1.0) d_r = rescaled_dd(d, rr);
  const std::vector<double>& dv = (rr != 1.0) ? d_r : d;
  // Native FP64 stencil steps after the first bracket ||w|| and ||p|| in FP32
  // and take the stop test from the brackets (the FP64 pipe bounds the
  // kernel, and this saves it two FMAs a point).  Where the brackets cannot
  // decide, the host takes the test with both norms formed, and every later
  // step of the loop forms them.  (The sliced CSR kernel measured slower with
  // brackets: 72.1 against 64.6 us a launch on the 2^20-node graph.)
  bool bracket = pre && !pair && P.fmt == VF_F64;
  int lj[128];          // first iteration index of each launch
  bool l2[128];         // whether that launch did two iterations
  bool lb[128];         // whether that launch bracketed the norms
  int j = 0, nl = 0;
  int batch = m_pred > 0 ? m_pred : 8;
  auto account = [&](int dg) -> ei_status {  // launches that started below dg did the work
    if (!c->profile) return EI_OK;
    for (int i = 0; i < nl; ++i) {
      if (lj[i] >= dg && !(i == 0 && dg == 0)) continue;
      float ms = 0.f;
      EI_TRY_CUDA(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
      c->newton_ms += ms;
      ++c->newton_timed;
      if (lb[i]) ++c->newton_bounded;
    }
    c->newton_fused = pair ? 2 : 1;
    return EI_OK;
  };
  while (true) {
    const int jend = (j + batch < m_max) ? j + batch : m_max;
    while (j < jend) {
      const bool two = pair && (j + 2 <= m_max);
      s.j = j;
      s.d_next = dv[j + 1];
      s.shift = cc / gamma + xi[j];
      s.xi = xi[j] / rr;
      s.bracket = (bracket && j >= 1) ? 1 : 0;
      if (two) {
        s.d_next2 = dv[j + 2];
        s.shift2 = cc / gamma + xi[j + 1];
        s.xi2 = xi[j + 1] / rr;
      }
      const void* w_in = (nl == 0) ? r : wbuf[(nl - 1) & 1];
      void* w_out = wbuf[nl & 1];
      if (c->profile) EI_TRY_CUDA(cudaEventRecord(c->ev[2 * nl], c->stream));
      if (cx) {
        s.d_next_im = cx->d_im[j + 1];
        ++c->launches;
        if (c->csr_lanes == 0 && P.sell_val) {
          SellDev sd{c->sell_slices, c->sell_perm, c->sell_rlen, c->sell_ptr, c->sell_col,
                     P.sell_val, qc};
          EI_TRY_CUDA(launch_csr_newton_sell_c(sd, w_in, w_out, cx->p, s, P.fmt, c->partials,
                                               c->ctl, c->stream));
        } else {
          EI_TRY_CUDA(launch_csr_newton_c(csr_view(c, P, qc), c->nnz, c->csr_lanes, w_in,
                                          w_out, cx->p, s, P.fmt, c->partials, c->ctl,
                                          c->stream));
        }
      } else if (two) {
        EI_TRY_CUDA(op_newton2(c, P, qc, w_in, w_out, s, pre));
      } else {
        EI_TRY_CUDA(op_newton(c, P, qc, w_in, w_out, s, pre));
      }
      if (c->profile) EI_TRY_CUDA(cudaEventRecord(c->ev[2 * nl + 1], c->stream));
      lj[nl] = j;
      l2[nl] = two;
      lb[nl] = s.bracket != 0;
      ++nl;
      j += two ? 2 : 1;
    }
    EI_TRY(read_ctl(c));
    const int done = c->h_ctl->done;
    if (done == 1 || done == 2) {
      *deg = c->h_ctl->degree;
      *ok = (done == 1);
      if (c->h_ctl->fixup) {
        // stopped at the first of a launch's two iterations: p holds p_{deg+1}
        for (int i = 0; i < nl; ++i)
          if (l2[i] && lj[i] == *deg - 1)
            EI_LAUNCH(launch_p_fixup(P.p, P.w[i & 1], P.fmt, P.n_alloc, dv[*deg + 1], c->stream));
      }
      return account(*deg);
    }
    if (done == 6) {
      // the norm brackets could not decide at degree dg: form both norms and
      // take the test as the other steps do; on a fail go on from dg with the
      // norms formed in every step
      const int dg = c->h_ctl->degree;
      ++c->p_rechecks;
      int made = -1;  // the launch that made degree dg; later ones exited at once
      for (int i = 0; i < nl; ++i)
        if (lj[i] == dg - 1) made = i;
      if (made < 0) return EI_ERR_STATE;
      EI_LAUNCH(launch_p_sqnorm(P.p, P.fmt, P.n_alloc, c->partials, c->ctl, c->stream));
      EI_TRY(read_ctl(c));
      const double np2 = c->h_ctl->sum0;
      EI_LAUNCH(launch_p_sqnorm(wbuf[made & 1], P.fmt, P.n_alloc, c->partials, c->ctl,
                                c->stream));
      EI_TRY(read_ctl(c));
      const double nw2 = c->h_ctl->sum0;
      if (!isfinite(np2) || !isfinite(nw2)) return EI_ERR_NONFINITE;
      if (fabs(dv[dg]) * sqrt(nw2) <= tol * sqrt(np2)) {
        *deg = dg;
        *ok = 1;
        return account(dg);
      }
      if (dg >= m_max) {
        *deg = m_max;
        *ok = 0;
        return account(dg);
      }
      nl = made + 1;
      j = dg;
      bracket = false;
      EI_TRY(reset_done(c));
      batch = 8;
      continue;
    }
    if (done == 4) return EI_ERR_NONFINITE;
    if (done == 5) return EI_ERR_TIMEOUT;
    if (j >= m_max) { *deg = m_max; *ok = 0; return EI_OK; }
    batch = 8;
  }
}

// Interval of the current operator: A alone, or J = A + diag(g'(u)).
static void interval(double alpha, double beta, double* cc, double* gamma) {
  *cc = 0.5 * (alpha + beta);
  *gamma = 0.25 * (beta - alpha);
}

static void stats_reset(ei_stats* st) {
  if (st) memset(st, 0, sizeof(*st));
}

// The float-float format carries 48 significand bits over FP32's exponent
// range, so it matches native FP64 only inside that range.  A float-float
// call runs there when the operator's spectral bound rho = max(|alpha|, |beta|)
// lies in [2^-60, 2^60] (or is 0) and the vector it acts on has
// max |x| in [2^-60, 2^50] (or is zero): every coefficient, iterate and
// squared-norm partial then stays inside FP32's exponents, and entries that
// underflow (below 2^-126) lie at least 2^-66 below the largest, far under the
// 1e-9 bound of the results.  Outside it the call runs in native FP64.
static bool df_rho_ok(double alpha, double beta) {
  const double rho = fmax(fabs(alpha), fabs(beta));
  return rho == 0.0 || (rho >= 0x1p-60 && rho <= 0x1p60);
}
static bool df_vec_ok(double vmax) {
  return vmax == 0.0 || (vmax >= 0x1p-60 && vmax <= 0x1p50);
}
// A step forms F = A u + g(u) in the format as well: u's largest magnitude U
// stays at or below 2^20 (so g(u) <= 2^41), rho U <= 2^40, and the squared
// norm of F, as the format computed it, lies in [2^-60, 2^100] (a zero or a
// smaller value may be an underflow: the step then reruns in native FP64,
// which also settles an exact equilibrium).
static bool df_step_ok(double alpha, double beta, double umax, double fnorm2) {
  const double rho = fmax(fabs(alpha), fabs(beta));
  return df_rho_ok(alpha, beta) && umax <= 0x1p20 && rho * umax <= 0x1p40 &&
         fnorm2 >= 0x1p-60 && fnorm2 <= 0x1p100;
}
// options of a call rerun in native FP64
static ei_options native_opts(const ei_options* opt) {
  ei_options o;
  if (opt) o = *opt;
  else memset(&o, 0, sizeof(o));
  o.arith = EI_ARITH_NATIVE_F64;
  return o;
}

// ===========================================================================
// Learned schedule: a network proposes (s, m); s substeps of exactly m Newton
// steps run with one check of the a posteriori estimate per substep and a
// single synchronisation; a failed check falls back to the plain method.
// ===========================================================================

// Coefficient statistics of the operator's inputs (computed once per operator).
static ei_status coef_stats(ei_ctx* c, double* ratio, double* pe) {
  if (!c->cs_valid) {
    double r = 1.0, p = 0.0;
    if (c->kind == KIND_STENCIL) {
      const int dim = c->sd.dim;
      bool arrays = c->Du != nullptr;
      for (int e = 0; e < dim; ++e) arrays = arrays || c->bu[e] != nullptr;
      if (!arrays) {
        for (int e = 0; e < dim; ++e)
          p = std::max(p, fabs(c->bcst[e]) * c->dx[e] / (2.0 * c->Dc));
      } else {
        const void* bptr[3] = {c->bu[0], c->bu[1], c->bu[2]};
        EI_TRY_CUDA(launch_coef_stats(c->n, 0, c->prec, dim, c->Du, c->Dc, bptr, c->bcst, c->dx,
                                      c->partials, c->ctl, c->stream));
        EI_TRY(read_ctl(c));
        r = c->h_ctl->cs_sum / ((double)c->n * c->h_ctl->cs_max);
        p = c->h_ctl->cs_pe;
      }
    } else if (c->diag_u) {
      const void* none[3] = {nullptr, nullptr, nullptr};
      const double zero[3] = {0, 0, 0}, one[3] = {1, 1, 1};
      EI_TRY_CUDA(launch_coef_stats(c->n, 1, c->prec, 1, c->diag_u, 0.0, none, zero, one,
                                    c->partials, c->ctl, c->stream));
      EI_TRY(read_ctl(c));
      r = c->h_ctl->cs_max > 0 ? c->h_ctl->cs_sum / ((double)c->n * c->h_ctl->cs_max) : 1.0;
    }
    c->cs_ratio = isfinite(r) ? r : 1.0;
    c->cs_pe = p;
    c->cs_valid = true;
  }
  *ratio = c->cs_ratio;
  *pe = c->cs_pe;
  return EI_OK;
}

// The twelve features of a phi_1 call at substep count s (see ei.h).
void ei::learned_features(double* f, double s, double h, double alpha, double beta, double tol,
                      int csr, int dim, int64_t n, double ratio, double pe, double vnorm) {
  const double cc = 0.5 * (alpha + beta), gamma = 0.25 * (beta - alpha);
  const double tau = h / s;
  const double rho = std::max(fabs(alpha), fabs(beta));
  const double rms = vnorm / sqrt((double)n);
  const double lr = rms > 0 ? std::min(30.0, std::max(-30.0, log10(rms))) : -30.0;
  f[0] = log10(tau * gamma);
  f[1] = std::max(-8.0, std::min(8.0, cc / gamma)) / 4.0;
  f[2] = log10(tol) / 10.0;
  f[3] = log2(s) / 10.0;
  f[4] = log10(h * rho) / 3.0;
  f[5] = 1.0;  // k
  f[6] = csr ? 1.0 : 0.0;
  f[7] = csr ? 0.0 : dim / 3.0;
  f[8] = ratio;
  f[9] = log10(1.0 + std::min(pe, 1e30));
  f[10] = lr / 10.0;
  f[11] = log10((double)n) / 8.0;
}

static ei_status fill_features(ei_ctx* c, ei_stats* st, int s, double h, double alpha,
                               double beta, double tol) {
  if (!st) return EI_OK;
  double ratio, pe;
  EI_TRY(coef_stats(c, &ratio, &pe));
  learned_features(st->features, (double)s, h, alpha, beta, tol, c->kind == KIND_CSR, c->sd.dim,
                   c->n, ratio, pe, sqrt(c->vnorm2));
  return EI_OK;
}

// Of the accepted q (output 1 >= z_min, the predicted degree with its
// margins within m_max) the one with the fewest operator applications
// 2^q (m_q + 1) - 1; ties go to the smaller q.
bool ei::learned_decide(const float* o, int rows, const ei_mlp_decision& D, int m_max, int* s,
                    int* m) {
  const int qn = std::min(D.q_max, rows - 1);
  bool found = false;
  double best = 0.0;
  for (int q = 0; q <= qn; ++q) {
    const double o0 = o[EI_MLP_OUTPUTS * q], o1 = o[EI_MLP_OUTPUTS * q + 1];
    const double need = m_max * o0 * (1.0 + D.rho_m) + D.delta_m;
    if (o1 >= D.z_min && need <= m_max) {
      const int mq = std::max(1, std::min(m_max, (int)ceil(need)));
      const double cost = ldexp((double)(mq + 1), q) - 1.0;
      if (!found || cost < best) {
        found = true;
        best = cost;
        *s = 1 << q;
        *m = mq;
      }
    }
  }
  return found;
}

// Exactly m Newton steps on r with no test in between: the kernels judge only
// degree m and count a failed check into ctl->fixfail.  Launches only.  With
// two-step launches an odd count starts with one single step, so the last
// launch ends at degree m.  timed: record events around each launch.
static ei_status newton_fixed(ei_ctx* c, Prepared& P, const void* qc, const void* r,
                              const std::vector<double>& d, double cc, double gamma, double tol,
                              int m, bool timed, int* n_launched) {
  const double* xi = leja_table();
  EI_TRY(reset_done(c));
  NewtonScalars s{};
  s.d0 = d[0];
  s.inv_gamma = 1.0 / gamma;
  s.tol = tol;
  s.m_max = m;
  s.fixed = 1;
  const bool pair = use_pair(c, P);
  const bool pre = wants_prescale(c, P);
  if (pre) EI_TRY(ensure_prescaled(c, P, qc, cc, gamma));
  std::vector<double> d_r;  // the rescaled basis, as in newton_loop
  const double rr = pre ? P.pre_ratio : 1.0;
  if (rr != 1.0) d_r = rescaled_dd(d, rr);
  const std::vector<double>& dv = (rr != 1.0) ? d_r : d;
  if (timed)
    while (c->ev.size() < (size_t)(2 * m + 2)) {
      cudaEvent_t e;
      EI_TRY_CUDA(cudaEventCreate(&e));
      c->ev.push_back(e);
    }
  int j = 0, nl = 0;
  while (j < m) {
    const bool two = pair && ((m - j) % 2 == 0);
    s.j = j;
    s.d_next = dv[j + 1];
    s.shift = cc / gamma + xi[j];
    s.xi = xi[j] / rr;
    if (two) {
      s.d_next2 = dv[j + 2];
      s.shift2 = cc / gamma + xi[j + 1];
      s.xi2 = xi[j + 1] / rr;
    }
    const void* w_in = (nl == 0) ? r : P.w[(nl - 1) & 1];
    void* w_out = P.w[nl & 1];
    if (timed) EI_TRY_CUDA(cudaEventRecord(c->ev[2 * nl], c->stream));
    if (two) {
      EI_TRY_CUDA(op_newton2(c, P, qc, w_in, w_out, s, pre));
    } else {
      EI_TRY_CUDA(op_newton(c, P, qc, w_in, w_out, s, pre));
    }
    if (timed) EI_TRY_CUDA(cudaEventRecord(c->ev[2 * nl + 1], c->stream));
    ++nl;
    j += two ? 2 : 1;
  }
  *n_launched = nl;
  return EI_OK;
}

// h phi_1(hJ) v by s substeps of exactly m Newton steps, then one
// synchronisation: *ok says every substep passed its check.
static ei_status phi1_fixed(ei_ctx* c, Prepared& P, const void* qc, double h, double cc,
                            double gamma, double tol, int s, int m, bool* ok,
                            const void** result, int* result_is_p, double* result_scale) {
  const double tau = h / s;
  std::vector<double> d(m + 1);
  divided_differences(1, tau, cc, gamma, m, d.data());
  EI_TRY_CUDA(cudaMemsetAsync(&c->ctl->fixfail, 0, sizeof(int), c->stream));
  if (s > 1) EI_LAUNCH(launch_zero(P.y, P.fmt, P.n_alloc, c->stream));
  int timed_launches = 0;
  for (int i = 0; i < s; ++i) {
    const void* r = P.v;
    if (i > 0) {
      EI_TRY_CUDA(op_residual(c, P, qc, P.y, P.v, P.r));
      r = P.r;
    }
    int nl = 0;
    const bool timed = c->profile && i == 0;  // the first substep's launches
    EI_TRY(newton_fixed(c, P, qc, r, d, cc, gamma, tol, m, timed, &nl));
    if (timed) timed_launches = nl;
    if (s > 1) EI_LAUNCH(launch_axpy(P.y, P.p, P.fmt, P.n_alloc, tau, c->stream));
  }
  EI_TRY(read_ctl(c));
  *ok = c->h_ctl->fixfail == 0;
  if (timed_launches) {
    for (int i = 0; i < timed_launches; ++i) {
      float ms = 0.f;
      EI_TRY_CUDA(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
      c->newton_ms += ms;
      ++c->newton_timed;
    }
    c->newton_fused = use_pair(c, P) ? 2 : 1;
  }
  if (s == 1) {
    *result = P.p;
    *result_is_p = 1;
    *result_scale = h;
  } else {
    *result = P.y;
    *result_is_p = 0;
    *result_scale = 1.0;
  }
  return EI_OK;
}

// Integrate y' = J y + v from 0 over h by s substeps: returns y_s in the
// buffer *result (vector format if *result_is_p == 0, Newton-sum format if 1).
// k = 1 only.  v: imported vector (P.v); qc: J's diagonal array.
// One attempt at s substeps with the per-substep a posteriori stop: d holds
// the divided differences of tau = h/s, m_pred the degree launched before the
// first look at the estimate.  *ok = every substep converged within m_max.
// Substep degrees go to st->degrees (first EI_STATS_MAX_SUBSTEPS).
static ei_status substep_attempt(ei_ctx* c, Prepared& P, const void* qc, double h, double cc,
                                 double gamma, double tol, int m_max, int s, int m_pred,
                                 const std::vector<double>& d, ei_stats* st, bool* ok_all,
                                 int* matvecs, int* dsum, int* dmax) {
  const double tau = h / s;
  if (s > 1) EI_LAUNCH(launch_zero(P.y, P.fmt, P.n_alloc, c->stream));
  *ok_all = true;
  *matvecs = *dsum = *dmax = 0;
  for (int i = 0; i < s; ++i) {
    const void* r = P.v;
    if (i > 0) {
      EI_TRY_CUDA(op_residual(c, P, qc, P.y, P.v, P.r));
      r = P.r;
      ++*matvecs;
    }
    int deg = 0, ok = 0;
    EI_TRY(newton_loop(c, P, qc, r, d, cc, gamma, tol, m_max, m_pred, &deg, &ok));
    *matvecs += deg;
    if (!ok) {
      *ok_all = false;
      return EI_OK;
    }
    if (st && i < EI_STATS_MAX_SUBSTEPS) st->degrees[i] = deg;
    *dsum += deg;
    if (deg > *dmax) *dmax = deg;
    if (s > 1) EI_LAUNCH(launch_axpy(P.y, P.p, P.fmt, P.n_alloc, tau, c->stream));
  }
  return EI_OK;
}

static void set_result(Prepared& P, int s, double h, const void** result, int* is_p,
                       double* scale) {
  if (s == 1) {  // y_1 = tau * p
    *result = P.p;
    *is_p = 1;
    *scale = h;
  } else {
    *result = P.y;
    *is_p = 0;
    *scale = 1.0;
  }
}

static ei_status phi1_substeps(ei_ctx* c, Prepared& P, const void* qc, double h, double alpha,
                               double beta, double tol, const ei_options* opt, ei_stats* st,
                               const void** result, int* result_is_p, double* result_scale) {
  double cc, gamma;
  interval(alpha, beta, &cc, &gamma);
  const int m_max = (opt && opt->m_max > 0 && opt->m_max <= 100) ? opt->m_max : 100;
  const int learned = opt ? opt->learned : 0;
  int wasted = 0;  // operator applications of a rejected learned proposal
  if ((learned == 1 || learned == 3) && c->model && !(opt && opt->fixed_s > 0)) {
    double ratio, pe;
    EI_TRY(coef_stats(c, &ratio, &pe));
    const ei_mlp_decision& D = mlp_decision(c->model);
    const int rows = D.q_max + 1;
    double feat[(EI_MLP_MAX_Q + 1) * EI_MLP_INPUTS];
    for (int q = 0; q < rows; ++q)
      learned_features(feat + EI_MLP_INPUTS * q, (double)(1 << q), h, alpha, beta, tol,
                       c->kind == KIND_CSR, c->sd.dim, c->n, ratio, pe, sqrt(c->vnorm2));
    float outs[(EI_MLP_MAX_Q + 1) * EI_MLP_OUTPUTS];
    EI_TRY(mlp_infer_host(c->model, feat, rows, outs));
    int s_l = 0, m_l = 0;
    if (learned_decide(outs, rows, D, m_max, &s_l, &m_l)) {
      int q_l = 0;
      while ((1 << q_l) < s_l) ++q_l;
      if (st) {
        st->learned_s = s_l;
        st->learned_m = m_l;
        memcpy(st->features, feat + EI_MLP_INPUTS * q_l, sizeof(st->features));
      }
      bool ok = false;
      int mv = 0, dsum = 0, dmax = 0;
      if (learned == 3) {  // fixed count
        EI_TRY(phi1_fixed(c, P, qc, h, cc, gamma, tol, s_l, m_l, &ok, result, result_is_p,
                          result_scale));
        mv = s_l * m_l + (s_l - 1);
        dsum = s_l * m_l;
        dmax = m_l;
        if (ok && st)
          for (int i = 0; i < s_l && i < EI_STATS_MAX_SUBSTEPS; ++i) st->degrees[i] = m_l;
      } else {  // adaptive: the proposal's s, the a posteriori stop in every substep
        std::vector<double> d(m_max + 1);
        divided_differences(1, h / s_l, cc, gamma, m_max, d.data());
        EI_TRY(substep_attempt(c, P, qc, h, cc, gamma, tol, m_max, s_l, m_l, d, st, &ok, &mv,
                               &dsum, &dmax));
        if (ok) set_result(P, s_l, h, result, result_is_p, result_scale);
      }
      if (ok) {
        if (st) {
          st->learned = 1;
          st->s = s_l;
          st->restarts = 0;
          st->matvecs += mv;
          st->degree_sum = dsum;
          st->degree_max = dmax;
          st->alpha = alpha;
          st->beta = beta;
        }
        return EI_OK;
      }
      if (st) {
        st->learned = 2;
        memset(st->degrees, 0, sizeof(st->degrees));
      }
      wasted = mv;
    } else if (st) {
      st->learned = 3;
    }
  }
  int s = 1, m_pred = 0;
  std::vector<double> d(m_max + 1);
  bool have_d = false;  // the schedule hands back the divided differences of its s
  auto& plan = c->phi1_plan;
  if (opt && opt->fixed_s > 0) {
    s = opt->fixed_s;
  } else if (plan.valid && plan.h == h && plan.cc == cc && plan.gamma == gamma &&
             plan.tol == tol && plan.m_max == m_max) {
    s = plan.s;  // the same rule on the same interval: its s, estimate and d
    m_pred = plan.m_pred;
    d = plan.d;
    have_d = true;
  } else if (schedule(1, h, cc, gamma, tol, m_max, &s, &m_pred, d.data()) != 0) {
    return EI_ERR_NOT_CONVERGED;
  } else {
    have_d = true;
    plan.valid = true;
    plan.h = h;
    plan.cc = cc;
    plan.gamma = gamma;
    plan.tol = tol;
    plan.m_max = m_max;
    plan.s = s;
    plan.m_pred = m_pred;
    plan.d = d;
  }
  if (st) st->m_sched = m_pred;
  int restarts = 0, matvecs = 0;
  while (s <= (1 << 20)) {
    if (!have_d) divided_differences(1, h / s, cc, gamma, m_max, d.data());
    have_d = false;
    bool ok_all = true;
    int mv = 0, dsum = 0, dmax = 0;
    EI_TRY(substep_attempt(c, P, qc, h, cc, gamma, tol, m_max, s, m_pred, d, st, &ok_all, &mv,
                           &dsum, &dmax));
    matvecs += mv;
    if (ok_all || (opt && opt->no_restart && opt->fixed_s > 0)) {
      if (st) {
        st->s = s;
        st->restarts = restarts;
        st->matvecs += matvecs + wasted;
        st->degree_sum = dsum;
        st->degree_max = dmax;
        st->alpha = alpha;
        st->beta = beta;
        if (learned == 2) {
          st->learned = 4;
          EI_TRY(fill_features(c, st, s, h, alpha, beta, tol));
        }
      }
      if (!ok_all) return EI_ERR_NOT_CONVERGED;
      set_result(P, s, h, result, result_is_p, result_scale);
      return EI_OK;
    }
    ++restarts;
    if (st) memset(st->degrees, 0, sizeof(st->degrees));
    s *= 2;
  }
  return EI_ERR_NOT_CONVERGED;
}

// The sliced form (SellDev) of the context's CSR operator, from its validated
// rowptr and col: rows sorted by length (longest first, stable) inside windows
// of kSellWindow rows, slices of 32, each slice padded to its longest row.
// The host builds the permutation, the slice offsets and the CSR entry of every
// sliced entry; the device gathers the columns (and, per format, the values in
// prepare).
static ei_status build_sell(ei_ctx* c) {
  const int64_t n = c->n;
  std::vector<int64_t> rp(n + 1);
  EI_TRY_CUDA(cudaMemcpyAsync(rp.data(), c->cd.rowptr, sizeof(int64_t) * (n + 1),
                              cudaMemcpyDeviceToHost, c->stream));
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t ns = (n + 31) / 32;
  std::vector<int32_t> perm(ns * 32, -1);
  std::vector<int32_t> idx;
  for (int64_t w0 = 0; w0 < n; w0 += kSellWindow) {
    const int64_t w1 = std::min(n, w0 + kSellWindow);
    idx.resize(w1 - w0);
    for (int64_t i = w0; i < w1; ++i) idx[i - w0] = (int32_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
      return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
    });
    std::copy(idx.begin(), idx.end(), perm.begin() + w0);
  }
  std::vector<int32_t> rlen(ns * 32, 0);
  for (int64_t i = 0; i < ns * 32; ++i)
    if (perm[i] >= 0) rlen[i] = (int32_t)(rp[perm[i] + 1] - rp[perm[i]]);
  std::vector<int64_t> sptr(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int64_t len = 0;
    for (int l = 0; l < 32; ++l) {
      const int32_t r = perm[sl * 32 + l];
      if (r >= 0) len = std::max(len, rp[r + 1] - rp[r]);
    }
    sptr[sl + 1] = sptr[sl] + 32 * len;
  }
  const int64_t e = sptr[ns];
  std::vector<int64_t> src(e > 0 ? e : 1, -1);
  for (int64_t sl = 0; sl < ns; ++sl) {
    const int64_t len = (sptr[sl + 1] - sptr[sl]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int32_t r = perm[sl * 32 + l];
      const int64_t rl = r >= 0 ? rp[r + 1] - rp[r] : 0;
      for (int64_t k = 0; k < rl; ++k) src[sptr[sl] + k * 32 + l] = rp[r] + k;
    }
    (void)len;
  }
  ei_status st;
  if ((st = alloc((void**)&c->sell_perm, sizeof(int32_t) * ns * 32)) != EI_OK) return st;
  if ((st = alloc((void**)&c->sell_rlen, sizeof(int32_t) * ns * 32)) != EI_OK) return st;
  if ((st = alloc((void**)&c->sell_ptr, sizeof(int64_t) * (ns + 1))) != EI_OK) return st;
  if ((st = alloc((void**)&c->sell_col, sizeof(int32_t) * (e > 0 ? e : 1))) != EI_OK) return st;
  if ((st = alloc((void**)&c->sell_src, sizeof(int64_t) * (e > 0 ? e : 1))) != EI_OK) return st;
  EI_TRY_CUDA(cudaMemcpyAsync(c->sell_perm, perm.data(), sizeof(int32_t) * ns * 32,
                              cudaMemcpyHostToDevice, c->stream));
  EI_TRY_CUDA(cudaMemcpyAsync(c->sell_rlen, rlen.data(), sizeof(int32_t) * ns * 32,
                              cudaMemcpyHostToDevice, c->stream));
  EI_TRY_CUDA(cudaMemcpyAsync(c->sell_ptr, sptr.data(), sizeof(int64_t) * (ns + 1),
                              cudaMemcpyHostToDevice, c->stream));
  EI_TRY_CUDA(cudaMemcpyAsync(c->sell_src, src.data(), sizeof(int64_t) * (e > 0 ? e : 1),
                              cudaMemcpyHostToDevice, c->stream));
  if (e > 0)
    EI_TRY_CUDA(launch_sell_gather(e, c->sell_src, c->cd.col, c->sell_col, nullptr, c->prec,
                                   nullptr, VF_F64, c->stream));
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));  // the host tables go out of scope
  c->sell_slices = ns;
  c->sell_entries = e;
  return EI_OK;
}

static void log_stats(const char* what, const ei_stats* st, ei_status rc) {
  if (!log_on() || !st) return;
  fprintf(stderr,
          "{\"ei\": \"%s\", \"status\": %d, \"alpha\": %.17g, \"beta\": %.17g, \"s\": %d, "
          "\"restarts\": %d, \"matvecs\": %d, \"degree_sum\": %d, \"degree_max\": %d, "
          "\"m_sched\": %d}\n",
          what, (int)rc, st->alpha, st->beta, st->s, st->restarts, st->matvecs, st->degree_sum,
          st->degree_max, st->m_sched);
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* ei_status_string(ei_status s) {
  switch (s) {
    case EI_OK: return "ok";
    case EI_ERR_INVALID_ARG: return "invalid argument";
    case EI_ERR_NONFINITE: return "non-finite value";
    case EI_ERR_NOT_CONVERGED: return "not converged";
    case EI_ERR_TIMEOUT: return "device wait timed out";
    case EI_ERR_CUDA: return "CUDA error";
    case EI_ERR_NOMEM: return "out of device memory";
    case EI_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

ei_status ei_create(ei_ctx** out, int device, void* stream) {
  if (!out) return EI_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? EI_ERR_INVALID_ARG : EI_ERR_CUDA;
  }
  EI_TRY_CUDA(cudaSetDevice(device));
  ei_ctx* c = new ei_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaMalloc(&c->ctl, sizeof(DevCtl)) != cudaSuccess ||
      cudaMallocHost(&c->h_ctl, sizeof(DevCtl)) != cudaSuccess) {
    cudaGetLastError();
    if (c->ctl) cudaFree(c->ctl);
    delete c;
    return EI_ERR_NOMEM;
  }
  cudaMemset(c->ctl, 0, sizeof(DevCtl));
  memset(c->h_ctl, 0, sizeof(DevCtl));
  *out = c;
  return EI_OK;
}

void ei_destroy(ei_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_operator(c);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->ctl) cudaFree(c->ctl);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  delete c;
}

ei_status ei_set_stream(ei_ctx* c, void* stream) {
  if (!c) return EI_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return EI_OK;
}

ei_status ei_set_operator_stencil(ei_ctx* c, int dim, const int64_t n[3], const double dx[3],
                                  const void* D, double D_const, const void* const b[3],
                                  const double b_const[3], const void* cdiag, double c_const,
                                  const int bc[6], int prec) {
  if (!c || !n || !dx || !bc || (dim != 2 && dim != 3) ||
      (prec != EI_PREC_F64 && prec != EI_PREC_F32))
    return EI_ERR_INVALID_ARG;
  int64_t ext[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
  for (int e = 0; e < 3; ++e)
    if (ext[e] < 1 || ext[e] > (1 << 30)) return EI_ERR_INVALID_ARG;
  for (int e = 0; e < dim; ++e)
    if (!(dx[e] > 0) || !isfinite(dx[e])) return EI_ERR_INVALID_ARG;
  for (int f = 0; f < 2 * dim; ++f)
    if (bc[f] != EI_BC_DIRICHLET0 && bc[f] != EI_BC_NEUMANN0) return EI_ERR_INVALID_ARG;
  if (!isfinite(D_const) || !isfinite(c_const)) return EI_ERR_INVALID_ARG;
  if (b_const)
    for (int e = 0; e < dim; ++e)
      if (!isfinite(b_const[e])) return EI_ERR_INVALID_ARG;
  // grid limits of the stencil kernels: 32 x 8 x 16 points per block
  if ((double)ext[0] * ext[1] * ext[2] > 4.0e9 || ext[1] > 65535 * 8 || ext[2] > 65535 * 16)
    return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  cudaStreamSynchronize(c->stream);
  free_operator(c);
  c->kind = KIND_STENCIL;
  c->prec = prec;
  c->n = ext[0] * ext[1] * ext[2];
  StencilDev& s = c->sd;
  s = StencilDev{};
  s.dim = dim;
  s.nx = (int)ext[0];
  s.ny = (int)ext[1];
  s.nz = (int)ext[2];
  s.pitch = (int)((ext[0] + 3) / 4 * 4);  // rows start on 16-byte boundaries
  for (int f = 0; f < 6; ++f) s.bc[f] = (f < 2 * dim) ? bc[f] : EI_BC_NEUMANN0;
  for (int e = 0; e < 3; ++e) c->dx[e] = (e < dim) ? dx[e] : 1.0;
  c->Du = D;
  c->Dc = D_const;
  for (int e = 0; e < 3; ++e) {
    c->bu[e] = (b && e < dim) ? b[e] : nullptr;
    c->bcst[e] = (b_const && e < dim) ? b_const[e] : 0.0;
  }
  c->cu = cdiag;
  c->cc = c_const;
  c->const_coef = !D && !cdiag;
  for (int e = 0; e < dim; ++e) c->const_coef = c->const_coef && !c->bu[e];
  // Gershgorin rows of A (FP64 from the caller's arrays) and reduction space
  int nb = newton_tma_blocks(s);
  if (nb < reduction_capacity()) nb = reduction_capacity();
  c->max_blocks = nb;
  ei_status st;
  if ((st = alloc((void**)&c->partials, sizeof(double) * 4 * nb)) != EI_OK) { free_operator(c); return st; }
  if ((st = alloc((void**)&c->ger_lo, sizeof(double) * c->n)) != EI_OK) { free_operator(c); return st; }
  if ((st = alloc((void**)&c->ger_hi, sizeof(double) * c->n)) != EI_OK) { free_operator(c); return st; }
  const void* bptr[3] = {c->bu[0], c->bu[1], c->bu[2]};
  cudaError_t e = launch_stencil_gershgorin(s, prec, c->dx, D, D_const, bptr, c->bcst, cdiag,
                                            c_const, c->ger_lo, c->ger_hi, c->partials, c->ctl,
                                            c->stream);
  if (e != cudaSuccess) { free_operator(c); return EI_ERR_CUDA; }
  if ((st = prepare(c, prec == EI_PREC_F32 ? VF_F32 : VF_DF)) != EI_OK) { free_operator(c); return st; }
  if ((st = read_ctl(c)) != EI_OK) { free_operator(c); return st; }
  c->alphaA = c->h_ctl->mn;
  c->betaA = c->h_ctl->mx;
  if (!isfinite(c->alphaA) || !isfinite(c->betaA)) { free_operator(c); return EI_ERR_NONFINITE; }
  return EI_OK;
}

ei_status ei_set_operator_csr(ei_ctx* c, int64_t n, int64_t nnz, const int64_t* rowptr,
                              const int32_t* col, const void* val, const void* diag, int prec) {
  if (!c || n < 1 || n > ((int64_t)1 << 31) - 1 || nnz < 0 || !rowptr ||
      (nnz > 0 && (!col || !val)) || (prec != EI_PREC_F64 && prec != EI_PREC_F32))
    return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  cudaStreamSynchronize(c->stream);
  free_operator(c);
  c->kind = KIND_CSR;
  c->prec = prec;
  c->n = n;
  c->nnz = nnz;
  c->val_u = val;
  c->diag_u = diag;
  c->cd = CsrDev{};
  c->cd.n = n;
  c->cd.rowptr = rowptr;
  c->cd.col = col;
  int nb = csr_blocks(n);
  if (nb < reduction_capacity()) nb = reduction_capacity();
  c->max_blocks = nb;
  ei_status st;
  if ((st = alloc((void**)&c->partials, sizeof(double) * 4 * nb)) != EI_OK) { free_operator(c); return st; }
  if ((st = alloc((void**)&c->ger_lo, sizeof(double) * n)) != EI_OK) { free_operator(c); return st; }
  if ((st = alloc((void**)&c->ger_hi, sizeof(double) * n)) != EI_OK) { free_operator(c); return st; }
  // the structure is checked before any kernel reads through rowptr and col
  if (cudaMemsetAsync(&c->ctl->csr_bad, 0, sizeof(int), c->stream) != cudaSuccess ||
      launch_csr_validate(n, nnz, rowptr, col, c->ctl, c->stream) != cudaSuccess) {
    cudaGetLastError();
    free_operator(c);
    return EI_ERR_CUDA;
  }
  if ((st = read_ctl(c)) != EI_OK) { free_operator(c); return st; }
  if (c->h_ctl->csr_bad) { free_operator(c); return EI_ERR_INVALID_ARG; }
  if ((st = build_sell(c)) != EI_OK) { free_operator(c); return st; }
  cudaError_t e = launch_csr_gershgorin(c->cd, prec, val, diag, c->ger_lo, c->ger_hi, c->partials,
                                        c->ctl, c->stream);
  if (e != cudaSuccess) { free_operator(c); return EI_ERR_CUDA; }
  if ((st = prepare(c, prec == EI_PREC_F32 ? VF_F32 : VF_DF)) != EI_OK) { free_operator(c); return st; }
  if ((st = read_ctl(c)) != EI_OK) { free_operator(c); return st; }
  c->alphaA = c->h_ctl->mn;
  c->betaA = c->h_ctl->mx;
  if (!isfinite(c->alphaA) || !isfinite(c->betaA)) { free_operator(c); return EI_ERR_NONFINITE; }
  return EI_OK;
}

ei_status ei_set_dirichlet_values(ei_ctx* c, const void* const faces[6]) {
  if (!c) return EI_ERR_INVALID_ARG;
  if (c->kind != KIND_STENCIL) return EI_ERR_STATE;
  const StencilDev& s = c->sd;
  for (int f = 0; f < 6 && faces; ++f)
    if (faces[f] && (f >= 2 * s.dim || s.bc[f] != EI_BC_DIRICHLET0)) return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  cudaStreamSynchronize(c->stream);
  free_faces(c);
  if (!faces) return EI_OK;
  for (int f = 0; f < 2 * s.dim; ++f) {
    if (!faces[f]) continue;
    const int ax = f / 2;
    const int64_t m = ax == 0 ? (int64_t)s.ny * s.nz : ax == 1 ? (int64_t)s.nx * s.nz
                                                              : (int64_t)s.nx * s.ny;
    ei_status st = alloc((void**)&c->face_term[f], sizeof(double) * m);
    if (st != EI_OK) { free_faces(c); return st; }
    if (launch_face_term(s, f, c->prec, c->dx, c->Du, c->Dc, c->bu[ax], c->bcst[ax], faces[f],
                         c->face_term[f], c->stream) != cudaSuccess) {
      cudaGetLastError();
      free_faces(c);
      return EI_ERR_CUDA;
    }
  }
  // the caller's arrays are read before the call returns
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return EI_OK;
}

ei_status ei_nonlinearity(int nonlin, int prec, int arith, int64_t n, const void* u, void* g,
                          void* dg, void* cuda_stream) {
  if (nonlin < EI_NONLIN_NONE || nonlin > EI_NONLIN_COMBUSTION_FAST ||
      (prec != EI_PREC_F64 && prec != EI_PREC_F32) ||
      (arith != EI_ARITH_DF && arith != EI_ARITH_NATIVE_F64) || n < 0 || (n > 0 && (!u || !g)))
    return EI_ERR_INVALID_ARG;
  if (n == 0) return EI_OK;
  if (launch_nonlinearity(nonlin, prec, arith, n, u, g, dg, (cudaStream_t)cuda_stream) !=
      cudaSuccess) {
    cudaGetLastError();
    return EI_ERR_CUDA;
  }
  return EI_OK;
}

ei_status ei_set_schedule_model(ei_ctx* c, const ei_mlp* model) {
  if (!c) return EI_ERR_INVALID_ARG;
  c->model = model;
  return EI_OK;
}

ei_status ei_estimate_spectrum(ei_ctx* c, double* alpha, double* beta) {
  if (!c || !alpha || !beta) return EI_ERR_INVALID_ARG;
  if (c->kind == KIND_NONE) return EI_ERR_STATE;
  *alpha = c->alphaA;
  *beta = c->betaA;
  return EI_OK;
}

static void acct_begin(ei_ctx* c, const ei_options* opt) {
  c->launches = 0;
  c->newton_timed = 0;
  c->newton_ms = 0.0;
  c->newton_fused = 1;
  c->p_rechecks = 0;
  c->newton_bounded = 0;
  c->coef_table = 0;
  c->profile = opt && opt->profile;
  c->fuse = opt ? opt->single_iter : 0;
  c->csr_lanes = opt ? opt->csr_lanes : 0;
}

static void acct_end(ei_ctx* c, ei_stats* st) {
  if (!st) return;
  st->launches = c->launches;
  st->newton_timed = c->newton_timed;
  st->newton_ms = c->newton_ms;
  st->newton_fused = c->newton_fused;
  st->p_rechecks = c->p_rechecks;
  st->newton_bounded = c->newton_bounded;
  st->coef_table = c->coef_table;
}

static ei_status phi_apply_impl(ei_ctx* c, int k, double h, const void* v, void* out, double tol,
                                const ei_options* opt, ei_stats* st);

ei_status ei_phi_apply(ei_ctx* c, int k, double h, const void* v, void* out, double tol,
                       const ei_options* opt, ei_stats* st) {
  stats_reset(st);
  if (!c || !v || !out) return EI_ERR_INVALID_ARG;
  acct_begin(c, opt);
  ei_status rc = phi_apply_impl(c, k, h, v, out, tol, opt, st);
  acct_end(c, st);
  log_stats("phi_apply", st, rc);
  return rc;
}

// phi_k(hA) v for k >= 2 by s substeps of y' = A y + t^{k-1}/(k-1)! v from 0
// (y(t) = t^k phi_k(tA) v).  A substep of length tau from t_i is
//   y_{i+1} = e^{tau A} y_i + psi_i(tau A) v,
//   psi_i(z) = sum_{j=1..k} t_i^{k-j}/(k-j)! tau^j phi_j(z)
// (variation of constants on the polynomial forcing): a Newton run of
// phi_0 = exp on y_i and one with the divided differences of psi_i (the same
// combination of the phi_j tables) on v.  psi_i is a positive combination,
// so nothing cancels.  The first substep is psi_0 = tau^k phi_k alone.  y_i
// is copied to P.r, a Newton input with a tensor map.  st->degrees holds the
// two runs' degrees summed per substep.
static ei_status phik_substeps(ei_ctx* c, Prepared& P, int k, double h, double cc,
                               double gamma, double tol, const ei_options* opt, ei_stats* st,
                               void* out) {
  const int fmt = P.fmt;
  const int64_t n = c->n;
  const int m_max = (opt && opt->m_max > 0 && opt->m_max <= 100) ? opt->m_max : 100;
  int s = 1, m_pred = 0;
  const bool fixed = opt && opt->fixed_s > 0;
  if (fixed) s = opt->fixed_s;
  else if (schedule(k, h, cc, gamma, tol, m_max, &s, &m_pred, nullptr) != 0)
    return EI_ERR_NOT_CONVERGED;
  if (st) st->m_sched = m_pred;
  const void* qc = base_diag(P);
  const size_t vbytes = vec_elem_bytes(fmt) * (size_t)P.n_alloc;
  std::vector<std::vector<double>> dj(k + 1, std::vector<double>(m_max + 1));
  std::vector<double> dpsi(m_max + 1);
  int restarts = 0;
  while (s <= (1 << 20)) {
    const double tau = h / s;
    for (int j = 0; j <= k; ++j) divided_differences(j, tau, cc, gamma, m_max, dj[j].data());
    bool ok_all = true;
    int dsum = 0, dmax = 0;
    for (int i = 0; i < s; ++i) {
      const double ti = i * tau;
      for (int q = 0; q <= m_max; ++q) dpsi[q] = 0.0;
      double fact = 1.0;  // (k-j)!, from j = k down
      for (int j = k; j >= 1; --j) {
        if (j < k) fact *= (k - j);
        const double bj = pow(ti, k - j) / fact * pow(tau, j);
        for (int q = 0; q <= m_max; ++q) dpsi[q] += bj * dj[j][q];
      }
      int deg = 0, d1 = 0, ok = 0;
      if (i > 0) {  // e^{tau A} y_i
        EI_TRY_CUDA(cudaMemcpyAsync(P.r, P.y, vbytes, cudaMemcpyDeviceToDevice, c->stream));
        EI_TRY(newton_loop(c, P, qc, P.r, dj[0], cc, gamma, tol, m_max, 0, &d1, &ok));
        deg += d1;
        if (!ok) { ok_all = false; break; }
        EI_LAUNCH(launch_p_to_vec(P.y, P.p, fmt, P.n_alloc, c->stream));
      }
      EI_TRY(newton_loop(c, P, qc, P.v, dpsi, cc, gamma, tol, m_max, m_pred, &d1, &ok));
      deg += d1;
      if (!ok) { ok_all = false; break; }
      if (i == 0) {
        if (s > 1) EI_LAUNCH(launch_p_to_vec(P.y, P.p, fmt, P.n_alloc, c->stream));
      } else {
        EI_LAUNCH(launch_axpy(P.y, P.p, fmt, P.n_alloc, 1.0, c->stream));
      }
      if (st) st->matvecs += deg;
      if (st && i < EI_STATS_MAX_SUBSTEPS) st->degrees[i] = deg;
      dsum += deg;
      if (deg > dmax) dmax = deg;
    }
    if (ok_all) {
      if (st) {
        st->s = s; st->restarts = restarts; st->degree_sum = dsum; st->degree_max = dmax;
      }
      const int geo_ny = c->kind == KIND_STENCIL ? c->sd.ny : 1;
      if (s == 1)
        EI_LAUNCH(launch_export(out, c->prec, P.p, fmt, 1, n, geo_nx(c), geo_ny, geo_pitch(c),
                                1.0 / pow(h, k), c->stream));
      else
        EI_LAUNCH(launch_export(out, c->prec, P.y, fmt, 0, n, geo_nx(c), geo_ny, geo_pitch(c),
                                1.0 / pow(h, k), c->stream));
      EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
      return EI_OK;
    }
    if (fixed) return EI_ERR_NOT_CONVERGED;
    ++restarts;
    s *= 2;
  }
  return EI_ERR_NOT_CONVERGED;
}

static ei_status phi_apply_impl(ei_ctx* c, int k, double h, const void* v, void* out, double tol,
                                const ei_options* opt, ei_stats* st) {
  if (c->kind == KIND_NONE) return EI_ERR_STATE;
  if (k < 0 || k > 8 || !(h > 0) || !isfinite(h) || !(tol > 0) || !isfinite(tol))
    return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  const int fmt = vec_fmt_for(c, opt);
  EI_TRY(prepare(c, fmt));
  Prepared& P = c->prep[fmt];
  const int64_t n = c->n;
  EI_LAUNCH(launch_import(P.v, fmt, v, c->prec, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), c->partials, c->ctl,
                         c->stream));
  EI_TRY(read_ctl(c));
  const double alpha = c->alphaA, beta = c->betaA;
  // outside the float-float range (where the format's own squared norm may
  // have overflowed): the native FP64 call, which also checks finiteness
  if (fmt == VF_DF && !(df_rho_ok(alpha, beta) && df_vec_ok(c->h_ctl->vmax))) {
    const ei_options o = native_opts(opt);
    return phi_apply_impl(c, k, h, v, out, tol, &o, st);
  }
  if (c->h_ctl->sum1 != 1.0) return EI_ERR_NONFINITE;
  const double vnorm2 = c->h_ctl->sum0;
  if (st) st->arith_used = fmt == VF_F64 ? EI_ARITH_NATIVE_F64 : EI_ARITH_DF;
  double cc, gamma;
  interval(alpha, beta, &cc, &gamma);
  if (st) { st->alpha = alpha; st->beta = beta; st->s = 1; }
  if (vnorm2 == 0.0) {  // phi_k(hA) 0 = 0
    EI_LAUNCH(launch_export(out, c->prec, P.v, fmt, 0, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), 0.0, c->stream));
    EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    return EI_OK;
  }
  if (gamma == 0.0) {  // A = cI
    EI_LAUNCH(launch_export(out, c->prec, P.v, fmt, 0, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), phi_scalar(k, h * cc),
                         c->stream));
    EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    return EI_OK;
  }
  ei_status rc = EI_OK;
  if (k == 1) {
    const void* res = nullptr;
    int is_p = 0;
    double scale = 1.0;
    c->vnorm2 = vnorm2;
    rc = phi1_substeps(c, P, base_diag(P), h, alpha, beta, tol, opt, st, &res, &is_p, &scale);
    if (rc == EI_OK) {
      EI_LAUNCH(launch_export(out, c->prec, res, fmt, is_p, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), scale / h, c->stream));
      EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    }
  } else if (k >= 2) {
    rc = phik_substeps(c, P, k, h, cc, gamma, tol, opt, st, out);
  } else {
    const int m_max = (opt && opt->m_max > 0 && opt->m_max <= 100) ? opt->m_max : 100;
    int s = 1, m_pred = 0;
    if (opt && opt->fixed_s > 0) s = opt->fixed_s;
    else if (schedule(k, h, cc, gamma, tol, m_max, &s, &m_pred, nullptr) != 0)
      return EI_ERR_NOT_CONVERGED;
    if (st) st->m_sched = m_pred;
    std::vector<double> d(m_max + 1);
    int restarts = 0;
    rc = EI_ERR_NOT_CONVERGED;
    while (s <= (1 << 20)) {  // k = 0: (e^{tau A})^s v
      const double tau = h / s;
      divided_differences(k, tau, cc, gamma, m_max, d.data());
      bool ok_all = true;
      int dsum = 0, dmax = 0;
      const void* cur = P.v;
      for (int i = 0; i < s; ++i) {
        if (i > 0) {
          EI_LAUNCH(launch_p_to_vec(P.r, P.p, fmt, P.n_alloc, c->stream));
          cur = P.r;
        }
        int deg = 0, ok = 0;
        EI_TRY(newton_loop(c, P, base_diag(P), cur, d, cc, gamma, tol, m_max, m_pred, &deg, &ok));
        if (st) st->matvecs += deg;
        if (!ok) { ok_all = false; break; }
        if (st && i < EI_STATS_MAX_SUBSTEPS) st->degrees[i] = deg;
        dsum += deg;
        if (deg > dmax) dmax = deg;
      }
      if (ok_all) {
        if (st) {
          st->s = s; st->restarts = restarts; st->degree_sum = dsum; st->degree_max = dmax;
        }
        EI_LAUNCH(launch_export(out, c->prec, P.p, fmt, 1, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), 1.0, c->stream));
        EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
        rc = EI_OK;
        break;
      }
      ++restarts;
      s *= 2;
    }
  }
  return rc;
}

// phi_k(-i h H) v, H the context's CSR operator (real symmetric), v complex
// (Sec. II-C with K = C).  The interval [alpha, beta] of H and the real Leja
// points are those of the real path; the divided differences of
// f(xi) = phi_k(-i tau (c + gamma xi)) are complex.  k = 0 applies
// e^{-i tau H} s times; k >= 1 takes one substep (s = 1).
static ei_status phi_imag_impl(ei_ctx* c, int k, double h, const void* v, void* out, double tol,
                               const ei_options* opt, ei_stats* st) {
  if (c->kind != KIND_CSR) return EI_ERR_STATE;  // no operator, or a stencil operator
  if (k < 0 || k > 8 || !(h > 0) || !isfinite(h) || !(tol > 0) || !isfinite(tol))
    return EI_ERR_INVALID_ARG;
  if (opt && opt->fixed_s > 1 && k >= 1) return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  const int fmt = vec_fmt_for(c, opt);
  EI_TRY(prepare(c, fmt));
  Prepared& P = c->prep[fmt];
  const int64_t n = c->n;
  if (c->cx_fmt != fmt) {
    for (auto& a : c->cx) {
      if (a) cudaFree(a);
      a = nullptr;
    }
    c->cx_fmt = -1;
    const size_t vb = 2 * vec_elem_bytes(fmt) * (size_t)n, pb = 2 * p_elem_bytes(fmt) * (size_t)n;
    for (int i = 0; i < 5; ++i) {
      ei_status r = alloc(&c->cx[i], i == 4 ? pb : vb);
      if (r != EI_OK) {
        for (auto& a : c->cx) {
          if (a) cudaFree(a);
          a = nullptr;
        }
        return r;
      }
    }
    c->cx_fmt = fmt;
  }
  void* cv = c->cx[0];
  void* cr = c->cx[1];
  CxRun run{nullptr, {c->cx[2], c->cx[3]}, c->cx[4]};
  // a complex vector of n is a real vector of 2n in the same format
  EI_LAUNCH(launch_import(cv, fmt, v, c->prec, 2 * n, (int)(2 * n), 1, (int)(2 * n), c->partials,
                          c->ctl, c->stream));
  EI_TRY(read_ctl(c));
  const double alpha = c->alphaA, beta = c->betaA;
  // outside the float-float range (where the format's own squared norm may
  // have overflowed): the native FP64 call, which also checks finiteness
  if (fmt == VF_DF && !(df_rho_ok(alpha, beta) && df_vec_ok(c->h_ctl->vmax))) {
    const ei_options o = native_opts(opt);
    return phi_imag_impl(c, k, h, v, out, tol, &o, st);
  }
  if (c->h_ctl->sum1 != 1.0) return EI_ERR_NONFINITE;
  const double vnorm2 = c->h_ctl->sum0;
  if (st) st->arith_used = fmt == VF_F64 ? EI_ARITH_NATIVE_F64 : EI_ARITH_DF;
  double cc, gamma;
  interval(alpha, beta, &cc, &gamma);
  if (st) { st->alpha = alpha; st->beta = beta; st->s = 1; }
  if (vnorm2 == 0.0 || gamma == 0.0) {  // 0, or H = cI: phi_k(-i h c) v
    double fr = 0.0, fi = 0.0;
    if (vnorm2 != 0.0) phi_imag(k, -h * cc, &fr, &fi);
    EI_LAUNCH(launch_cexport(out, c->prec, cv, fmt, 0, n, fr, fi, c->stream));
    EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    return EI_OK;
  }
  const int m_max = (opt && opt->m_max > 0 && opt->m_max <= 100) ? opt->m_max : 100;
  int s = 1, m_pred = 0;
  const bool fixed = opt && opt->fixed_s > 0;
  auto& plan = c->cx_plan;
  const bool cached = !fixed && plan.valid && plan.k == k && plan.h == h && plan.cc == cc &&
                      plan.gamma == gamma && plan.tol == tol && plan.m_max == m_max;
  std::vector<double> dd(2 * (m_max + 1)), d(m_max + 1), di(m_max + 1);
  if (fixed) {
    s = opt->fixed_s;
  } else if (cached) {
    s = plan.s;
    m_pred = plan.m_pred;
  } else {
    if (schedule_imag(k, h, cc, gamma, tol, m_max, &s, &m_pred, dd.data()) != 0)
      return EI_ERR_NOT_CONVERGED;
    plan.valid = true;
    plan.k = k;
    plan.h = h;
    plan.cc = cc;
    plan.gamma = gamma;
    plan.tol = tol;
    plan.m_max = m_max;
    plan.s = s;
    plan.m_pred = m_pred;
    plan.dd = dd;
  }
  if (st) st->m_sched = m_pred;
  int restarts = 0;
  while (s <= (1 << 20)) {
    if (k >= 1 && s > 1) return EI_ERR_NOT_CONVERGED;  // one substep only for k >= 1
    const double tau = h / s;
    if (!fixed && plan.valid && plan.k == k && plan.h == h && plan.cc == cc &&
        plan.gamma == gamma && plan.tol == tol && plan.m_max == m_max && plan.s == s)
      dd = plan.dd;  // the rule's own divided differences at this s
    else
      divided_differences_imag(k, tau, cc, gamma, m_max, dd.data());
    for (int j = 0; j <= m_max; ++j) {
      d[j] = dd[2 * j];
      di[j] = dd[2 * j + 1];
    }
    run.d_im = di.data();
    bool ok_all = true;
    int dsum = 0, dmax = 0;
    const void* cur = cv;
    for (int i = 0; i < s; ++i) {
      if (i > 0) {
        EI_LAUNCH(launch_p_to_vec(cr, run.p, fmt, 2 * n, c->stream));
        cur = cr;
      }
      int deg = 0, ok = 0;
      EI_TRY(newton_loop(c, P, base_diag(P), cur, d, cc, gamma, tol, m_max, m_pred, &deg, &ok,
                         &run));
      if (st) st->matvecs += deg;
      if (!ok) { ok_all = false; break; }
      if (st && i < EI_STATS_MAX_SUBSTEPS) st->degrees[i] = deg;
      dsum += deg;
      if (deg > dmax) dmax = deg;
    }
    if (ok_all) {
      if (st) {
        st->s = s; st->restarts = restarts; st->degree_sum = dsum; st->degree_max = dmax;
      }
      EI_LAUNCH(launch_export(out, c->prec, run.p, fmt, 1, 2 * n, (int)(2 * n), 1, (int)(2 * n),
                              1.0, c->stream));
      EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
      return EI_OK;
    }
    if (fixed) return EI_ERR_NOT_CONVERGED;
    ++restarts;
    s *= 2;
  }
  return EI_ERR_NOT_CONVERGED;
}

ei_status ei_phi_apply_imag(ei_ctx* c, int k, double h, const void* v, void* out, double tol,
                            const ei_options* opt, ei_stats* st) {
  stats_reset(st);
  if (!c || !v || !out) return EI_ERR_INVALID_ARG;
  acct_begin(c, opt);
  ei_status rc = phi_imag_impl(c, k, h, v, out, tol, opt, st);
  acct_end(c, st);
  log_stats("phi_apply_imag", st, rc);
  return rc;
}

// One step on the device vector u.  src/dst (optional): the step reads u_n
// from src, keeping a copy in u, and writes u_{n+1} to dst instead of u (a
// mapped host buffer: no separate copies).
static ei_status step_impl(ei_ctx* c, int method, double h, void* u, int nonlin, double tol,
                           const ei_options* opt, ei_stats* st, const void* src = nullptr,
                           void* dst = nullptr) {
  const int fmt = vec_fmt_for(c, opt);
  EI_TRY(prepare(c, fmt));
  Prepared& P = c->prep[fmt];
  const int64_t n = c->n;
  const int rosen = (method == EI_EXP_ROSENBROCK);
  // stencils: F (with any Dirichlet data's face terms), J's diagonal and J's
  // interval in one pass on the TMA z-march
  const bool f_tma = c->kind == KIND_STENCIL;
  // There the native FP64 and FP32 formats read the caller's u in place when
  // it already has the library's layout (rows of a multiple of 4 elements)
  // and a 16-byte aligned base: the import would only copy it (its norm is
  // the F pass's to give, its largest magnitude only float-float's to use).
  bool in_place = f_tma && !src && fmt != VF_DF && c->sd.pitch == c->sd.nx &&
                  (reinterpret_cast<uintptr_t>(u) & 15u) == 0;
  if (in_place && (c->umap_ptr != u || c->umap_fmt != fmt)) {
    in_place = encode_map(&c->umap, u, (int)vec_elem_bytes(fmt), c->sd, 1);
    c->umap_ptr = in_place ? u : nullptr;
    c->umap_fmt = fmt;
  }
  // import u; F = A u + g(u); J's diagonal; the interval of J
  if (!in_place)
    EI_LAUNCH(launch_import(P.u, fmt, src ? src : u, c->prec, n, geo_nx(c),
                            c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), c->partials,
                            c->ctl, c->stream, src ? u : nullptr));
  if (f_tma) {
    NewtonMaps M;
    M.w = in_place ? c->umap : P.map_u;
    for (int k = 0; k < 6; ++k) M.c[k] = P.map_c[k];
    M.c[6] = P.map_diagA;
    M.p = P.map_p;
    FStepArgs fa;
    fa.lo = c->ger_lo;
    fa.hi = c->ger_hi;
    fa.u = u;
    fa.nonlin = nonlin;
    fa.rosen = rosen;
    for (int f = 0; f < 6; ++f) fa.face[f] = c->face_term[f];
    EI_LAUNCH(launch_f_tma(stencil_view(c, P, base_diag(P)), M, P.v, P.qc, fa, fmt,
                           c->partials, c->ctl, c->stream));
    ++P.qc_ver;  // qc now holds this step's J diagonal
  } else {
    EI_LAUNCH(launch_csr_F(csr_view(c, P, P.cbase), P.u, P.v, P.qc, P.cbase, nonlin, rosen,
                             fmt, c->partials, c->ctl, c->stream));
  }
  if (rosen && !f_tma)
    EI_LAUNCH(launch_shifted_minmax(n, c->ger_lo, c->ger_hi, u, c->prec, nonlin, c->partials,
                                      c->ctl, c->stream));
  EI_TRY(read_ctl(c));
  const double alpha = rosen ? c->h_ctl->mn : c->alphaA;
  const double beta = rosen ? c->h_ctl->mx : c->betaA;
  if (fmt == VF_DF && isfinite(alpha) && isfinite(beta) &&
      !df_step_ok(alpha, beta, c->h_ctl->vmax, c->h_ctl->sum1 == 1.0 ? c->h_ctl->sum0 : 0.0)) {
    const ei_options o = native_opts(opt);  // outside the float-float range
    return step_impl(c, method, h, u, nonlin, tol, &o, st, src, dst);
  }
  if (c->h_ctl->sum1 != 1.0) return EI_ERR_NONFINITE;
  const double fnorm2 = c->h_ctl->sum0;
  if (!isfinite(alpha) || !isfinite(beta)) return EI_ERR_NONFINITE;
  if (st) st->arith_used = fmt == VF_F64 ? EI_ARITH_NATIVE_F64 : EI_ARITH_DF;
  if (st) { st->alpha = alpha; st->beta = beta; st->s = 1; st->matvecs = 1; }
  if (fnorm2 == 0.0) return EI_OK;  // u is an equilibrium: u_{n+1} = u_n
  double cc, gamma;
  interval(alpha, beta, &cc, &gamma);
  const void* qc = rosen ? P.qc : base_diag(P);
  if (gamma == 0.0) {  // J = cI: z(h) = h phi_1(hc) F
    EI_LAUNCH(launch_add_export(u, c->prec, P.v, fmt, 0, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c),
                            h * phi_scalar(1, h * cc), c->stream, dst));
    EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
    return EI_OK;
  }
  const void* res = nullptr;
  int is_p = 0;
  double scale = 1.0;
  c->vnorm2 = fnorm2;
  // the scaled operator of the Newton kernels goes out now, so the device
  // makes it while the host works out the schedule
  if (wants_prescale(c, P)) EI_TRY(ensure_prescaled(c, P, qc, cc, gamma));
  EI_TRY(phi1_substeps(c, P, qc, h, alpha, beta, tol, opt, st, &res, &is_p, &scale));
  EI_LAUNCH(launch_add_export(u, c->prec, res, fmt, is_p, n, geo_nx(c), c->kind == KIND_STENCIL ? c->sd.ny : 1, geo_pitch(c), scale, c->stream, dst));
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return EI_OK;
}

ei_status ei_step(ei_ctx* c, int method, double h, void* u, int nonlin, double tol,
                  const ei_options* opt, ei_stats* st) {
  stats_reset(st);
  if (!c || !u) return EI_ERR_INVALID_ARG;
  if (c->kind == KIND_NONE) return EI_ERR_STATE;
  if ((method != EI_EXP_EULER && method != EI_EXP_ROSENBROCK) ||
      nonlin < EI_NONLIN_NONE || nonlin > EI_NONLIN_COMBUSTION_FAST || !(h > 0) || !isfinite(h) ||
      !(tol > 0) || !isfinite(tol))
    return EI_ERR_INVALID_ARG;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  acct_begin(c, opt);
  ei_status rc = step_impl(c, method, h, u, nonlin, tol, opt, st);
  acct_end(c, st);
  log_stats("step", st, rc);
  return rc;
}

ei_status ei_step_host(ei_ctx* c, int method, double h, void* u_host, int nonlin, double tol,
                       const ei_options* opt, ei_stats* st) {
  stats_reset(st);
  if (!c || !u_host) return EI_ERR_INVALID_ARG;
  if (c->kind == KIND_NONE) return EI_ERR_STATE;
  EI_TRY_CUDA(cudaSetDevice(c->device));
  const size_t bytes = (size_t)c->n * (c->prec == EI_PREC_F32 ? 4 : 8);
  if (!c->host_stage) {
    ei_status s = alloc(&c->host_stage, bytes);
    if (s != EI_OK) return s;
  }
  // pinned host memory with a device mapping (GB300's host memory is
  // reachable over NVLink-C2C): the import kernel reads it and the final
  // update writes it directly; other host memory goes through copies
  cudaPointerAttributes attr{};
  const bool mapped = cudaPointerGetAttributes(&attr, u_host) == cudaSuccess &&
                      attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr;
  if (!mapped) cudaGetLastError();
  if (mapped) {
    if ((method != EI_EXP_EULER && method != EI_EXP_ROSENBROCK) ||
        nonlin < EI_NONLIN_NONE || nonlin > EI_NONLIN_COMBUSTION_FAST || !(h > 0) ||
        !isfinite(h) || !(tol > 0) || !isfinite(tol))
      return EI_ERR_INVALID_ARG;
    acct_begin(c, opt);
    ei_status rc = step_impl(c, method, h, c->host_stage, nonlin, tol, opt, st,
                             attr.devicePointer, attr.devicePointer);
    acct_end(c, st);
    log_stats("step_host", st, rc);
    return rc;
  }
  EI_TRY_CUDA(cudaMemcpyAsync(c->host_stage, u_host, bytes, cudaMemcpyHostToDevice, c->stream));
  ei_status rc = ei_step(c, method, h, c->host_stage, nonlin, tol, opt, st);
  if (rc != EI_OK) return rc;
  EI_TRY_CUDA(cudaMemcpyAsync(u_host, c->host_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
  EI_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return EI_OK;
}

}  // extern "C"
