// Internal interface between the host orchestration (ei_api.cpp) and the
// CUDA kernels (ei_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ei {

// Vector element formats inside the library.
enum VecFmt { VF_DF = 0, VF_F64 = 1, VF_F32 = 2 };

// Device-side control block: last-block reduction counter, Newton status and
// the results of the small reductions.  One per context.
struct DevCtl {
  unsigned int count;  // arrivals of the current launch (reset by its last block)
  int done;            // Newton: 0 running, 1 converged, 2 m_max reached, 3 zero input, 4 non-finite
  int degree;          // Newton degree at stop
  int pad;
  double sum0, sum1;   // import / F / residual: squared norm, finiteness flag (1 = finite)
  double mn, mx;       // Gershgorin reductions: min_i (a_ii - r_i), max_i (a_ii + r_i)
  double nw2, np2;     // squared norms of the last Newton iterate / sum
};

// Stencil operator as the kernels see it.  Arrays are in the context's
// vector format (df pairs, double or float); D is pre-scaled by 1/(2 dx_x^2),
// B_e by 1/(2 dx_e); qc is the diagonal term (c_i + g'(u_i)).
struct StencilDev {
  int dim;
  int nx, ny, nz;
  int bc[6];
  const void* D;
  const void* B[3];
  const void* qc;
  double ratio[3];     // k_e / k_x with k_e = 1/(2 dx_e^2)
  int uniform;         // all ratios == 1
};

// CSR operator: y = W x + diag .* x.
struct CsrDev {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;     // W values (double or float, matching the precision)
  const void* qc;      // diagonal (c + g'), in vector format
};

struct NewtonScalars {
  double d_next;       // d_{j+1}
  double d0;           // d_0 (used when j == 0)
  double inv_gamma;    // 1/gamma
  double shift;        // c/gamma + xi_j
  double tol;
  int j;
  int m_max;
};

// ---- launchers (all asynchronous on `st`) ----------------------------------
// number of blocks the stencil kernels use for a grid (partials capacity)
int stencil_blocks(const StencilDev& op);
int csr_blocks(int64_t n);
// upper bound of the block count of every grid-stride (elementwise, CSR) kernel
int reduction_capacity();

// Per-row Gershgorin bounds of the stencil operator A (FP64, from the user's
// arrays), written to lo/hi, and their min/max reduced into ctl->mn/mx.
cudaError_t launch_stencil_gershgorin(const StencilDev& user, int user_prec, const double dx[3],
                                      const void* Duser, double Dconst, const void* const buser[3],
                                      const double bconst[3], const void* cuser, double cconst,
                                      double* lo, double* hi, double* partials, DevCtl* ctl,
                                      cudaStream_t st);
cudaError_t launch_csr_gershgorin(const CsrDev& op, int prec, const void* val_user,
                                  const void* diag_user, double* lo, double* hi,
                                  double* partials, DevCtl* ctl, cudaStream_t st);
// min/max over rows of (lo + q), (hi + q) with q = g'(u) (Rosenbrock), or of lo, hi
cudaError_t launch_shifted_minmax(int64_t n, const double* lo, const double* hi, const void* u,
                                  int prec, int nonlin, double* partials, DevCtl* ctl,
                                  cudaStream_t st);

// Fill a coefficient array in vector format from a user array or a constant,
// times `scale`.
cudaError_t launch_fill_coef(void* dst, int fmt, int64_t n, const void* src, int src_prec,
                             double cst, double scale, cudaStream_t st);

// dst (vector format) = src (user precision); sum of squares into ctl->sum0 and
// a finiteness flag into ctl->sum1 (1 if finite).
cudaError_t launch_import(void* dst, int fmt, const void* src, int src_prec, int64_t n,
                          double* partials, DevCtl* ctl, cudaStream_t st);
// dst (user precision) = scale * src; src in vector format (src_is_p = 0) or
// in the Newton-sum format (src_is_p = 1)
cudaError_t launch_export(void* dst, int dst_prec, const void* src, int fmt, int src_is_p,
                          int64_t n, double scale, cudaStream_t st);
// u (user precision) += scale * y; y in vector or Newton-sum format
cudaError_t launch_add_export(void* u, int prec, const void* y, int fmt, int src_is_p,
                              int64_t n, double scale, cudaStream_t st);
// dst (vector format) = src (Newton-sum format)
cudaError_t launch_p_to_vec(void* dst, const void* p, int fmt, int64_t n, cudaStream_t st);
// y (vector format) += tau * p (p float-float or double)
cudaError_t launch_axpy(void* y, const void* p, int fmt, int64_t n, double tau, cudaStream_t st);
cudaError_t launch_zero(void* x, int fmt, int64_t n, cudaStream_t st);

// Step start: F = A u + g(u) and qc = c + g'(u) (Rosenbrock) or c.  u in vector
// format.  ||F||^2 into ctl->sum0, finiteness into ctl->sum1.
cudaError_t launch_stencil_F(const StencilDev& op, const void* u, void* F, void* qc_out,
                             const void* c_base, int nonlin, int rosenbrock, int fmt,
                             double* partials, DevCtl* ctl, cudaStream_t st);
cudaError_t launch_csr_F(const CsrDev& op, const void* u, void* F, void* qc_out,
                         const void* c_base, int nonlin, int rosenbrock, int fmt,
                         double* partials, DevCtl* ctl, cudaStream_t st);

// r = A y + v (substep residual, A includes qc); ||r||^2 into ctl->sum0.
cudaError_t launch_stencil_residual(const StencilDev& op, const void* y, const void* v, void* r,
                                    int fmt, double* partials, DevCtl* ctl, cudaStream_t st);
cudaError_t launch_csr_residual(const CsrDev& op, const void* y, const void* v, void* r, int fmt,
                                double* partials, DevCtl* ctl, cudaStream_t st);

// One Newton iteration j: w_out = (A w_in)/gamma - shift w_in; p += d_{j+1} w_out;
// norms and the device-side stop test.  Skips itself when ctl->done != 0.
cudaError_t launch_stencil_newton(const StencilDev& op, const void* w_in, void* w_out, void* p,
                                  const NewtonScalars& s, int fmt, double* partials,
                                  DevCtl* ctl, cudaStream_t st);
cudaError_t launch_csr_newton(const CsrDev& op, const void* w_in, void* w_out, void* p,
                              const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                              cudaStream_t st);

// size in bytes of one vector element / of the p element
inline size_t vec_elem_bytes(int fmt) { return fmt == VF_F32 ? 4 : 8; }
inline size_t p_elem_bytes(int fmt) { return 8; }

}  // namespace ei
