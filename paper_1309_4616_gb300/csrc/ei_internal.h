// Internal interface between the host orchestration (ei_api.cpp) and the
// CUDA kernels (ei_kernels.cu, ei_newton_tma.cu).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ei.h"

namespace ei {

// Vector element formats inside the library.
enum VecFmt { VF_DF = 0, VF_F64 = 1, VF_F32 = 2 };

// Device-side control block: last-block reduction counter, Newton status and
// the results of the small reductions.  One per context.
struct DevCtl {
  unsigned int count;  // arrivals of the current launch (reset by its last block)
  int done;            // Newton: 0 running, 1 converged, 2 m_max reached,
                       //         4 non-finite, 5 a bounded device wait ran out,
                       //         6 the norm brackets could not decide (the host
                       //         takes the test with both norms formed)
  int degree;          // Newton degree at stop
  int err;             // set by a block whose bounded wait ran out
  int fixup;           // two-iteration kernel stopped at its first iteration: p holds
                       // p_{j+2}; subtract d_{j+2} w_{j+2} to get p_{j+1}
  int fixfail;         // fixed-count mode: substeps whose final check failed (sticky
                       // across substeps; reset by the host once per call)
  int csr_bad;         // set by the CSR structure check (launch_csr_validate)
  int pad2;
  double sum0, sum1;   // import / F / residual: squared norm, finiteness flag (1 = finite)
  double mn, mx;       // Gershgorin reductions: min_i (a_ii - r_i), max_i (a_ii + r_i)
  double nw2, np2;     // squared norms of the last Newton iterate / sum
  double cs_sum, cs_max, cs_pe;  // coefficient statistics (launch_coef_stats)
  double vmax;         // import: largest magnitude of the imported vector (exact)
};

// Grid geometry of the stencil operator.  Library-owned arrays are stored
// with a padded row pitch (a multiple of 4 elements, so every row starts on a
// 16-byte boundary as TMA requires): element (x, y, z) is at
// (z*ny + y)*pitch + x; padding elements hold zeros.
struct StencilDev {
  int dim;
  int nx, ny, nz, pitch;
  int bc[6];
  const void* a[6];    // neighbour coefficients x-, x+, y-, y+, z-, z+ (0 at a boundary)
  const void* diag;    // diagonal of the operator in use (A, or J = A + diag g'(u))
};

// CSR operator: y = W x + diag .* x.
struct CsrDev {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;     // W values in the vector format
  const void* qc;      // diagonal, in the vector format
};

// Sliced form of a CSR operator (SELL-32-sigma): rows sorted by length
// (longest first) inside windows of kSellWindow consecutive rows, then cut
// into slices of 32; a slice stores its entries column by column (entry k of
// its 32 rows contiguous), padded to its longest row with column -1, value 0.
// A warp takes a slice, a lane a row: the column and value loads of entry k
// are one 32-wide access, independent of any per-row pointer, and a lane
// loads only its own row's entries, so with the rows longest first the lanes
// still loading form a prefix and the padding is never read.  A small window
// keeps a slice's rows close: their w gathers hit nearby lines, and their own
// w, p and diagonal few lines.  On a 2^20-node random geometric graph in Morton
// order, 64 and 128 measured alike in float-float, 32 pads more and 256 and up
// scatter more; native FP64, which pays for padded multiply-adds, ran 63.7
// against 64.8 us an iteration at 128.
constexpr int64_t kSellWindow = 128;
struct SellDev {
  int64_t nslices;
  const int32_t* perm;  // row of each slice position (-1: past the last row), 32 nslices
  const int32_t* rlen;  // entries of the row at each slice position (0 past the last row)
  const int64_t* sptr;  // first entry of each slice, nslices + 1
  const int32_t* col;   // column of each entry (-1: padding)
  const void* val;      // value of each entry in the vector format (0: padding)
  const void* qc;       // diagonal, in the vector format (indexed by row)
};

struct NewtonScalars {
  double d_next;       // d_{j+1}
  double d0;           // d_0 (used when j == 0)
  double inv_gamma;    // 1/gamma
  double shift;        // c/gamma + xi_j
  double tol;
  int j;
  int m_max;
  double d_next2;      // two-iteration kernel: d_{j+2}
  double shift2;       // two-iteration kernel: c/gamma + xi_{j+1}
  int fixed;           // 1: fixed-count mode, m_max steps exactly; only degree m_max
                       //    is tested and a failure counts into ctl->fixfail
  double d_next_im;    // complex Newton sum (k_csr_newton_c): Im d_{j+1}
  double d0_im;        //   and Im d_0
  double xi;           // the Leja point xi_j (kernels on the scaled operator; in
                       // the rescaled basis, xi_j / r)
  double xi2;          // two-iteration kernel on the scaled operator: xi_{j+1} (/ r)
  int bracket;         // 1: this step brackets ||w_{j+1}||^2 and ||p_{j+1}||^2 in
                       //    FP32 instead of forming them in FP64; the stop test
                       //    is decided from the brackets, or reported as done = 6
                       //    where they overlap (the host then forms both norms)
};

// Tensor maps of the TMA-staged Newton kernel (3D maps over the padded
// arrays; x extent = nx, so columns beyond nx and planes outside [0, nz) read
// as zeros).
struct NewtonMaps {
  CUtensorMap w;       // w_in, halo box
  CUtensorMap c[7];    // a[0..5], diag (interior box)
  CUtensorMap p;       // Newton sum, interior box
};

// The step's F pass on the TMA z-march (native FP64 stencils): F = A u + g(u)
// into w_out, with a Rosenbrock step J's diagonal diag(A) + g'(u) into p and
// the interval min/max of (lo + g'(u), hi + g'(u)) over the Gershgorin rows of
// A (lo, hi: contiguous, n entries).
struct FStepArgs {
  const double* lo = nullptr;
  const double* hi = nullptr;
  const void* u = nullptr;  // the caller's u (contiguous; float for FP32 storage):
                            // g'(u) of the interval in the float-float and FP32
                            // formats, taken in FP64 as the separate pass takes it
  int nonlin = 0;
  int rosen = 0;
  // inhomogeneous Dirichlet data: per face x-, x+, y-, y+, z-, z+ the FP64 face
  // terms added at the rows next to it (nullptr: none): x- and x+ faces indexed
  // z * ny + y, y- and y+ faces z * nx + x, z- and z+ faces y * nx + x
  const double* face[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

// ---- launchers (all asynchronous on `st`) ----------------------------------
int csr_blocks(int64_t n);
int reduction_capacity();        // block bound of the grid-stride kernels
int sm_count();                  // SMs of the current device
// the largest block count any TMA Newton launch on this grid uses
int newton_tma_blocks(const StencilDev& op);

// tensor maps: encode one 3D map over a padded array (elem 4 or 8 bytes);
// halo = 1 widens the box by the 16-byte aligned x halo (16/elem_bytes
// columns each side) and one row in y, halo = 2 by the same x halo and two
// rows.
bool encode_map(CUtensorMap* m, const void* base, int elem_bytes, const StencilDev& g, int halo);

// Coefficients of the stencil operator in the vector format (coef7 layout),
// from the caller's arrays (FP64 arithmetic).
cudaError_t launch_stencil_coef(const StencilDev& g, int user_prec, const double dx[3],
                                const void* D, double Dc, const void* const b[3],
                                const double bc[3], const void* c, double cc, void* const a[6],
                                void* diag, int fmt, cudaStream_t st);
// Per-row Gershgorin bounds of the stencil operator A (FP64, from the caller's
// arrays, contiguous layout), written to lo/hi, min/max into ctl->mn/mx.
cudaError_t launch_stencil_gershgorin(const StencilDev& g, int user_prec, const double dx[3],
                                      const void* D, double Dc, const void* const b[3],
                                      const double bc[3], const void* c, double cc, double* lo,
                                      double* hi, double* partials, DevCtl* ctl, cudaStream_t st);
// pointwise nonlinearity over n elements (ei_nonlinearity)
cudaError_t launch_nonlinearity(int nonlin, int prec, int arith, int64_t n, const void* u,
                                void* g, void* dg, cudaStream_t stm);
// CSR structure check: rowptr[0] == 0, rowptr[n] == nnz, rowptr nondecreasing,
// every column in [0, n); a violation sets ctl->csr_bad (reset it first).
cudaError_t launch_csr_validate(int64_t n, int64_t nnz, const int64_t* rowptr,
                                const int32_t* col, DevCtl* ctl, cudaStream_t stm);
cudaError_t launch_csr_gershgorin(const CsrDev& op, int prec, const void* val_user,
                                  const void* diag_user, double* lo, double* hi,
                                  double* partials, DevCtl* ctl, cudaStream_t st);
// min/max over rows of (lo + q), (hi + q) with q = g'(u) (Rosenbrock)
cudaError_t launch_shifted_minmax(int64_t n, const double* lo, const double* hi, const void* u,
                                  int prec, int nonlin, double* partials, DevCtl* ctl,
                                  cudaStream_t st);

// Coefficient statistics of the caller's operator inputs, for the learned
// schedule's features.  Stencil (csr = 0): over the n grid points, sum and max
// of D and max over axes e < dim of |b_e| dx_e / (2 D) (arrays in `prec`, or
// the constants where a pointer is NULL).  CSR (csr = 1): sum and max of
// |diag|.  Into ctl->cs_sum, cs_max, cs_pe.
cudaError_t launch_coef_stats(int64_t n, int csr, int prec, int dim, const void* D, double Dc,
                              const void* const b[3], const double bcst[3], const double dx[3],
                              double* partials, DevCtl* ctl, cudaStream_t st);

// dst (vector format, padded by (nx, ny, pitch)) = scale * (src or cst)
cudaError_t launch_fill_coef(void* dst, int fmt, int64_t n, int nx, int ny, int pitch,
                             const void* src, int src_prec, double cst, double scale,
                             cudaStream_t st);
// dst (vector format, padded) = src (caller precision, contiguous); squared
// norm into ctl->sum0, finiteness flag into ctl->sum1, max |src| into ctl->vmax.
// raw (optional): also copy src there, in the caller's precision
cudaError_t launch_import(void* dst, int fmt, const void* src, int src_prec, int64_t n, int nx,
                          int ny, int pitch, double* partials, DevCtl* ctl, cudaStream_t st,
                          void* raw = nullptr);
// dst (caller precision, contiguous) = scale * src (vector or Newton-sum format)
cudaError_t launch_export(void* dst, int dst_prec, const void* src, int fmt, int src_is_p,
                          int64_t n, int nx, int ny, int pitch, double scale, cudaStream_t st);
// u (caller precision, contiguous) += scale * y (vector or Newton-sum format);
// out (optional): write the sum there instead of into u
cudaError_t launch_add_export(void* u, int prec, const void* y, int fmt, int src_is_p, int64_t n,
                              int nx, int ny, int pitch, double scale, cudaStream_t st,
                              void* out = nullptr);
// elementwise over whole (padded) arrays of n_alloc elements
cudaError_t launch_p_to_vec(void* dst, const void* p, int fmt, int64_t n_alloc, cudaStream_t st);
cudaError_t launch_axpy(void* y, const void* p, int fmt, int64_t n_alloc, double tau,
                        cudaStream_t st);
cudaError_t launch_zero(void* x, int fmt, int64_t n_alloc, cudaStream_t st);
cudaError_t launch_csr_F(const CsrDev& op, const void* u, void* F, void* qc_out,
                         const void* c_base, int nonlin, int rosenbrock, int fmt,
                         double* partials, DevCtl* ctl, cudaStream_t st);

// r = J y + v (substep residual); ||r||^2 into ctl->sum0.
cudaError_t launch_stencil_residual(const StencilDev& op, const void* y, const void* v, void* r,
                                    int fmt, double* partials, DevCtl* ctl, cudaStream_t st);
cudaError_t launch_csr_residual(const CsrDev& op, const void* y, const void* v, void* r, int fmt,
                                double* partials, DevCtl* ctl, cudaStream_t st);

// One Newton iteration j: w_out = (J w_in)/gamma - shift w_in; p += d_{j+1} w_out;
// norms and the device-side stop test.  Skips itself when ctl->done != 0.
// prescaled (native FP64 only): M.c holds the scaled operator (J - cI)/gamma0
// (launch_prescale) and w_out = M.c-product of w_in - s.xi w_in (the caller
// passes s.xi = xi_j gamma/gamma0 and the d_j of the rescaled basis).
cudaError_t launch_newton_tma(const StencilDev& op, const NewtonMaps& M, void* w_out, void* p,
                              const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                              cudaStream_t st, bool prescaled = false);
// inhomogeneous Dirichlet data: the FP64 face term of face f (face coefficient
// x prescribed value, added to A u at the rows next to that face) from the
// caller's values (operator precision prec)
cudaError_t launch_face_term(const StencilDev& g, int face, int prec, const double dx[3],
                             const void* D, double D_const, const void* b_axis,
                             double b_const, const void* vals, double* out, cudaStream_t stm);
// F = A u + g(u) (any EI_NONLIN_*) on the TMA z-march, in the vector format
// fmt (native FP64, float-float or FP32): M.w maps u (halo box), M.c the raw
// coefficients a[0..5]
// and diag(A).  ctl->sum0 gets ||F||^2 and ctl->sum1 its finiteness (1 or 0);
// with fa.rosen, J's diagonal goes to dout and the interval of J to ctl->mn,
// ctl->mx (NaN: -inf, inf).
cudaError_t launch_f_tma(const StencilDev& op, const NewtonMaps& M, void* F, void* dout,
                         const FStepArgs& fa, int fmt, double* partials, DevCtl* ctl,
                         cudaStream_t st);
// ||x||^2 of n_alloc elements of a Newton sum (format fmt) into ctl->sum0
cudaError_t launch_p_sqnorm(const void* x, int fmt, int64_t n_alloc, double* partials,
                            DevCtl* ctl, cudaStream_t st);
// the scaled operator of the Newton kernels (native FP64 and float-float fmt),
// elementwise over the padded arrays: sa[k] = a[k] / gamma (k < 6),
// sa[6] = (diag - c) / gamma
cudaError_t launch_prescale(void* const sa[7], const void* const a[6], const void* diag,
                            int64_t n_alloc, double c, double inv_gamma, int fmt,
                            cudaStream_t st);
// its diagonal alone: sa6 = (diag - c) * inv_gamma
cudaError_t launch_prescale_diag(void* sa6, const void* diag, int64_t n_alloc, double c,
                                 double inv_gamma, int fmt, cudaStream_t st);
// Two Newton iterations j+1 and j+2 in one pass (explicit-coefficient stencil,
// all formats): w_{j+1} is formed on chip over the tile and a one-point
// halo; only w_{j+2} and p_{j+2} are written.  M.w must be a halo-2 map.
// ctab (float-float on the scaled operator only, or null): the operator's
// coefficients as a kConstTab-entry table, for an operator whose D, b and c
// are constants (launch_const_table); the kernel then reads no coefficient
// tiles.
cudaError_t launch_newton2_tma(const StencilDev& op, const NewtonMaps& M, void* w_out, void* p,
                               const NewtonScalars& s, int fmt, double* partials, DevCtl* ctl,
                               cudaStream_t st, bool prescaled = false,
                               const void* ctab = nullptr);
// A stencil operator with constant D, b and c has the same six off-diagonals
// at every point (a neighbour outside the grid multiplies a zero ghost or is
// folded into the diagonal), and its diagonal depends only on the faces the
// point touches: 64 classes cx + 4 cy + 16 cz, bit 0 of each on the low face,
// bit 1 on the high one.  The table holds the off-diagonals a[0..5] at entries
// 0-5 and the diagonal of class k at entry 6 + k, each gathered from the
// coefficient arrays sa[0..6] (vector format) at the padded index idx[entry]
// of one point where it applies (-1: no such point; the entry is 0 and unused).
constexpr int kConstTab = 70;
struct ConstTabIdx {
  int64_t idx[kConstTab];
};
cudaError_t launch_const_table(const void* const sa[7], const ConstTabIdx& ix, void* ctab,
                               int fmt, cudaStream_t st);
// p -= d * w (elementwise, Newton-sum format p, vector format w)
cudaError_t launch_p_fixup(void* p, const void* w, int fmt, int64_t n_alloc, double d,
                           cudaStream_t st);
// lanes: lanes per row (1, 2, 4, 8, 16, 32; any other value: csr_lanes_for's rule)
cudaError_t launch_csr_newton(const CsrDev& op, int64_t nnz, int lanes, const void* w_in,
                              void* w_out, void* p, const NewtonScalars& s, int fmt,
                              double* partials, DevCtl* ctl, cudaStream_t st);
// lanes per row of the CSR Newton kernels: `lanes` when valid, else by the
// mean row length (1 below 8 entries, 2 below 64, 4 below 128, else 8)
int csr_lanes_for(int64_t n, int64_t nnz, int lanes);
// One Newton iteration of a CSR operator in the sliced form (a warp a slice).
cudaError_t launch_csr_newton_sell(const SellDev& op, const void* w_in, void* w_out, void* p,
                                   const NewtonScalars& s, int fmt, double* partials,
                                   DevCtl* ctl, cudaStream_t st);
// The sliced entries from the CSR arrays: src[i] is the CSR entry of sliced
// entry i (-1: padding).  col_out[i] = col[src[i]] (or -1); val_out (vector
// format fmt) = val[src[i]] (caller precision val_prec, or 0).
cudaError_t launch_sell_gather(int64_t e, const int64_t* src, const int32_t* col,
                               int32_t* col_out, const void* val, int val_prec, void* val_out,
                               int fmt, cudaStream_t st);

// Complex vectors for phi_k(-i h H) v, H real symmetric (ei_complex.cu):
// interleaved (re, im) elements of the vector format (df: re.hi, re.lo,
// im.hi, im.lo) and of the Newton-sum format.  A complex vector of n
// elements is a real vector of 2n in the same format, so import, the
// Newton-sum -> vector copy and unscaled export are the real launchers on 2n.
// One Newton step of the CSR operator on complex w with complex d_j
// (s.d_next + i s.d_next_im, s.d0 + i s.d0_im); verdict on |d_{j+1}|.
// lanes: lanes per row (1, 2, 4, 8, 16, 32; other values: by nnz / n).
cudaError_t launch_csr_newton_c(const CsrDev& op, int64_t nnz, int lanes, const void* w_in,
                                void* w_out, void* p, const NewtonScalars& s, int fmt,
                                double* partials, DevCtl* ctl, cudaStream_t st);
// the same on the sliced form of the operator (SellDev)
cudaError_t launch_csr_newton_sell_c(const SellDev& op, const void* w_in, void* w_out, void* p,
                                     const NewtonScalars& s, int fmt, double* partials,
                                     DevCtl* ctl, cudaStream_t st);
// dst = (sr + i si) * src, src a Newton sum (src_is_p) or a vector of format fmt
cudaError_t launch_cexport(void* dst, int prec, const void* src, int fmt, int src_is_p,
                           int64_t n, double sr, double si, cudaStream_t st);

// The schedule network (ei_mlp.cu): outputs (rows x EI_MLP_OUTPUTS, FP32
// rounding) for host feature rows (FP64); synchronises the model's stream.
ei_status mlp_infer_host(const ei_mlp* model, const double* features, int rows, float* out);
const ei_mlp_decision& mlp_decision(const ei_mlp* model);
// The twelve features of a phi_1 call at substep count s (definition in ei.h)
// and the decision rule over the outputs of q = 0..rows-1 (ei_api.cpp).
void learned_features(double* f, double s, double h, double alpha, double beta, double tol,
                      int csr, int dim, int64_t n, double ratio, double pe, double vnorm);
bool learned_decide(const float* outputs, int rows, const ei_mlp_decision& D, int m_max, int* s,
                    int* m);
// the same for any number of rows (staging grows as needed)
ei_status mlp_infer_rows(const ei_mlp* model, const double* features, int64_t rows, float* out);

// size in bytes of one vector element / of one Newton-sum element
inline size_t vec_elem_bytes(int fmt) { return fmt == VF_F32 ? 4 : 8; }
inline size_t p_elem_bytes(int) { return 8; }

}  // namespace ei
