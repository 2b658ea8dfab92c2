/*
 * ei.h — C ABI of the GB300 exponential-integrator library.
 *
 * The library computes the action phi_k(hA)v of the phi-functions of a large
 * sparse matrix A by Newton interpolation at real Leja points on the
 * Gershgorin interval of A, and takes exponential Euler and exponential
 * Rosenbrock-Euler steps with it.  Paper: Einkemmer & Ostermann,
 * "Exponential Integrators on Graphic Processing Units" (HPCS 2013):
 *   - the semilinear problem and the exponential Euler method, Sec. II-C,
 *     Eq. (1)-(2);
 *   - matrix functions by polynomial interpolation on a bound of the field of
 *     values, reduced by Horner's scheme to products (alpha*A + beta*I)x,
 *     Sec. II-C, Eq. (3); interpolation at Leja points, Sec. III-C;
 *   - stencil operators with boundary conditions and position-dependent
 *     coefficients folded into the kernel, Sec. III-A and III-B;
 *   - CSR operators for unstructured A, Sec. III-D.
 *
 * Sign convention: the library integrates u' = A u + g(u).  The paper writes
 * u' + A_p u = g(u), i.e. A = -A_p; the spectrum of A lies in Re <= ~0.
 *
 * General rules for every call:
 *   - Return codes only; nothing is thrown across the ABI.  A failed call
 *     leaves every caller buffer it would have written unmodified and the
 *     context usable.
 *   - Vectors and coefficient arrays are DEVICE pointers on the context's
 *     device, owned by the caller, contiguous, x fastest ([z][y][x]).  The
 *     library keeps coefficient pointers by reference until the next
 *     set_operator or ei_destroy and never frees them.  Workspaces are owned
 *     by the library: allocated by set_operator, freed by ei_destroy.
 *   - All device work is ordered on the context's CUDA stream.  Calls that
 *     return results to the host (spectrum, stats) synchronise that stream.
 *   - Element type of vectors and coefficient arrays follows the operator's
 *     precision: EI_PREC_F64 -> double, EI_PREC_F32 -> float.
 */
#ifndef EI_H
#define EI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ei_ctx ei_ctx; /* opaque, library-owned */

typedef enum {
  EI_OK = 0,
  EI_ERR_INVALID_ARG = 1,   /* bad size, null pointer, k < 0, h <= 0, tol <= 0 ... */
  EI_ERR_NONFINITE = 2,     /* NaN/Inf met in the input vector or the iteration */
  EI_ERR_NOT_CONVERGED = 3, /* no substep count s <= 2^20 met tol */
  EI_ERR_TIMEOUT = 4,       /* a bounded device wait ran out */
  EI_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  EI_ERR_NOMEM = 6,         /* workspace allocation failed */
  EI_ERR_STATE = 7          /* call out of order (e.g. phi_apply before set_operator) */
} ei_status;

/* Boundary condition per face (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi),
 * Sec. III-A: homogeneous conditions folded into the kernel.
 *   DIRICHLET0: ghost value 0 one spacing outside the face (vertex-centred grids).
 *   NEUMANN0:   ghost mirrors the boundary value (cell-centred grids): no
 *               diffusive flux through the face, one-sided advection. */
enum { EI_BC_DIRICHLET0 = 0, EI_BC_NEUMANN0 = 1 };

/* Storage/arithmetic precision of vectors and of the matvec.
 *   F64: vectors exchanged as double; the arithmetic is chosen by
 *        ei_options.arith (below).
 *   F32: vectors and stencil matvec in float with float accumulation; the
 *        divided differences, the spectral interval and the Newton sum p
 *        (float-float) keep FP64-class precision. */
enum { EI_PREC_F64 = 0, EI_PREC_F32 = 1 };

/* Arithmetic of the F64 path (ei_options.arith).
 *   EI_ARITH_DF: the Newton vectors, coefficients and sums are float-float
 *     pairs (hi + lo floats: a 48-bit significand with FP32's exponent range)
 *     on the FP32 pipes, which GB300 runs far faster than its FP64 pipe.  The
 *     format matches native FP64 only inside its range, so a call runs in it
 *     only when the operator's bound rho = max(|alpha|, |beta|) lies in
 *     [2^-60, 2^60] (or is 0) and the vector it acts on (v, or u for a step)
 *     has max |x| in [2^-60, 2^50] (or is zero); a step also needs
 *     max |u| <= 2^20, rho max|u| <= 2^40 and ||A u + g(u)||^2 in
 *     [2^-60, 2^100].  Any other call runs in native FP64, and
 *     ei_stats.arith_used says which arithmetic ran.
 *   EI_ARITH_NATIVE_F64: every vector value in IEEE double.  On stencil
 *     operators the Newton steps after a loop's first bracket the squared
 *     norms of the stop test in FP32, with proven bounds, and take any test
 *     the brackets cannot decide with FP64 norms (ei_stats.p_rechecks): each
 *     decision is the one the exact norms give. */
enum { EI_ARITH_DF = 0, EI_ARITH_NATIVE_F64 = 1 };

enum { EI_EXP_EULER = 0, EI_EXP_ROSENBROCK = 1 };
/* g = 0 | g = u(1-u) | the combustion term of Sec. III-C,
 * g = (2-u) e^{20(1-1/u)}/4, at the format's precision | the same with FP32
 * hardware approximations of exp and division (the paper's fast math) */
enum { EI_NONLIN_NONE = 0, EI_NONLIN_LOGISTIC = 1, EI_NONLIN_COMBUSTION = 2,
       EI_NONLIN_COMBUSTION_FAST = 3 };

typedef struct {
  int m_max;      /* largest Newton degree per substep; 0 -> 100 (max 100) */
  int arith;      /* EI_ARITH_*, F64 operators only; default EI_ARITH_DF */
  int fixed_s;    /* > 0: use this substep count instead of the a-priori rule */
  int profile;    /* 1: time every Newton-iteration launch with CUDA events on the
                     context's stream (stats.newton_ms / newton_timed) */
  int single_iter; /* Newton iterations per stencil kernel launch: 0 the format's
                      default (two for float-float and FP32, whose kernels HBM
                      bounds; one for native FP64, which its FP64 arithmetic
                      bounds); 1 one; 2 two */
  int tile_rows;   /* batched form: height in rows (1 to 1024) of a strip, the
                      32-column unit of work of one warp; 0 = the autotuner's
                      choice */
  int learned;     /* phi_1 schedule: 0 the plain a-priori rule; 1 the learned
                      schedule of the model set by ei_set_schedule_model, adaptive
                      (the proposal's s, the per-substep a posteriori stop; m sets
                      the launches issued before the first look); 3 the learned
                      schedule with a fixed count of m steps per substep; both fall
                      back to the plain rule; 2 the plain rule, reporting
                      stats.features */
  int no_restart;  /* with fixed_s: an attempt that reaches m_max returns
                      EI_ERR_NOT_CONVERGED instead of doubling s (stats keep the
                      degrees reached; u and out are left unmodified) */
  int csr_lanes;   /* CSR operators' Newton kernels (real and complex): 0
                      (default) runs on the sliced copy the library builds at
                      set_operator (rows sorted by length within windows of 64,
                      slices of 32 stored column by column: a warp a slice, a
                      lane a row, every column and value load one coalesced
                      access); 1, 2, 4, 8, 16 or 32 run on the caller's CSR
                      arrays with that many lanes of a warp per row; any other
                      value chooses the lanes by the mean row length (1 below
                      8 entries, 2 below 64, 4 below 128, else 8). */
} ei_options;

#define EI_STATS_MAX_SUBSTEPS 64
typedef struct {
  double alpha, beta;   /* Gershgorin interval used */
  int s;                /* substeps of the accepted attempt */
  int restarts;         /* attempts rejected (m_max reached) before it */
  int matvecs;          /* operator applications, all attempts */
  int degree_sum;       /* sum of Newton degrees of the accepted attempt */
  int degree_max;
  int m_sched;          /* degree the a-priori rule predicted */
  int degrees[EI_STATS_MAX_SUBSTEPS]; /* per substep, first 64 substeps */
  int launches;         /* kernels this call launched */
  int newton_timed;     /* Newton-iteration launches timed (options.profile) */
  int newton_fused;     /* Newton iterations per timed launch (1 or 2) */
  double newton_ms;     /* their summed device time (launches that did work) */
  int learned;          /* 0 plain rule; 1 learned proposal accepted; 2 proposal
                           failed its check (plain fallback); 3 no q accepted
                           (plain); 4 features only (options.learned = 2) */
  int learned_s;        /* the proposal (learned = 1 or 2) */
  int learned_m;
  int learned_pad;
  double features[12];  /* features of the call at the substep count used
                           (options.learned != 0); see ei_mlp below */
  int arith_used;       /* EI_ARITH_* the Newton iteration ran in (F64 operators;
                           a float-float call outside the format's range runs
                           in native FP64) */
  int p_rechecks;       /* native FP64 stencils: Newton steps after the first
                           bracket ||w|| and ||p|| in FP32 and take the stop
                           test from the brackets; steps whose brackets could
                           not decide, where the host formed both norms to
                           take the test */
  int newton_bounded;   /* of the newton_timed launches, those that bracketed
                           the norms */
  int coef_table;       /* stencil operators whose D, b and c are all constants
                           (float-float): two-iteration Newton launches that
                           read the operator from a table of 70 coefficients
                           (six off-diagonals, the diagonal of each of the 64
                           classes of points by the faces they touch) instead
                           of the seven coefficient arrays */
} ei_stats;

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context; on error *out is NULL. */
ei_status ei_create(ei_ctx** out, int device, void* cuda_stream);

/* Destroy the context and free its workspaces (after a stream sync). */
void ei_destroy(ei_ctx* ctx);

/* Change the stream later calls are ordered on. */
ei_status ei_set_stream(ei_ctx* ctx, void* cuda_stream);

/* Stencil operator, Sec. III-A (seven-point formula) and III-B
 * (position-dependent diffusion), conservative form:
 *   (A u)_i = sum_e [ D_{i+e/2}(u_{i+e} - u_i) + D_{i-e/2}(u_{i-e} - u_i) ] / dx_e^2
 *           + sum_e b_e,i (u_{i+e} - u_{i-e}) / (2 dx_e) + c_i u_i,
 *   D_{i+e/2} = (D_i + D_{i+e}) / 2  (at a face, the ghost D is D_i).
 * dim      2 or 3 (dim 2: n[2], dx[2], b[2], bc[4..5] are ignored).
 * n        grid points per axis (x, y, z), each >= 1.
 * dx       spacing per axis, > 0.
 * D        device array of n0*n1*n2 values, or NULL to use D_const.
 * b        three device arrays or NULLs; a NULL component uses b_const[e].
 * c        device array or NULL to use c_const (a fixed diagonal term).
 * bc       six face codes EI_BC_*.
 * prec     EI_PREC_F64 (arrays of double) or EI_PREC_F32 (arrays of float).
 * Allocates the library's workspaces (about 8 vectors of the grid size).
 * With D, every b component and c given as constants (NULL arrays), the
 * float-float Newton iterations on A (ei_phi_apply, exponential Euler) read
 * the operator from a table of 70 coefficients instead of its coefficient
 * arrays (ei_stats.coef_table); results agree with the array form to the
 * format's rounding. */
ei_status ei_set_operator_stencil(ei_ctx* ctx, int dim, const int64_t n[3], const double dx[3],
                                  const void* D, double D_const, const void* const b[3],
                                  const double b_const[3], const void* c, double c_const,
                                  const int bc[6], int prec);

/* Sparse operator in CSR, Sec. III-D: A = W + diag(diag).
 * rowptr  int64[n+1] (device), nondecreasing from rowptr[0] = 0 to
 *         rowptr[n] = nnz; col int32[nnz] (device), each in [0, n);
 *         val[nnz] (device).  The structure is checked on the device before
 *         use: a violation returns EI_ERR_INVALID_ARG.  The library then
 *         builds a sliced copy of the structure (host sort of the row
 *         lengths, about 20 bytes per entry of device memory; the values are
 *         copied per format on first use) for the real Newton kernel.
 * diag    device array of n values or NULL (zero).  Entries with col == row
 *         are allowed and count as diagonal.  prec as above. */
ei_status ei_set_operator_csr(ei_ctx* ctx, int64_t n, int64_t nnz, const int64_t* rowptr,
                              const int32_t* col, const void* val, const void* diag, int prec);

/* Gershgorin interval of the operator (FP64):
 *   alpha = min_i (a_ii - r_i),  beta = max_i (a_ii + r_i),  r_i = sum_{j!=i} |a_ij|.
 * Sec. II-C of the paper presupposes a bound on the field of values that is
 * available in advance; this interval is that bound for the real-Leja
 * method.  Host outputs. */
ei_status ei_estimate_spectrum(ei_ctx* ctx, double* alpha, double* beta);

/* Gershgorin interval of a stencil operator, computed with no device memory
 * allocation at all.  (The paper has no counterpart: this entry exists for
 * callers that must not allocate.)  Callers that cannot call cudaMalloc:
 * real-time or budgeted code that reserves all device memory up front (an
 * allocation there can fail or stall on a device-wide synchronisation), and
 * hosts whose framework owns the GPU's memory through its own pool allocator.
 * The arguments describe the operator exactly as for ei_set_operator_stencil
 * (device arrays or constants); the result equals the ei_estimate_spectrum
 * interval of that operator.  No context is needed.
 *   device, cuda_stream: where the reduction runs; the caller's current device
 *     is restored before returning.  The call synchronises the stream.
 *   alpha, beta: host outputs.
 * Scratch: a fixed ~256 KB array inside the library, one per GPU that loads
 * the library, held until the process exits.  It bounds the operator to
 * n0*n1*n2 <= 2^27 points (512^3); larger operators return
 * EI_ERR_INVALID_ARG.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress, with that device current) and keeps it
 * for the life of the process, so that first call should come before any
 * stream capture; after cudaDeviceReset the kept address is stale, so do not
 * call this entry point on a device that was reset.
 * Every call shares the array and the call clears its arrival counter first:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.
 * Errors: EI_ERR_INVALID_ARG (bad arguments, too many points), EI_ERR_CUDA,
 * EI_ERR_NONFINITE (NaN/Inf in the coefficients). */
ei_status ei_estimate_spectrum_stencil_noalloc(int device, void* cuda_stream, int dim,
                                               const int64_t n[3], const double dx[3],
                                               const void* D, double D_const,
                                               const void* const b[3], const double b_const[3],
                                               const void* c, double c_const, const int bc[6],
                                               int prec, double* alpha, double* beta);

/* out = phi_k(hA) v  (Eq. (2) for k = 1; phi_0 = exp).  v, out: device
 * vectors of the operator's size and precision; they may alias.
 * k = 1: substepped ODE form; k = 0: (e^{(h/s)A})^s v; k >= 2 (k <= 8): s
 * substeps of y' = A y + t^{k-1}/(k-1)! v from 0, each
 * y_{i+1} = e^{tau A} y_i + psi_i(tau A) v with psi_i a positive combination
 * of tau^j phi_j (two Newton runs; stats.degrees sums them per substep).
 * tol: relative stop tolerance of the a-posteriori estimate
 *   |d_{j+1}| ||w_{j+1}||_2 <= tol ||p_{j+1}||_2, per substep.
 * k = 1 with the a-priori rule: the context keeps the rule's last plan (s, its
 * degree estimate, the divided differences at h/s) and reuses it for a call
 * with the same h, tol and m_max on the same interval (bit-identical results;
 * only host time is saved).  Setting an operator clears it.
 * opt may be NULL (defaults).  stats may be NULL. */
ei_status ei_phi_apply(ei_ctx* ctx, int k, double h, const void* v, void* out, double tol,
                       const ei_options* opt, ei_stats* stats);

/* out = phi_k(-i h H) v for the context's CSR operator H, read as a real
 * symmetric (Hermitian) matrix: the products (alpha A + beta I) x of Eq. (3)
 * with K = C (Sec. II-C), for psi' = -i H psi (the spin system of
 * Sec. III-D).  The interpolation runs on H's Gershgorin interval
 * [alpha, beta] with the real Leja points; the divided differences of
 * f(xi) = phi_k(-i tau (c + gamma xi)) are complex (ei_divided_differences_imag)
 * and the Newton basis is H's real recurrence applied to complex vectors.
 *   v, out: device arrays of n complex numbers, interleaved (re, im): double
 *     pairs for EI_PREC_F64 (16-byte aligned), float pairs for EI_PREC_F32
 *     (8-byte aligned); they may alias.  Read and written on the context's
 *     stream; the call synchronises it.
 *   k = 0: (e^{-i (h/s) H})^s v, s from ei_schedule_imag (or opt->fixed_s);
 *     k >= 1 (k <= 8): one substep, s = 1.
 *   tol: per-substep stop rule |d_{j+1}| ||w_{j+1}||_2 <= tol ||p_{j+1}||_2
 *     with |d| the complex modulus and 2-norms over both parts.
 * The context keeps the last plan (s, the degree estimate, the divided
 * differences) and reuses it for a call with the same k, h, tol and m_max:
 * bit-identical results, less host time.  Setting an operator clears it.
 * Only the operator's symmetry is assumed, not checked: for a non-symmetric
 * operator the interval does not bound the spectrum and the result is not
 * phi_k(-i h H) v.
 * Errors: EI_ERR_STATE (no operator, or a stencil operator),
 * EI_ERR_INVALID_ARG (k, h, tol; opt->fixed_s > 1 with k >= 1),
 * EI_ERR_NONFINITE (NaN/Inf in v or in the iteration), EI_ERR_NOT_CONVERGED
 * (k >= 1 needing s > 1, or no s <= 2^20), EI_ERR_NOMEM (the five complex
 * workspaces, allocated on first use per format), EI_ERR_CUDA. */
ei_status ei_phi_apply_imag(ei_ctx* ctx, int k, double h, const void* v, void* out, double tol,
                            const ei_options* opt, ei_stats* stats);

/* One step of size h of u' = A u + g(u), in place on the device vector u.
 * method EI_EXP_EULER:      u <- u + h phi_1(hA)(A u + g(u))          (Eq. (2))
 * method EI_EXP_ROSENBROCK: u <- u + h phi_1(hJ)(A u + g(u)), J = A + diag(g'(u))
 * nonlin EI_NONLIN_*: g = 0, u(1-u), or the combustion term of Sec. III-C
 *        (g and g' fused into the kernel that forms A u + g(u); the full form
 *        at the format's precision, float-float for EI_ARITH_DF; the fast form
 *        in FP32 with __expf / __fdividef). */
ei_status ei_step(ei_ctx* ctx, int method, double h, void* u, int nonlin, double tol,
                  const ei_options* opt, ei_stats* stats);

/* ei_step on a HOST vector of the operator's size and precision, on the
 * context's stream.  Pinned host memory with a device mapping (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) is read by the import kernel and written
 * by the final update directly (over NVLink-C2C on GB300), with a device copy
 * of u_n kept for the step; other host memory is copied in and out.  Either
 * way u_host holds u_{n+1} when the call returns, and is unchanged on error. */
ei_status ei_step_host(ei_ctx* ctx, int method, double h, void* u_host, int nonlin, double tol,
                       const ei_options* opt, ei_stats* stats);

/* Inhomogeneous Dirichlet data (Sec. III-A: boundary functions f on the
 * faces of the domain).  faces[f], f < 2*dim (f = 2*axis + side, side 0 the
 * lower face): NULL (homogeneous: ghost value 0) or a device array of the
 * prescribed values at the face's ghost points, in the operator's precision:
 *   faces 0, 1 (x = lower, upper): ny*nz values, index z*ny + y;
 *   faces 2, 3 (y): nx*nz values, index z*nx + x;
 *   faces 4, 5 (z, 3D only): nx*ny values, index y*nx + x.
 * The arrays are read before the call returns (the library keeps its own
 * FP64 face terms: face coefficient D_i/dx^2 +- b_i/(2dx) x value).
 * Effect: ei_step forms A u + b_D + g(u), b_D the face terms at the rows next
 * to each face; b_D is a constant forcing, so the Newton loop, the Rosenbrock
 * Jacobian and ei_phi_apply use the linear A.  faces == NULL (or all NULL)
 * clears the data; ei_set_operator_* clears it too.
 * Errors: EI_ERR_STATE without a stencil operator; EI_ERR_INVALID_ARG for
 * data on a Neumann face or on a face beyond 2*dim. */
ei_status ei_set_dirichlet_values(ei_ctx* ctx, const void* const faces[6]);

/* Pointwise nonlinearity, Sec. III-C (the paper's Table 3 times exactly this
 * evaluation): g[i] = g(u[i]) and, when dg is not NULL, dg[i] = g'(u[i]),
 * for 0 <= i < n.
 *   nonlin  EI_NONLIN_* (NONE gives zeros).
 *   prec    EI_PREC_F64 (double arrays) or EI_PREC_F32 (float arrays).
 *   arith   FP64 arrays only: EI_ARITH_DF evaluates in float-float on the
 *           FP32 pipes, EI_ARITH_NATIVE_F64 with the FP64 math library.
 *   u, g, dg  device arrays of n elements, caller-owned; g or dg may alias u.
 *   cuda_stream  the kernel is queued there; the call does not synchronise.
 * Errors: EI_ERR_INVALID_ARG for an unknown nonlin, prec or arith, n < 0, or
 * a NULL u or g with n > 0; EI_ERR_CUDA if the launch fails. */
ei_status ei_nonlinearity(int nonlin, int prec, int arith, int64_t n, const void* u, void* g,
                          void* dg, void* cuda_stream);

/* Host-side pieces of the method, exported for inspection and tests. */
/* Leja points xi_0..xi_m on [-2,2]: xi_0 = 2, xi_j maximises prod_{i<j}|x - xi_i|,
 * ties to the larger x.  out: host array of m+1 doubles, m <= 100. */
ei_status ei_leja_points(int m, double* out);
/* Divided differences d_j = f[xi_0..xi_j], f(xi) = phi_k(tau*c + tau*gamma*xi),
 * j = 0..m (m <= 100), by Opitz's theorem: the first column of
 * phi_k(tau*c*I + tau*gamma*Z), Z lower bidiagonal (diag xi, subdiag 1),
 * evaluated by scaling and squaring on a shifted nonnegative matrix.  Host out. */
ei_status ei_divided_differences(int k, double tau, double c, double gamma, int m, double* out);
/* The a-priori substep rule: smallest s = 2^q such that some degree <= m_max
 * meets max_G |f - p_m| <= tol max_G |f| on 2001 points G of [-2,2]. */
ei_status ei_schedule(int k, double h, double c, double gamma, double tol, int m_max,
                      int* s_out, int* m_out);
/* The skew case of ei_phi_apply_imag: d_j of f(xi) = phi_k(-i tau (c + gamma xi)),
 * complex, j = 0..m (m <= 100), from Opitz's matrix with complex entries
 * (scaling, a Taylor polynomial and squaring).  out: host array of 2(m+1)
 * doubles, interleaved (Re d_j, Im d_j). */
ei_status ei_divided_differences_imag(int k, double tau, double c, double gamma, int m,
                                      double* out);
/* The a-priori rule of ei_schedule with that complex f (max_G |f - p_m| with
 * the complex modulus). */
ei_status ei_schedule_imag(int k, double h, double c, double gamma, double tol, int m_max,
                           int* s_out, int* m_out);

/* ---- Learned schedule ------------------------------------------------------
 * A small network proposes the substep count and the Leja degree of a phi_1
 * call instead of the conservative a priori rule (Sec. III-C); the a
 * posteriori estimate still accepts or rejects the proposal.  Network:
 * EI_MLP_INPUTS inputs, three hidden layers of 64 with ReLU, EI_MLP_OUTPUTS
 * linear outputs, FP32, parameters one flat vector (per layer W, out x in,
 * row major, then b).  For candidate q = 0..q_max (s = 2^q) output 0 is the
 * degree the estimate will need as a fraction of m_max and output 1 the logit
 * of meeting it within m_max.  A candidate q is accepted when o1 >= z_min and
 * need = m_max o0 (1 + rho_m) + delta_m <= m_max, with
 * m_q = clamp(ceil(need), 1, m_max); the call takes the accepted q with the
 * fewest operator applications 2^q (m_q + 1) - 1 (ties: the smaller q), runs
 * s = 2^q substeps.  Adaptive mode (ei_options.learned = 1) ends every
 * substep at the first degree whose estimate |d_j| ||w_j|| <= tol ||p_j||
 * passes, as the plain method does, after issuing m_q steps before the first
 * look; a substep reaching m_max sends the call to the plain method.  Fixed
 * count (learned = 3) runs exactly m_q Newton steps in each substep with no
 * test in between and checks the estimate once per substep.  Any failed
 * check, or no accepted q, redoes the call by the plain method.
 * Features of a call with interval [alpha, beta], c = (alpha+beta)/2,
 * gamma = (beta-alpha)/4, tau = h/s, rho = max(|alpha|, |beta|):
 *   0 log10(tau gamma)        1 clip(c/gamma, -8, 8)/4   2 log10(tol)/10
 *   3 log2(s)/10              4 log10(h rho)/3           5 k (1)
 *   6 1 for CSR, else 0       7 dim/3 (CSR: 0)
 *   8 coefficient ratio: stencil mean(D)/max(D); CSR mean|diag|/max|diag|
 *   9 log10(1 + min(Pe, 1e30)), Pe = max over points and axes of
 *     |b_e| dx_e / (2 D) (stencil), 0 (CSR)
 *  10 clip(log10(||v||_2 / sqrt(n)), -30, 30)/10    11 log10(n)/8
 * (v is the vector phi_1 acts on: the input of ei_phi_apply, F_n of ei_step). */
#define EI_MLP_INPUTS 12
#define EI_MLP_OUTPUTS 2
#define EI_MLP_PARAMS 9282
#define EI_MLP_MAX_Q 12

typedef struct ei_mlp ei_mlp; /* opaque, library-owned: parameters and Adam state */

typedef struct {
  double z_min;    /* acceptance threshold on output 1 (a logit) */
  double rho_m;    /* relative margin on the predicted degree, >= 0 */
  double delta_m;  /* absolute margin on the predicted degree */
  int q_max;       /* largest candidate q, 0..EI_MLP_MAX_Q */
  int pad;
} ei_mlp_decision;

/* Create a network on `device` (parameters zero; decision z_min 0, rho_m 0.05,
 * delta_m 2, q_max EI_MLP_MAX_Q), ordering its work on `cuda_stream`. */
ei_status ei_mlp_create(ei_mlp** out, int device, void* cuda_stream);
void ei_mlp_destroy(ei_mlp* m);
/* Parameters from / to a host array of EI_MLP_PARAMS floats.  Setting them
 * clears the Adam state.  Non-finite values: EI_ERR_NONFINITE. */
ei_status ei_mlp_set_params(ei_mlp* m, const float* theta);
ei_status ei_mlp_get_params(ei_mlp* m, float* theta);
ei_status ei_mlp_set_decision(ei_mlp* m, const ei_mlp_decision* d);
ei_status ei_mlp_get_decision(const ei_mlp* m, ei_mlp_decision* d);
/* out (device, rows x EI_MLP_OUTPUTS) = network(x) for x (device,
 * rows x EI_MLP_INPUTS, row major).  Asynchronous on the model's stream. */
ei_status ei_mlp_forward(ei_mlp* m, const float* x, int64_t rows, float* out);
/* Loss of a batch and its gradient: x as above, y (device, rows x 2: target
 * degree fraction, converged 0/1), mask (device, rows: 1 where y[.,0] is
 * defined).  loss = mean over rows of mask k(e) e^2 + lam (softplus(o1) - y1 o1),
 * e = o0 - y0, k = kappa if e < 0 else 1.  grad: device, EI_MLP_PARAMS floats.
 * *loss (host, may be NULL) is written after a stream synchronisation. */
ei_status ei_mlp_loss_grad(ei_mlp* m, const float* x, const float* y, const float* mask,
                           int64_t rows, double lam, double kappa, double* loss, float* grad);
/* One Adam step (b1 0.9, b2 0.999, eps 1e-8, learning rate lr) on the batch's
 * gradient.  *loss (may be NULL) receives the batch loss before the step. */
ei_status ei_mlp_train_step(ei_mlp* m, const float* x, const float* y, const float* mask,
                            int64_t rows, double lam, double kappa, double lr, double* loss);
/* Use `model` (NULL: none) for calls with ei_options.learned = 1.  The
 * context keeps the pointer; the caller keeps the model alive meanwhile. */
ei_status ei_set_schedule_model(ei_ctx* ctx, const ei_mlp* model);

/* ---- Batched form ---------------------------------------------------------
 * Many independent problems of uneven size, each a 2D stencil operator with
 * constant coefficients (the rows of Sec. III-A with constant D, b, c and its
 * own per-side homogeneous boundary conditions), advanced together: all the
 * phi_1(h_i A_i) v_i are computed by ONE persistent kernel launch, replayed
 * from a captured CUDA graph.  Blocks claim (problem, tile) work items from a
 * device work queue; the block that finishes a problem's last tile reduces
 * its norms in tile order, takes the stop test and publishes the problem's
 * next phase, so no block ever waits for another.  Tile heights per
 * problem-size class come from a built-in autotuner (timed on the device the
 * first time a class is seen, cached per process and device). */
typedef struct {
  int64_t nx, ny;   /* grid points, each >= 1 */
  double dx, dy;    /* spacings, > 0 */
  double D;         /* diffusion coefficient */
  double bx, by;    /* advection b (the operator uses + b . grad u) */
  double c;         /* reaction/diagonal term */
  int bc[4];        /* EI_BC_* of faces x-lo, x-hi, y-lo, y-hi */
  double h;         /* step, > 0 */
} ei_batch_problem;

typedef struct {
  double alpha, beta; /* Gershgorin interval */
  int s;              /* substeps of the accepted attempt */
  int degree_sum;     /* Newton degrees summed over substeps */
  int restarts;       /* attempts rejected (m_max reached) */
  int tile_rows;      /* strip height (rows) the autotuner chose for its size class */
  int learned;        /* with a schedule model: 1 the network's s kept, 2 it reached
                         m_max and the a-priori rule took over, 0 no q accepted */
  int pad;
} ei_batch_stats;

typedef struct ei_batch ei_batch; /* opaque, library-owned */

/* Set up `count` problems on `device`: per-problem Gershgorin interval,
 * a-priori schedule and divided differences (host, FP64), workspaces for all
 * problems in one device pool, and the tile choice.  prec: EI_PREC_F64 or
 * EI_PREC_F32 (vectors and matvec in float).  tol: Leja tolerance for every
 * problem.  opt may be NULL.  Synchronous. */
ei_status ei_batch_create(ei_batch** out, int device, int count, const ei_batch_problem* problems,
                          int prec, double tol, const ei_options* opt);
/* offsets[0..count]: element offsets of each problem's vector in the packed
 * layout ei_batch_phi1 reads and writes (problem i occupies
 * [offsets[i], offsets[i+1]), x fastest).  Host array. */
ei_status ei_batch_offsets(const ei_batch* b, int64_t* offsets);
/* out_i = phi_1(h_i A_i) v_i for every problem.  v, out: device arrays in the
 * packed layout, in the batch's precision; ordered on `cuda_stream`.  The
 * first call captures the launch sequence into a CUDA graph, later calls
 * replay it.  per_problem: host array of `count` stats, or NULL.  Returns
 * after completion. */
ei_status ei_batch_phi1(ei_batch* b, void* cuda_stream, const void* v, void* out,
                        ei_batch_stats* per_problem);
/* The persistent kernel's bounded wait: a warp that finds no work to claim
 * gives up after limit_us microseconds without progress anywhere in the batch
 * (<= 0: the default, 5 s); ei_batch_phi1 then returns EI_ERR_TIMEOUT.  A
 * pass never waits on a warp, so a healthy pass only meets a limit far below
 * its own strips' durations (a test sets one to see the error path).  On a
 * timeout in the first pass out is left unmodified; in a rerun of restarted
 * problems out holds the problems that converged in the first pass.  The
 * next call runs with the new limit (its graph is re-captured). */
ei_status ei_batch_set_wait_limit(ei_batch* b, int64_t limit_us);
/* Plan every later ei_batch_phi1 call with the schedule network `model`
 * (NULL: the a-priori rule), in the adaptive mode of ei_options.learned = 1:
 * per problem the network's substep count with the per-substep a posteriori
 * stop; a problem whose proposal reaches m_max is redone with the a-priori
 * rule.  The plan is made at each call (it depends on ||v_i||); divided
 * differences are kept per problem and substep count.  A batch created with
 * ei_options.learned = 1 skips the a-priori plans at creation. */
ei_status ei_batch_set_schedule_model(ei_batch* b, const ei_mlp* model);
void ei_batch_destroy(ei_batch* b);

const char* ei_status_string(ei_status st);

#ifdef __cplusplus
}
#endif
#endif /* EI_H */
