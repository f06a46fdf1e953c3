/*
 * gpe.h -- C ABI of libgpe: the hot path of the preconditioned nonlinear
 * conjugate gradient method (PCG_C) of Antoine, Levitt and Tang,
 * "Efficient spectral computation of the stationary states of rotating
 * Bose-Einstein condensates by the preconditioned nonlinear conjugate
 * gradient method" (arXiv:1611.02045), on one GB300 GPU.
 *
 * Problem (paper Section 2): minimise, over ||phi|| = 1,
 *   E(phi) = int 1/2|grad phi|^2 + V|phi|^2 + eta/2 |phi|^4 - omega conj(phi) L_z phi,
 *   L_z = -i (x d_y - y d_x),
 * discretised on the periodic grid of Section 3: x_k = -L + k h, h = 2L/M,
 * Fourier frequencies xi_p = p pi / L for p = -M/2 .. M/2-1, derivatives by
 * per-axis DFTs (eq. FFTdiscret).
 *
 * Conventions shared by every entry point
 *  - Fields are complex arrays stored [z][y][x], x fastest, interleaved
 *    (re, im).  Their element type is the context's working precision:
 *    complex128 for GPE_FP64, complex64 for GPE_MIXED (the exception is
 *    gpe_pcg_solve, whose phi is always complex128).
 *  - Inner products carry the quadrature weight h^d:
 *    <f, g> = h_x h_y [h_z] sum conj(f_k) g_k, so ||phi||^2 = h^d sum |phi_k|^2.
 *  - Pointers named *_dev must be device memory of the current device;
 *    pointers documented "host or device" are classified with
 *    cudaPointerGetAttributes and copied as needed.
 *  - All work is ordered on the stream given to gpe_create.  Calls that
 *    return host scalars (gpe_energy, gpe_pcg_solve) synchronise it.
 *  - No exception crosses the ABI: every call returns a gpe_status and, on
 *    failure, gpe_last_error() describes the cause.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef GPE_H
#define GPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPE_OK = 0,
  GPE_ERR_ARG = 1,           /* invalid argument (sizes, null pointers, L <= 0, ...) */
  GPE_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  GPE_ERR_NOT_CONVERGED = 3, /* max_iter reached before the stopping rule held */
  GPE_ERR_NONFINITE = 4,     /* NaN/Inf met in a reduction */
  GPE_ERR_PRECOND = 5,       /* alpha + V + eta|phi|^2 <= 0 somewhere (P_V undefined) */
  GPE_ERR_TIMEOUT = 6,       /* reserved: a bounded device wait gave up */
  GPE_ERR_UNSUPPORTED = 7    /* configuration not supported by this build */
} gpe_status;

typedef enum {
  GPE_FP64 = 0,  /* complex128 fields, FP64 everywhere */
  GPE_MIXED = 1  /* complex64 transforms and pointwise work, FP64 reductions,
                    then a complex128 refinement phase */
} gpe_precision;

/* Discrete problem (Sections 2-3).  n[i]: points on axis i (x, y, z), each a
 * power of two in [8, 512]; L[i] > 0: the domain is [-L_i, L_i).  dim = 2
 * ignores n[2], L[2].  Rotation is about the z axis. */
typedef struct {
  int dim;
  int n[3];
  double L[3];
  double eta;    /* nonlinearity (the paper's eta) */
  double omega;  /* rotation speed (the paper's omega) */
  gpe_precision prec;
} gpe_problem;

/* Solver options.  gpe_solve_opts_default fills the values in brackets. */
typedef struct {
  double tol_res_inf;   /* stop when ||H phi_n - lambda_n phi_n||_inf < tol (eq. Stop_Residual) [1e-8] */
  double tol_dE;        /* > 0: also stop when |E_{n+1} - E_n| <= tol_dE (eq. Stop_Energy) [0] */
  int max_iter;         /* total iteration cap over both phases [20000] */
  double theta_default; /* trial step when the model curvature is <= 0 (Section 5.1) [0.1] */
  int max_backtracks;   /* trial step halvings before a step is taken anyway [30] */
  int cg;               /* 1: Algorithm 2 (PCG), 0: Algorithm 1 (PG) [1] */
  /* GPE_MIXED only: the complex64 phase ends, and the complex128 phase
   * starts (see refine_restart), when ||r||_inf falls below
   * switch_res, or -- switch_res <= 0 -- below 4x an estimate of the
   * single-precision floor, eps32 (max_k |k|^2/2 + max V + |lambda|) max|phi|;
   * or when ||r||_inf has not halved within stall_window iterations while
   * within 3x of that threshold. */
  int stall_window;     /* [500] */
  double switch_res;    /* [0: automatic] */
  int max_iter_lo;      /* cap on complex64-phase iterations [max_iter] */
  int use_graph;        /* how the iteration loop runs [3]:
                         * 3: GPE_MIXED 2D grids with nx == ny in [32, 256]: the complex64 phase runs in one
                         *    thread-block cluster with every field in distributed shared memory; other
                         *    phases and grids use 1;
                         * 1: one CUDA graph launch whose WHILE node repeats the per-pass kernels;
                         * 2: one persistent cooperative kernel for the whole loop, its passes separated
                         *    by grid barriers (square 2D grids with n in [64,512], cubic 3D grids with
                         *    n in [64,256]; others fall back to 1);
                         * 0: the per-pass kernels launched from a host loop. */
  int refine_restart;   /* GPE_MIXED: 1 restarts the conjugate directions (beta = 0, p = 0) when the
                         * complex128 phase starts; 0 carries the last complex64 direction p_{n-1},
                         * r_{n-1} and <r_{n-1}, P r_{n-1}> over [1] */
  int precond;          /* [GPE_PRECOND_C] preconditioner of Section 5.4 (below) */
  int beta_rule;        /* [GPE_BETA_PR] conjugation coefficient (below) */
  int line_search;      /* [GPE_LINE_MODEL] step size (below) */
  int wait_polls;       /* use_graph = 2: polls (>= 32 ns apart) of each grid-barrier wait before the
                         * persistent kernel gives up, leaves its loop and the solve returns
                         * GPE_ERR_TIMEOUT with the context still usable; 0 = 2^26 (seconds) [0] */
} gpe_solve_opts;

/* gpe_solve_opts.precond, with alpha = lambda~_n (eq. Opt_Alpha) in every case:
 *  GPE_PRECOND_C     P_V^{1/2} P_Delta P_V^{1/2}            (eq. combinedP_12)
 *  GPE_PRECOND_DELTA P_Delta = (alpha - Delta/2)^{-1}          (eq. PDelta)
 *  GPE_PRECOND_V     P_V = (alpha + V + eta|phi_n|^2)^{-1}     (eq. PV)
 *  GPE_PRECOND_C1    P_V P_Delta                              (eq. combinedP)
 *  GPE_PRECOND_C2    P_Delta P_V                              (eq. combinedP)
 *  GPE_PRECOND_NONE  identity
 * gpe_solve_opts.beta_rule:
 *  GPE_BETA_PR  max(beta_PR, 0) with beta_PR = Re<r_n - r_{n-1}, P r_n> / <r_{n-1}, P r_{n-1}> (eq. CG:PR)
 *  GPE_BETA_FR  <r_n, P r_n> / <r_{n-1}, P r_{n-1}> (eq. CG:FR) */
enum { GPE_PRECOND_C = 0, GPE_PRECOND_DELTA = 1, GPE_PRECOND_V = 2, GPE_PRECOND_C1 = 3, GPE_PRECOND_C2 = 4,
       GPE_PRECOND_NONE = 5 };
enum { GPE_BETA_PR = 0, GPE_BETA_FR = 1 };
/* gpe_solve_opts.line_search (Section 5.1; the energy-decrease backtracking
 * applies after either):
 *  GPE_LINE_MODEL  theta_0 = -Re<H phi, q> / (T2(q) - lambda), the minimiser of
 *                  the second-order model (theta_default when the curvature is <= 0)
 *  GPE_LINE_EXACT  Newton's method from theta_0 on d/dtheta of the exact energy
 *                  change E(cos t phi + sin t q) - E(phi), a trigonometric
 *                  polynomial in t fixed by the step moments (full line search) */
enum { GPE_LINE_MODEL = 0, GPE_LINE_EXACT = 1 };

/* Per-iteration log row, doubles: */
#define GPE_LOG_FIELDS 12
/* n, phase (0 = complex64, 1 = refinement or the FP64 solve, 2 = FP64 completion of a
 * stalled refinement), E_n, lambda_n, ||r_n||_inf,
 * ||r_n||_2, alpha_n (shift of P_C), beta_n (after max(.,0) and the
 * descent check), theta_n, Delta E_n (accepted step), fallback (1 = gradient
 * step taken), backtracks */

typedef struct {
  int status;        /* gpe_status of the solve */
  int iters;         /* iterations n performed (phi returned is phi_n) */
  int iters_lo;      /* of which in the complex64 phase */
  int fallbacks;     /* gradient-step fallbacks (Section 5.2) */
  int backtracks;    /* total step halvings */
  double E;          /* E(phi_n) */
  double lambda;     /* lambda_n = <phi_n, H phi_n> */
  double res_inf;    /* ||r_n||_inf */
  double res_l2;     /* ||r_n||_2 (weighted) */
  int log_cap;       /* in: rows available in log (0: no log) */
  int log_len;       /* out: rows written (min(iters + 1, log_cap)) */
  double* log;       /* in: host array [log_cap][GPE_LOG_FIELDS] or NULL */
  int loop_kind;     /* out: loop style that ran (for GPE_MIXED: of the complex64 phase):
                      * 3 cluster, 2 persistent, 1 graph, 0 host loop */
  int iters_fp64;    /* GPE_MIXED: iterations of the FP64 completion phase (0 unless the
                      * refinement stalled, see gpe_pcg_solve) */
} gpe_report;

typedef struct gpe_ctx gpe_ctx;

/* Fill *opts with the defaults above.  Returns GPE_ERR_ARG if opts is NULL. */
gpe_status gpe_solve_opts_default(gpe_solve_opts* opts);

/* Create a context for problem *prob.
 *  V      : real potential on the grid, float64, [z][y][x]; host or device;
 *           copied (the caller keeps ownership); must be finite.
 *  stream : cudaStream_t (NULL = legacy default stream) that orders all work.
 * Allocates all device workspace (fields, tables, reduction buffers) once.
 * Errors: GPE_ERR_ARG (null pointers, dim not 2/3, n not a power of two in
 * [8,512], L <= 0, non-finite eta/omega), GPE_ERR_CUDA. */
gpe_status gpe_create(const gpe_problem* prob, const double* V, void* stream, gpe_ctx** out);

/* Synchronise the context's stream, then release everything the context owns
 * (device workspace, tables, graphs).  Caller-owned fields are untouched.
 * NULL is accepted.  Always returns GPE_OK. */
gpe_status gpe_destroy(gpe_ctx* ctx);

/* out = H_phi f = -1/2 Delta f + V f + eta |phi|^2 f - omega L_z f
 * (Section 2; discrete operators of eq. FFTdiscret).  phi_dev, f_dev,
 * out_dev: device fields in working precision; out may alias f but not phi.
 * Asynchronous.  Errors: GPE_ERR_ARG, GPE_ERR_CUDA. */
gpe_status gpe_apply_H(gpe_ctx* ctx, const void* phi_dev, const void* f_dev, void* out_dev);

/* out_b = H_{phi_b} f_b for b = 0 .. nbatch-1 (the operator of gpe_apply_H,
 * Section 2 / eq. FFTdiscret), on nbatch fields stored one after another
 * (stride nx*ny elements), all with the context's V, eta and omega.  2D
 * contexts with nx == ny in [32, 256] only.  Global memory is read and written
 * once per point (the output is written by the row part and completed by the
 * column part while still in L2).  Forms, by plan mode 3 of gpe_set_plan:
 *  - single precision, 256 x 256, f == phi, 16-byte aligned fields and V,
 *    E = 16 with width 16 (the default): a dataflow of row units and column
 *    units (16 lines each) taken by persistent blocks on every SM from one
 *    ticket queue, inputs copied by the TMA; a field's column units add their
 *    part after its row units have stored theirs.  Uses a counter array of the
 *    context (nbatch + 2 ints, allocated on first use and when the batch
 *    grows; zero between calls), so one such call runs at a time per context;
 *  - otherwise one thread-block cluster per field (16 rows per CTA) in
 *    distributed shared memory; in single precision with n >= 64 and 16-byte
 *    aligned phi and f the resident clusters loop over the fields and copy the
 *    next field's rows while transforming the current one (E = 16, 16 or 32
 *    rows per CTA; E = 8 selects one field per cluster).
 * phi_dev, f_dev, out_dev: device arrays in working precision; f may equal
 * phi; out must not overlap phi or f.  Asynchronous.  A bounded wait of the
 * dataflow form that gives up (never expected) marks the context's API status
 * GPE_ERR_TIMEOUT.  Errors: GPE_ERR_ARG, GPE_ERR_UNSUPPORTED (other grids),
 * GPE_ERR_CUDA. */
gpe_status gpe_apply_H_batch(gpe_ctx* ctx, int nbatch, const void* phi_dev, const void* f_dev, void* out_dev);

/* out = P_C r = P_V^{1/2} P_Delta P_V^{1/2} r (eq. combinedP_12) with
 * P_Delta = (alpha - Delta/2)^{-1} (eq. PDelta) and
 * P_V = (alpha + V + eta |phi|^2)^{-1} (eq. PV).  alpha <= 0 selects the
 * paper's adaptive shift lambda~(phi) = int 1/2|grad phi|^2 + V|phi|^2 +
 * eta|phi|^4 (eq. Opt_Alpha), computed on the device.  Fields as for
 * gpe_apply_H; out may alias r.  Asynchronous.  Errors: GPE_ERR_ARG,
 * GPE_ERR_CUDA. */
gpe_status gpe_precond(gpe_ctx* ctx, const void* phi_dev, const void* r_dev, double alpha, void* out_dev);

/* Energy terms of phi (Section 2), host doubles:
 * out[0] kinetic int 1/2|grad phi|^2, out[1] potential int V|phi|^2,
 * out[2] interaction eta/2 int |phi|^4, out[3] rotation -omega <phi, L_z phi>,
 * out[4] total E, out[5] lambda = <phi, H_phi phi>, out[6] lambda~ (eq. Opt_Alpha),
 * out[7] ||phi||^2.  phi is not normalised first.  Synchronises the stream.
 * Errors: GPE_ERR_ARG, GPE_ERR_CUDA. */
gpe_status gpe_energy(gpe_ctx* ctx, const void* phi_dev, double out[8]);

/* Replace the context's potential and coupling constants without
 * re-creating it (parameter sweeps, finite differences, fitting V).
 *  V     : new real potential, float64 [z][y][x], host or device; NULL keeps
 *          the current one.  Must be finite.
 *  eta, omega : new nonlinearity and rotation speed (Section 2), finite.
 * Every later call uses the new problem; CUDA graphs captured for the old one
 * are discarded.  Synchronises the stream.  Errors: GPE_ERR_ARG,
 * GPE_ERR_CUDA. */
gpe_status gpe_set_problem(gpe_ctx* ctx, const double* V, double eta, double omega);

/* Derivatives of the discrete energy (Section 2, with the discretisation of
 * Section 3) at phi, for phi held fixed:
 *  grad_phi_dev : if not NULL, receives nabla E(phi) = 2 h^d H_phi phi, the
 *                 gradient of E with respect to the real and imaginary parts
 *                 of the grid values (d E / d Re phi_k + i d E / d Im phi_k);
 *                 Section 2 gives nabla E = 2 H_phi phi for the weighted inner
 *                 product, h^d converts it to the coefficient vector.  Field
 *                 in working precision; must not overlap phi.
 *  grad_V_dev   : if not NULL, float64 [z][y][x]: d E / d V_k = h^d |phi_k|^2.
 *  out          : out[0] E, out[1] d E / d eta = 1/2 int |phi|^4,
 *                 out[2] d E / d omega = -<phi, L_z phi>, out[3] lambda =
 *                 <phi, H_phi phi>, out[4] ||phi||^2.
 * At a normalised critical point phi* (a ground state from gpe_pcg_solve) the
 * constraint terms vanish, so out[1], out[2] and grad_V are the derivatives
 * of the ground-state energy E*(V, eta, omega) itself (Hellmann-Feynman).
 * Synchronises the stream.  Errors: GPE_ERR_ARG, GPE_ERR_CUDA. */
gpe_status gpe_energy_grad(gpe_ctx* ctx, const void* phi_dev, void* grad_phi_dev, double* grad_V_dev, double out[5]);

/* Tangent-space adjoint solve at a ground state: find z with <phi, z> = 0 and
 *   P K z = P rhs,   K f = H_phi f + eta |phi|^2 f + eta phi^2 conj(f) - lambda f,
 * P h = h - <phi, h> phi.  K is the operator of the second-order form
 * 1/2 grad^2 E(phi)[f, f] - lambda ||f||^2 of Section 2 (with the term
 * eta int |phi|^2 |f|^2 the printed formula omits), lambda = <phi, H_phi phi>;
 * P is the tangent projector M_phi of Section 2 with the phase direction
 * i phi also removed (K (i phi) = 0 at a critical point).  Section 2's
 * second-order condition makes K positive on that space at a local minimum.
 * Differentiating H_phi phi = lambda phi, ||phi|| = 1 gives K dphi = -P(dV phi),
 * so with rhs = the weighted gradient of a loss L(phi) (dL = Re<rhs, dphi>),
 * dL/dV_k = -h^d Re(conj(z_k) phi_k).
 * Method: conjugate gradients in the real inner product Re<.,.>, the
 * preconditioner P P_C P (eq. combinedP_12 with the shift lambda~ of eq.
 * Opt_Alpha at phi), stopped when ||r|| <= tol ||P rhs||.
 *  phi_dev : normalised ground state (working precision);
 *  rhs_dev : right-hand side (working precision);
 *  z_dev   : solution (working precision), must not overlap phi or rhs;
 *  iters, rel_res : may be NULL; iterations and ||r|| / ||P rhs||.
 * Synchronises the stream.  Errors: GPE_ERR_ARG, GPE_ERR_CUDA,
 * GPE_ERR_NOT_CONVERGED (max_iter reached; z holds the last iterate),
 * GPE_ERR_NONFINITE (K or P_C not positive -- phi is not a local minimum --
 * or a non-finite residual). */
gpe_status gpe_tangent_solve(gpe_ctx* ctx, const void* phi_dev, const void* rhs_dev, void* z_dev, double tol,
                             int max_iter, int* iters, double* rel_res);

/* Gradient with respect to V of a loss L(rho) of the ground-state density
 * rho = |phi*|^2, through the tangent-space adjoint solve above:
 *   rhs = (2 / h^d) g_rho phi  (so that dL = Re<rhs, dphi>),
 *   z   = gpe_tangent_solve(phi, rhs),
 *   grad_V[k] = dL/dV_k = -h^d Re(conj(z_k) phi_k).
 *  phi_dev    : normalised ground state for the context's V, eta, omega
 *               (working precision);
 *  g_rho_dev  : float64 dL/drho_k per grid point (device);
 *  grad_V_dev : float64 output (device).
 * tol, max_iter, iters, rel_res as for gpe_tangent_solve.  Synchronises the
 * stream.  Errors as gpe_tangent_solve; on GPE_ERR_NOT_CONVERGED grad_V is
 * computed from the last iterate. */
gpe_status gpe_density_adjoint(gpe_ctx* ctx, const void* phi_dev, const double* g_rho_dev, double* grad_V_dev,
                               double tol, int max_iter, int* iters, double* rel_res);

/* Thomas-Fermi initial data (Section 6, eq. TF_App): phi_0 = sqrt(max(mu - V, 0) / eta),
 * with mu fixed by the normalisation h^d sum max(mu - V, 0) / eta = 1 (so that
 * ||phi_0|| = 1), found by bisection on the device (120 halvings of the bracket
 * [min V, max V + eta / (h^d N)]).  The closed forms of eq. TF_Rdius hold for
 * the paper's harmonic traps only; the normalisation holds for any V.
 *  phi_out : complex128 [z][y][x], host or device.
 *  mu_out  : may be NULL; receives mu.
 * Synchronises the stream.  Errors: GPE_ERR_ARG (eta <= 0), GPE_ERR_CUDA. */
gpe_status gpe_thomas_fermi(gpe_ctx* ctx, void* phi_out, double* mu_out);

/* Spectral interpolation for multigrid continuation (Section 6: the ground
 * state on M_p points per axis is interpolated onto M_{p+1} = 2 M_p points and
 * used as the initial data there).  Along every axis where fine->n = 2 coarse->n,
 * each line is replaced by the samples at the fine points of its
 * trigonometric interpolant (1/Mc) sum_p F_p e^{i xi_p (x + L)}, F = DFT(line),
 * with the Nyquist coefficient shared equally by the modes -Mc/2 and +Mc/2;
 * axes with equal sizes are copied.  Complex128 throughout.
 *  coarse, fine : contexts on the same domain (equal L), same dimension, each
 *                 fine axis equal to or twice the coarse one (coarse axes
 *                 refined: at most 256 points).
 *  phi_c  : complex128 coarse field, host or device.
 *  phi_f  : complex128 fine field, host or device, not overlapping phi_c.
 * Uses the fine context's stream and work buffers; synchronises.  Errors:
 * GPE_ERR_ARG, GPE_ERR_UNSUPPORTED, GPE_ERR_CUDA (messages on fine). */
gpe_status gpe_interpolate(gpe_ctx* coarse, const void* phi_c, gpe_ctx* fine, void* phi_f);

/* Ground state by Algorithm 2 (PCG) with the symmetric combined
 * preconditioner P_C, the Polak-Ribiere coefficient beta = max(beta_PR, 0)
 * (eq. CG:PR), the descent check of Section 5.2, the step-size heuristic and
 * energy-decrease backtracking of Section 5.1, and renormalisation after
 * every step.
 *  phi_inout : complex128 [z][y][x], host or device.  In: initial guess (need
 *              not be normalised).  Out: the last iterate phi_n.
 *  opts      : NULL = defaults.
 *  report    : may be NULL.
 * GPE_MIXED runs a complex64 phase, then a refinement phase from its result
 * (double-single state and H phi, single-precision direction); if the
 * refinement's ||r||_inf fails to halve within 4 opts->stall_window iterations
 * (a near-flat energy direction whose curvature single-precision step
 * moments cannot resolve), the solve is completed in FP64 from there.
 * Synchronises the stream.  Returns GPE_OK when the stopping rule held, else
 * GPE_ERR_NOT_CONVERGED / GPE_ERR_NONFINITE / GPE_ERR_PRECOND / GPE_ERR_ARG /
 * GPE_ERR_CUDA (report->status carries the same code). */
gpe_status gpe_pcg_solve(gpe_ctx* ctx, void* phi_inout, const gpe_solve_opts* opts, gpe_report* report);

/* Allocation-free H_phi f.  The paper has no counterpart: this is an
 * interface addition for callers that cannot allocate device memory --
 * code running under a memory manager that owns the whole device, inside a
 * library that promised never to call the allocator, or with the device
 * memory already exhausted -- and so cannot create a context.
 *
 * Computes the same out = H_phi f as gpe_apply_H with the same pass kernels,
 * under default plans (a context's tuned plans may sum in another order, so
 * results agree to rounding), but takes the problem directly and keeps its
 * intermediate field, grid tables, reduction partials and control block in
 * one fixed static device array of libgpe (about 17 MiB, held by every GPU
 * that loads the library until the process exits).  It calls no
 * cudaMalloc/cudaFree and no allocating library.
 *  prob    : as for gpe_create; prob->prec selects the element types.
 *  V_dev   : real potential on the device, float64 for GPE_FP64, float32 for
 *            GPE_MIXED, [z][y][x].
 *  phi_dev, f_dev, out_dev : device fields, complex128 (GPE_FP64) or
 *            complex64 (GPE_MIXED); out may alias f.
 *  stream  : cudaStream_t ordering the work (NULL = legacy default stream).
 *  err, err_len : optional buffer for a message (NUL-terminated), may be NULL.
 * Limits: N * sizeof(element) <= 16 MiB, i.e. at most 2^20 complex128 or 2^21
 * complex64 points; and at most 8192 thread blocks in any axis's pass (the
 * partials the array holds), which excludes some flat 3D grids such as
 * 512 x 8 x 512.  Both are checked before any work is queued: such calls
 * return GPE_ERR_UNSUPPORTED with the sizes in err and leave out untouched.
 * Each call outside a stream capture looks up the array's device address on
 * the current device (cudaGetSymbolAddress); a call inside a capture uses the
 * address of the last uncaptured call on that device, so make one call on
 * each device before capturing.  Every call reuses the same array and leaves
 * its last contents there, so calls whose GPU work can overlap (other
 * streams, other host threads) race: serialise them.  Asynchronous.  Errors:
 * GPE_ERR_ARG, GPE_ERR_UNSUPPORTED, GPE_ERR_CUDA. */
gpe_status gpe_apply_H_noalloc(const gpe_problem* prob, const void* V_dev, const void* phi_dev, const void* f_dev,
                               void* out_dev, void* stream, char* err, size_t err_len);

/* ---- Plans of the pass kernels and the tuner ------------------------------
 * Every grid pass transforms lines of M points held by M/E threads with E
 * values each (E = 8 or 4: the radix structure of the Stockham line transform,
 * radix 8 then 8/4/2 stages for E = 8, radix-4 stages for E = 4), blocks of
 * `width` lines (x passes) or tiles of `width` adjacent x-columns (y, z
 * passes).  A plan (E, width) is kept per launch mode (0: complex64 passes,
 * 1: FP64 passes, 2: refinement passes) and axis; the defaults are E = 8 and
 * widths from a block-count heuristic.  Plans change the order of floating-
 * point sums, not the method.  The paper has no counterpart (it runs serial
 * full-grid FFTs). */
typedef struct {
  int cached;           /* 1: every plan came from an earlier tuning of the same grid in this process */
  int candidates;       /* plans timed */
  double us_before[3];  /* per mode: microseconds per iteration with the plans in use before the call
                         * (0: mode not used by the context, or cached) */
  double us_after[3];   /* with the chosen plans */
  int E[3][3];          /* chosen [mode][axis] */
  int width[3][3];
} gpe_tune_report;

/* Time candidate plans on this context's grid and keep the fastest per mode
 * and axis: `iters` solver iterations (host-launched passes, from a
 * normalised Gaussian) per candidate, coordinate descent over the axes, a new
 * choice must be 2% faster.  use_cache != 0 reuses the plans tuned earlier in
 * this process for the same grid and mode.  Overwrites the context's solver
 * work buffers; discards its captured graphs.  Synchronises the stream.
 * report may be NULL.  Errors: GPE_ERR_ARG, GPE_ERR_CUDA. */
gpe_status gpe_autotune(gpe_ctx* ctx, int iters, int use_cache, gpe_tune_report* report);

/* Set / read the plan of (mode, axis).  gpe_set_plan rejects plans the kernels
 * cannot run (E not 4 or 8, E = 4 below M = 32, width not a power of two, more
 * threads than the mode's kernels allow, too much shared memory, more blocks
 * than the context's reduction buffers) with GPE_ERR_ARG.  Mode 3, axis 0 is
 * the kernel of gpe_apply_H_batch: E = 8 (one field per cluster, 16 rows per
 * CTA) or E = 16 (single precision, n >= 64) with width 16 (the dataflow form
 * where it applies, else the streaming form with a cluster of n/16 CTAs) or
 * 32 (the streaming form with n/32 CTAs, so an 8-CTA cluster at n = 256). */
gpe_status gpe_set_plan(gpe_ctx* ctx, int mode, int axis, int E, int width);
/* The plan in use for (mode, axis): *E values per thread and *width (lines per
 * block on axis 0, tile columns on the others; rows per CTA for mode 3), host
 * ints written by the call.  Errors: GPE_ERR_ARG (null pointers, mode outside
 * 0..2, axis outside the grid, mode 3 on a context the batched H kernel does
 * not take). */
gpe_status gpe_get_plan(const gpe_ctx* ctx, int mode, int axis, int* E, int* width);

/* ---- Batched solves ------------------------------------------------------
 * Many independent ground states (different grids, eta, omega, V; Section 2
 * problems, each solved by the gpe_pcg_solve algorithm) in ONE graph launch.
 * The batch holds one context per instance and one CUDA graph with one
 * branch per instance; the branches run concurrently on the GPU.  A mixed
 * instance's branch is: the complex64 phase (one thread-block-cluster kernel
 * for 2D square grids of 32..256 points, else a device-side loop of the pass
 * kernels), a device-side decision whether to refine, and the refinement
 * loop; nothing returns to the host until the whole batch is done.  The
 * paper solves one problem at a time: batching is an interface addition. */
typedef struct gpe_batch gpe_batch;

/* count instances; probs[i] and V[i] as for gpe_create (V[i] host or device
 * float64).  stream orders all work.  Errors: GPE_ERR_ARG, GPE_ERR_CUDA (the
 * message names the instance; read it with gpe_batch_last_error(NULL)). */
gpe_status gpe_batch_create(int count, const gpe_problem* probs, const double* const* V, void* stream,
                            gpe_batch** out);

/* Solve every instance from phi_inout[i] (complex128, host or device; in:
 * initial guess, out: last iterate), with the same options for all (NULL =
 * defaults; refine_restart, use_graph and the log are ignored: the batch always
 * restarts beta at the refinement and keeps no log).  reports: NULL or an
 * array of count reports.  The graph is built by the first call.  Synchronises
 * the stream.  Returns GPE_OK when every instance met the stopping rule, else
 * the first failing instance's status (each report carries its own).  Errors:
 * GPE_ERR_ARG (NULL batch or phi array or entry, invalid options),
 * GPE_ERR_CUDA; the per-instance statuses are those of gpe_pcg_solve. */
gpe_status gpe_batch_solve(gpe_batch* batch, void* const* phi_inout, const gpe_solve_opts* opts, gpe_report* reports);

/* Synchronise the batch's stream and release the batch, its graph and every
 * instance's context.  NULL is accepted.  Always returns GPE_OK. */
gpe_status gpe_batch_destroy(gpe_batch* batch);

/* gpe_autotune (with the process cache) on every instance's context; the
 * batch graph is rebuilt with the chosen plans by the next gpe_batch_solve.
 * Overwrites the instances' solver work buffers; synchronises the stream.
 * Errors: GPE_ERR_ARG (NULL batch, iters < 1), GPE_ERR_CUDA (the message, read
 * with gpe_batch_last_error, is that of the failing instance). */
gpe_status gpe_batch_autotune(gpe_batch* batch, int iters);

/* Last failure on batch ("" if none); NULL: the last failed gpe_batch_create.
 * The string is owned by the batch (or the library) and valid until the next
 * call on it. */
const char* gpe_batch_last_error(const gpe_batch* batch);

/* ---- Measurement ---------------------------------------------------------
 * Arithmetic-pipe rate of the current device, the roof of the kernels that
 * memory does not bound (FP64 passes: FP64 pipe; double-single and
 * single-precision transforms: FP32 pipe).  Not part of the method (the paper
 * has no counterpart): independent fused multiply-add chains in registers,
 * 8 blocks of 256 threads per SM, best of 3 CUDA-event-timed launches after a
 * warm-up, at the clocks of the moment.
 *  kind   : 0 FP64 fma, 1 FP32 fma, 2 packed two-wide FP32 fma (fma.rn.f32x2).
 *  stream : cudaStream_t (NULL = legacy default stream); synchronised.
 *  gflops : out, 10^9 floating-point operations per second (an FMA is 2).
 * Allocates and frees a small result buffer.  Errors: GPE_ERR_ARG (kind
 * outside 0..2, NULL gflops), GPE_ERR_CUDA. */
gpe_status gpe_alu_peak(int kind, void* stream, double* gflops);

/* Human-readable description of the last failure on ctx ("" if none).
 * The string is owned by ctx and valid until its next call. ctx NULL gives
 * the message of the last failed gpe_create. */
const char* gpe_last_error(const gpe_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GPE_H */
