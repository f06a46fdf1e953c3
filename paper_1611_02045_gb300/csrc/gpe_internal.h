// gpe_internal.h -- device control block and pass-launch interface shared by
// the kernel translation units and the C ABI (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace gpe {

// Per-device "done once" flag for kernel attribute set-up
// (cudaFuncSetAttribute applies to the current device's context only).
// Thread-safe; devices 0..63 (others redo the set-up on every launch, which is
// correct, only slower).  Setting an attribute twice is harmless.
struct DeviceOnce {
  std::atomic<unsigned long long> bits{0};
  static int device() {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess ? d : -1;
  }
  bool done(int dev) const { return dev >= 0 && dev < 64 && ((bits.load(std::memory_order_acquire) >> dev) & 1ull); }
  void set(int dev) {
    if (dev >= 0 && dev < 64) bits.fetch_or(1ull << dev, std::memory_order_release);
  }
};

// Number of doubles in one per-iteration log row (matches GPE_LOG_FIELDS).
constexpr int kLogFields = 12;
// Max reduction slots per pass.
constexpr int kMaxMoments = 12;

// Device-resident scalar state of one solve (or of one API call).  Kernels
// read the scalars they need at entry; the last thread block of each
// reducing pass writes the reduced moments and runs the scalar logic.
struct Ctl {
  // ---- options (set by the host before a solve) ----
  double tol_res_inf, tol_dE, theta_default, switch_res;
  int max_iter, max_backtracks, cg, stall_window, max_iter_phase, phase;
  int lo_phase;  // 1 while running the complex64 phase of a mixed solve
  int pc_kind;   // preconditioner: 0 P_C (symmetric combined), 1 P_Delta, 2 P_V, 3 P_C1 = P_V P_Delta,
                 // 4 P_C2 = P_Delta P_V, 5 none
  int beta_rule; // 0 Polak-Ribiere beta+ (eq. CG:PR), 1 Fletcher-Reeves (eq. CG:FR)
  int line_search;  // 0 model step theta_0 + backtracking; 1 Newton on the exact step polynomial from theta_0
  // ---- loop state ----
  int iter;        // n (global over both phases)
  int iter_phase0; // value of iter when this phase started
  int iters_lo;    // batched mixed solve: iterations of the complex64 phase
  int iters_hi;    // batched mixed solve: iteration count when the FP64 completion phase started (0: none)
  int stall_switch;  // 1 in the refinement phase: a stall (no halving of ||r||_inf in stall_window
                     // iterations) ends it with switch_req, and the solve is completed in FP64
  int done;        // 1 once the loop must stop
  int status;      // gpe_status of the solve
  int restart;     // 1: next direction uses beta = 0 (first iteration of a phase)
  int retract;     // 1: the next H pass first forms phi_{n+1} from (phi_n, p_n)
  int fallback;    // gradient step taken this iteration
  int fallbacks, backtracks_total, backtracks;
  int switch_req;  // complex64 phase asked for the complex128 phase
  int stop_dE;     // energy criterion met at the last step
  // ---- per-iterate scalars ----
  double kin, rot, pot, U0, norm2;      // <phi,-Lap/2 phi>, <phi,-omega Lz phi>, <phi,V phi>, int|phi|^4, ||phi||^2
  double Lz;                            // <phi, L_z phi> (real: L_z is Hermitian)
  double lam, alpha, E;                 // lambda_n, lambda~_n, E_n
  double res_inf, res_l2;
  double rPr, rPr_prev;                 // <r_n, P r_n>, previous
  double beta, gamma;                   // beta_n, Re<d_n, phi_n>
  double theta, c, s, inv_np, inv_nrm;  // retraction scalars for the next H pass
  double dE;
  double anchor_res; int anchor_iter;   // stall detection (mixed phase)
  int pad0;
  double phimax;      // max |phi_n| (H x pass)
  double floor_coef;  // eps32 (max 1/2|k|^2 + max V): complex64 residual floor per unit |phi|
  double switch_fac;  // complex64 phase ends when ||r||_inf < switch_fac * floor estimate
  // ---- raw sums written by pass finalisers ----
  double hsum[3][kMaxMoments];  // H passes, per axis
  double psum[kMaxMoments];     // P_C passes
  double asum[3][kMaxMoments];  // A p passes, per axis
  // ---- log ----
  double* log;
  int log_cap;
  int log_len;
};

enum Pass : int {
  P_HX = 0,     // x: [retraction] t = A_x f + (V + eta|phi|^2) f
  P_HMID = 1,   // y/z: t += A_axis f
  P_C1 = 2,     // x: s = FFT_x(P_V^{1/2} r)
  P_CFWD = 3,   // y (3D): s = FFT_y s
  P_CCORE = 4,  // last axis: s = IFFT(FFT(s) / (alpha + |k|^2/2)) / N
  P_CINV = 5,   // y (3D): s = IFFT_y s
  P_C3 = 6,     // x: Pr = P_V^{1/2} IFFT_x s (+ solver reductions)
  P_AX = 7,     // x: p = -Pr + beta p_prev - gamma phi; Parseval moments
  P_AMID = 8,   // y/z: Parseval moments of A_axis p
  P_NUM = 9
};

// Everything a pass kernel needs, passed by value.
struct PassArgs {
  int dim, nx, ny, nz;
  int axis;        // physical axis transformed by this pass
  int M;           // length along that axis
  int E;           // values per thread of the line transforms: 4, or 8 (also when 0)
  int lpb;         // contiguous passes: lines per block
  int row0;        // contiguous passes: global row of line 0 (field slices held by one CTA)
  int tx;          // strided passes: tile width in x
  long long stride;        // strided: element stride along the axis
  long long outer_stride;  // strided: element stride of the outer index
  int ntx;         // strided: nx / tx
  int nblocks;     // grid size
  int pf;          // contiguous H pass outside a solve: L2 prefetch of the rows of unit + pf (0: none)
  int solver;      // 1: inside a solve (uses ctl scalars, solver reductions)
  int nomoments;   // 1: the caller needs no reductions (H phi as a plain operator): passes skip them
  int last_axis;   // 1: this pass is the final one of its operator (runs the finaliser)
  double weight;   // h^d
  double eta, omega;
  // device tables, in the kernel's precision (T*), stored as void*
  const void* xi[3];   // frequencies per axis, DFT order
  const void* xc[3];   // coordinates per axis
  const void* tw;      // twiddles e^{-2 pi i m/M}, m < M, for this axis
  const void* V;       // potential, real
  // fields (complex, kernel precision)
  const void* phi;     // phi_n (or phi_{n} before retraction)
  void* phi_out;       // HX: where phi_{n+1} is written (solver, retract)
  const void* f;       // operand (API apply_H: f; solver: = phi)
  void* p;             // direction p (read in HX for retraction, written in AX)
  void* t;             // H accumulator / H phi
  void* s;             // P_C workspace (s_hat, then P r)
  void* r_prev;        // r_{n-1}, overwritten with r_n by P_C3 (solver)
  const void* r_in;    // API precond input r
  void* out;           // API output
  double api_alpha;    // API precond shift (> 0)
  Ctl* ctl;
  double* partials;    // [nblocks][kMaxMoments]
  unsigned int* ticket;
  unsigned long long cond;  // cudaGraphConditionalHandle (0 = none)
};

// Launch one pass.  mode 0: complex64; 1: complex128; 2: refinement split
// (FP64 phi, H phi, r and V; FP32 P_C workspace and direction p; the x pass
// of H phi reads p in FP32).  Returns cudaSuccess or the launch error.
cudaError_t launch_pass(int mode, Pass pass, const PassArgs& a, cudaStream_t st);

// The y / z passes in complex64 (roles P_HMID, P_CFWD, P_CCORE, P_CINV,
// P_AMID) fed by tensor-map (TMA) tile loads in a persistent, double-buffered
// kernel (gpe_k_tma.cu); *used = false when the plan or the fields do not
// allow it (E = 8, even tile width, 16-byte aligned inputs) or the field is
// too small for every block to get two tiles: the caller then launches the
// standard pass kernel.
cudaError_t launch_strided_tma(Pass pass, const PassArgs& a, cudaStream_t st, bool* used);
// The x pass of H phi in complex64 fed by 1D bulk copies (phi, f or p, V rows)
// in a persistent, double-buffered kernel (gpe_k_tma.cu); *used = false when
// it does not apply (E = 8, M in 64 .. 512, 16-byte aligned fields, at least
// two units per block).
cudaError_t launch_hx_bulk(const PassArgs& a, cudaStream_t st, bool* used);
// C1, C3, AX of a complex64 solve through the bulk-copy pipeline (gpe_k_tma.cu).
cudaError_t launch_xc_bulk(Pass pass, const PassArgs& a, cudaStream_t st, bool* used);

// Per-group launchers (gpe_k_<prec>_<group>.cu).
cudaError_t launch_group_f32_h(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f32_c(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f32_a(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_h(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_c(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_a(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_split(Pass pass, const PassArgs& a, cudaStream_t st);
// The same groups with E = 4 values per thread (PassArgs::E == 4; M >= 32).
cudaError_t launch_group_f32_h_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f32_c_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f32_a_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_h_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_c_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_f64_a_e4(Pass pass, const PassArgs& a, cudaStream_t st);
cudaError_t launch_group_split_e4(Pass pass, const PassArgs& a, cudaStream_t st);

// H phi on a batch of 2D fields, one thread-block cluster per field
// (gpe_cluster.cu); args is a ClusterHArgs (gpe_cluster.cuh).
struct ClusterHArgs;
cudaError_t launch_cluster_apply_H(int is_double, const ClusterHArgs& a, cudaStream_t st);

// The complex64 phase of a 2D solve in one thread-block cluster's shared
// memory (gpe_csolve.cuh; M = nx = ny in [32, 256]).
struct ClusterSolveArgs;
cudaError_t launch_cluster_solve(int M, const ClusterSolveArgs& P, cudaStream_t st);

// Small elementwise/control kernels (gpe_misc.cu).
cudaError_t launch_convert_c128_to_c64(const void* src, void* dst, long long n, cudaStream_t st);
cudaError_t launch_convert_c64_to_c128(const void* src, void* dst, long long n, cudaStream_t st);
cudaError_t launch_d2f(const double* src, float* dst, long long n, cudaStream_t st);
cudaError_t launch_d2ds(const double* src, void* dst, long long n, cudaStream_t st);
cudaError_t launch_convert_c64_to_ds(const void* src, void* dst, long long n, cudaStream_t st);
cudaError_t launch_convert_ds_to_c128(const void* src, void* dst, long long n, cudaStream_t st);
// ctl->c = 1, s = 0, inv_nrm = 1 / ||phi||, retract = 1 (weighted norm), so
// that the next H pass normalises phi in place.
// prec: 0 complex64, 1 complex128, 2 double-single.
// partials: >= 1024 doubles of scratch; ticket: the reduction ticket (0 on entry, 0 on exit).
cudaError_t launch_init_norm(int prec, const void* phi, long long n, double weight, Ctl* ctl, double* partials,
                             unsigned* ticket, cudaStream_t st);
// Tangent-space adjoint solve (gpe_adjoint.cu): device scalars of the
// projected conjugate gradient iteration, and its kernels.  Each reduction
// launcher sums weighted inner products into S and runs the scalar step
// `stage`; update kernels read their coefficients from S and do nothing once
// S->stop is set (converged: ||r||^2 <= tol2 ||r_0||^2, or broken down: bad).
struct AdjScalars {
  double c_re, c_im;  // projection coefficient <phi, h> of the last projected field
  double a, beta;     // step length and conjugation coefficient
  double ry, rr, bb, pq, tol2;
  int bad;    // 1: Re<p, K p> <= 0; 2: Re<r, P_C r> <= 0; 3: non-finite residual
  int stop;
  int iters;
};
enum AdjStage { ADJ_PROJ = 0, ADJ_BB = 1, ADJ_PQ = 2, ADJ_RR = 3, ADJ_RY = 4, ADJ_RY_FIRST = 5 };
cudaError_t adj_dots(int prec, const void* x0, const void* y0, const void* x1, const void* y1, const void* x2,
                     const void* y2, long long n, double weight, int stage, AdjScalars* S, double* partials,
                     int max_blocks, cudaStream_t st);
cudaError_t adj_hess_epi(int prec, const void* phi, const void* p, void* q, long long n, double eta, double lam,
                         double weight, AdjScalars* S, double* partials, int max_blocks, cudaStream_t st);
cudaError_t adj_step(int prec, void* z, void* r, const void* p, const void* q, const void* phi, long long n,
                     double weight, AdjScalars* S, double* partials, int max_blocks, cudaStream_t st);
cudaError_t adj_proj(int prec, const void* h_in, void* h_out, const void* phi, long long n, const AdjScalars* S,
                     cudaStream_t st);
cudaError_t adj_dir(int prec, void* p, const void* y, const void* phi, long long n, const AdjScalars* S,
                    cudaStream_t st);
// rhs = s g_rho phi; grad_V = -weight Re(conj(z) phi)
cudaError_t adj_density_rhs(int prec, const void* phi, const double* g_rho, void* rhs, long long n, double s,
                            cudaStream_t st);
cudaError_t adj_dV_from_z(int prec, const void* phi, const void* z, double* gV, long long n, double weight,
                          cudaStream_t st);

// Between the phases of a batched mixed solve (the host logic of
// gpe_pcg_solve, on the device so that a whole batch is one graph):
//  batch_between: unless the complex64 phase failed (non-finite, P_V
//    undefined), phi128 = phi64 and phids = phi64;
//  batch_gate (one thread): records iters_lo; if the complex64 phase asked for
//    refinement (or "converged" in single precision) and iterations remain,
//    re-arms ctl for the refinement phase (beta restart) and sets the
//    refinement loop's condition to 1, else to 0;
//  batch_final: if the refinement ran and did not fail, phi128 = phids.
cudaError_t launch_batch_between(const void* phi64, void* phi128, void* phids, long long n, const Ctl* ctl,
                                 cudaStream_t st);
cudaError_t launch_batch_gate(Ctl* ctl, unsigned long long cond, cudaStream_t st);
cudaError_t launch_batch_final(const void* phids, void* phi128, long long n, const Ctl* ctl, cudaStream_t st);
//  batch_gate64 (one thread): if the refinement stalled and iterations remain,
//    re-arms ctl for the FP64 completion phase and sets its loop condition.
cudaError_t launch_batch_gate64(Ctl* ctl, unsigned long long cond, cudaStream_t st);
// Set the cluster solve kernel's attributes for grid size M (before capture).
cudaError_t prepare_cluster_solve(int M);

// Thomas-Fermi initial data (eq. TF_App): mu solving h^d sum max(mu - V, 0) / eta = 1
// by bisection (state[0] = lo, state[1] = hi on entry; each launch halves the
// bracket), then phi = sqrt(max(mu - V, 0) / eta) as complex128.
cudaError_t launch_tf_bisect(const double* V, long long n, double weight, double eta, double* state,
                             double* partials, unsigned* ticket, cudaStream_t st);
cudaError_t launch_tf_fill(const double* V, long long n, double eta, const double* state, void* phi128,
                           cudaStream_t st);

// Spectral interpolation onto a grid twice as fine along one axis
// (gpe_interp.cu).  Line l = (outer, inner), inner < inner_count, starts at
// outer * *_outer + inner * *_inner and its points are *_stride apart; Mc
// coarse points in, 2 Mc fine points out, complex128.
struct InterpArgs {
  const double2* in;
  double2* out;
  long long lines, inner_count;
  long long in_outer, out_outer, in_inner, out_inner, in_stride, out_stride;
  const double2* tw_c;  // e^{-2 pi i m / Mc}
  const double2* tw_f;  // e^{-2 pi i m / (2 Mc)}
};
cudaError_t launch_interp(int Mc, const InterpArgs& a, cudaStream_t st);

// grad_phi <- 2 weight grad_phi (in place), grad_V = weight |phi|^2 (float64);
// prec 0 complex64, 1 complex128; null outputs are skipped.
cudaError_t launch_grad_epilogue(int prec, const void* phi, void* gphi, double* gV, long long n, double weight,
                                 cudaStream_t st);

}  // namespace gpe
