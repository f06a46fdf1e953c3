// gpe_passes.cuh -- the per-axis pass kernels of one PCG_C iteration
// (arXiv:1611.02045, Algorithm 2 with the operators of Sections 2, 3, 5.5).
//
// Each pass streams every point of a field once along one axis: it loads a
// line (x) or a tile of TX adjacent lines (y, z) into registers, applies a
// pointwise prologue, a line DFT (gpe_fft.cuh), a Fourier-space multiplier,
// optionally the inverse DFT, and a pointwise epilogue, then writes the
// result.  Reductions are accumulated per thread, combined per block in FP64
// and summed over blocks in a fixed order by the last block to finish, which
// then runs the scalar step that belongs after that pass (chemical potential,
// convergence test, Polak-Ribiere coefficient, step size).
//
// Pass roles (Pass enum in gpe_internal.h), 2D order per iteration:
//   HX   : [phi <- (c phi + s p/|p|)/nrm] ; t = (1/2 xi^2 + omega y xi) f + (V + eta|phi|^2) f
//   HMID : t += (1/2 mu^2 - omega x mu) f   (y)      or  (1/2 zeta^2) f  (z)
//   C1   : s = FFT_x[ P_V^{1/2} (t - lambda phi) ]
//   CCORE: s = IFFT_y[ FFT_y(s) / (alpha + |k|^2/2) ] / N
//   C3   : Pr = P_V^{1/2} IFFT_x[s]; r_prev <- r
//   AX   : p = -Pr + beta p_prev - gamma phi;  moments of p and of FFT_x p
//   AMID : moments of FFT_y p
// (3D inserts HMID for z, CFWD/CINV for y around CCORE on z, AMID for z.)
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "gpe_fft.cuh"
#include "gpe_internal.h"

namespace gpe {

enum StatusCode { ST_OK = 0, ST_ARG = 1, ST_CUDA = 2, ST_NOT_CONVERGED = 3, ST_NONFINITE = 4, ST_PRECOND = 5 };

// A line of M points is held by Tl = M / E threads, E values each (E = 8 by
// default; E = 4 doubles the threads per line for latency-bound passes).
template <int M, int EV = 8> struct LineCfg {
  static constexpr int E = EV;      // values per thread
  static constexpr int Tl = M / E;  // threads per line
  static_assert(M >= 8 && (M & (M - 1)) == 0, "M must be a power of two >= 8");
  static_assert((EV == 4 || EV == 8) && M >= EV, "E must be 4 or 8");
};

// ---------------------------------------------------------------------------
// Reductions.
//
// Sums are accumulated in double-single arithmetic: an unevaluated pair of
// FP32 numbers (hi, lo), added with Knuth's TwoSum error-free transformation
// (D. E. Knuth, TAOCP vol. 2, 4.2.2) followed by a fast renormalisation
// (T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971).  The pair carries ~48 significant bits
// (relative error ~2^-47 per addition), so sums of FP32 terms lose nothing
// and sums of FP64 terms lose ~1e-14 relative.  On GB300 an FP64 warp
// instruction occupies the FP64 pipe ~64x longer than an FP32 one, so the
// pair arithmetic keeps the many-level block and grid reductions off that
// pipe; totals are converted to FP64 once, for the scalar steps.
// Slots flagged in MAXMASK take the maximum instead (of non-negative values).
// ---------------------------------------------------------------------------
struct Acc {
  float hi, lo;
};

__device__ __forceinline__ Acc acc_from(float x) { return Acc{x, 0.0f}; }
__device__ __forceinline__ Acc acc_from(double x) {
  const float h = (float)x;
  return Acc{h, (float)(x - (double)h)};
}
__device__ __forceinline__ Acc acc_from(dsf x) { return Acc{x.hi, x.lo}; }
__device__ __forceinline__ double acc_to_double(Acc a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ Acc acc_add(Acc a, Acc b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);  // TwoSum: s + e = a.hi + b.hi exactly
  e += a.lo + b.lo;
  const float h = s + e;                      // renormalise (|e| <= ulp(s))
  return Acc{h, e - (h - s)};
}
__device__ __forceinline__ Acc acc_max(Acc a, Acc b) {
  return (b.hi > a.hi || (b.hi == a.hi && b.lo > a.lo)) ? b : a;
}

template <unsigned MAXMASK>
__device__ __forceinline__ Acc red_op(Acc a, Acc b, int k) {
  return ((MAXMASK >> k) & 1u) ? acc_max(a, b) : acc_add(a, b);
}

// Two double-single additions at once on the packed two-wide FP32 pipe: lane by
// lane the same operations in the same order as acc_add (each lane rounds like
// the scalar .rn operation), so the sums are bit-identical with half the
// floating-point instructions.
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ void acc_add2(Acc& a0, Acc& a1, Acc b0, Acc b1) {
  const unsigned long long ah = f2_pack(a0.hi, a1.hi), al = f2_pack(a0.lo, a1.lo);
  const unsigned long long bh = f2_pack(b0.hi, b1.hi), bl = f2_pack(b0.lo, b1.lo);
  const unsigned long long sm = f2add(ah, bh);
  const unsigned long long bp = f2sub(sm, ah);
  unsigned long long e = f2add(f2sub(ah, f2sub(sm, bp)), f2sub(bh, bp));
  e = f2add(e, f2add(al, bl));
  const unsigned long long h = f2add(sm, e);
  const unsigned long long lo = f2sub(e, f2sub(h, sm));
  const float2 H = f2_unpack(h), Lo = f2_unpack(lo);
  a0 = Acc{H.x, Lo.x};
  a1 = Acc{H.y, Lo.y};
}

// v[k] = red_op(v[k], w[k]) for every slot; pairs of sum slots go through acc_add2.
template <int K, unsigned MAXMASK>
__device__ __forceinline__ void red_all(Acc (&v)[K], const Acc (&w)[K]) {
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    if (k + 1 < K && !((MAXMASK >> k) & 1u) && !((MAXMASK >> (k + 1)) & 1u)) {
      acc_add2(v[k], v[k + 1], w[k], w[k + 1]);
    } else {
      v[k] = red_op<MAXMASK>(v[k], w[k], k);
      if (k + 1 < K) v[k + 1] = red_op<MAXMASK>(v[k + 1], w[k + 1], k + 1);
    }
  }
}

__device__ __forceinline__ Acc shfl_acc(unsigned mask, Acc v, int o) {
  return Acc{__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o)};
}

// Fixed-order butterfly over the 32 lanes of a warp (lanes beyond the data
// hold the identity, 0, which also serves the max slots: they are >= 0).
template <int K, unsigned MAXMASK>
__device__ __forceinline__ void warp_tree(Acc (&v)[K]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Acc w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = shfl_acc(0xffffffffu, v[k], o);
    red_all<K, MAXMASK>(v, w);
  }
}

// Block total of v[k] (fixed tree); valid in thread 0 on return.  Warp sums
// by shuffles, then warp 0 combines the per-warp sums with a second shuffle
// tree (no serial loop over warps).
// LEAD = false skips the barrier that protects red_sm from the previous call's
// readers: for callers that alternate between two red_sm buffers, whose other
// barriers already order a buffer's readers before its next writers.
template <int K, unsigned MAXMASK, bool LEAD = true>
__device__ __forceinline__ void block_reduce(Acc (&v)[K], Acc* red_sm) {
  // blockDim.x is a power of two: either a multiple of 32 or one partial warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const int width = blockDim.x < 32 ? (int)blockDim.x : 32;
  const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < width) {
      Acc w[K];
#pragma unroll
      for (int k = 0; k < K; ++k) w[k] = shfl_acc(mask, v[k], o);
      red_all<K, MAXMASK>(v, w);
    }
  }
  if (nw == 1) return;
  if constexpr (LEAD) __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red_sm[warp * K + k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = lane < nw ? red_sm[lane * K + k] : Acc{0.0f, 0.0f};
    warp_tree<K, MAXMASK>(v);
  }
}

// Partials live in a double-sized slot each (an Acc is 8 bytes).
__device__ __forceinline__ Acc* acc_slots(double* p) { return reinterpret_cast<Acc*>(p); }

// Per-block partials, then the last block to finish sums them in a fixed
// order.  Returns true in the last block, with tot[] (FP64) valid in thread 0.
template <int K, unsigned MAXMASK>
__device__ __forceinline__ bool grid_reduce(Acc (&v)[K], const PassArgs& a, double (&tot)[K]) {
  __shared__ Acc red_sm[32 * K];
  __shared__ int s_last;
  block_reduce<K, MAXMASK>(v, red_sm);
  Acc* part = acc_slots(a.partials);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[(size_t)blockIdx.x * kMaxMoments + k] = v[k];
    __threadfence();
    const unsigned prev = atomicAdd(a.ticket, 1u);
    s_last = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  Acc w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = Acc{0.0f, 0.0f};
  // L2-coherent loads, unrolled so that several blocks' partials are in
  // flight at once; the summation order stays fixed.
#pragma unroll 4
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const float2* pb = reinterpret_cast<const float2*>(part + (size_t)b * kMaxMoments);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 x = __ldcg(pb + k);
      w[k] = red_op<MAXMASK>(w[k], Acc{x.x, x.y}, k);
    }
  }
  block_reduce<K, MAXMASK>(w, red_sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = acc_to_double(w[k]);
    *a.ticket = 0u;  // ready for the next pass
  }
  return true;
}

// ---------------------------------------------------------------------------
// Scalar steps (run by one thread of the last block)
// ---------------------------------------------------------------------------
// Constants the scalar steps need (from the pass arguments).
struct Fin {
  double weight, eta, omega;
  int dim, solver;
};

__device__ __forceinline__ Fin fin_of(const PassArgs& a) { return Fin{a.weight, a.eta, a.omega, a.dim, a.solver}; }

// Row n of the iteration log, or null (no log, full, or not the writing block).
__device__ __forceinline__ double* log_row(Ctl* c, bool writer) {
  return (writer && c->log && c->iter < c->log_cap) ? c->log + (size_t)c->iter * kLogFields : nullptr;
}

// After the last H pass: energy terms, lambda_n, lambda~_n, E_n (Section 2, eq. Opt_Alpha).
static __device__ void finalize_H(Ctl* c, const Fin& a, bool writer) {
  const double w = a.weight;
  double kin = 0.0, lz = 0.0;
  for (int ax = 0; ax < a.dim; ++ax) { kin += c->hsum[ax][0]; lz += c->hsum[ax][1]; }
  c->kin = w * kin;
  c->Lz = -w * lz;          // <phi, L_z phi>: the passes sum the symbol without omega
  c->rot = -a.omega * c->Lz;
  c->pot = w * c->hsum[0][2];
  c->U0 = w * c->hsum[0][3];
  c->norm2 = w * c->hsum[0][4];
  c->phimax = sqrt(c->hsum[0][5]);
  const double quad = c->kin + c->rot + c->pot;
  c->lam = quad + a.eta * c->U0;                           // <phi, H phi>
  c->alpha = c->kin + c->pot + a.eta * c->U0;              // lambda~ (no rotation term)
  c->E = quad + 0.5 * a.eta * c->U0;
  if (a.solver) {
    double* row = log_row(c, writer);
    if (row) {
      row[0] = c->iter; row[1] = c->phase; row[2] = c->E; row[3] = c->lam;
      row[6] = c->alpha;
      row[4] = row[5] = row[7] = row[8] = row[9] = row[10] = row[11] = 0.0;
    }
    if (c->log && c->iter + 1 > c->log_len) c->log_len = (c->iter + 1 < c->log_cap) ? c->iter + 1 : c->log_cap;
  }
}

// After C1: residual norms and the stopping rule (eq. Stop_Residual), the
// iteration cap, the optional energy rule, and (mixed phase) stall detection.
static __device__ void finalize_C1(Ctl* c, const Fin& a, const double (&tot)[3], bool writer) {
  c->res_inf = sqrt(tot[0]);
  c->res_l2 = sqrt(a.weight * tot[1]);
  double* row = log_row(c, writer);
  if (row) { row[4] = c->res_inf; row[5] = c->res_l2; }
  const int nphase = c->iter - c->iter_phase0;
  if (!isfinite(c->E) || !isfinite(c->res_inf) || !isfinite(c->lam)) {
    c->status = ST_NONFINITE; c->done = 1;
  } else if (tot[2] > 0.0) {
    c->status = ST_PRECOND; c->done = 1;
  } else if (c->res_inf < c->tol_res_inf || c->stop_dE) {
    c->status = ST_OK; c->done = 1;
  } else if (c->iter >= c->max_iter) {
    c->status = ST_NOT_CONVERGED; c->done = 1;
  } else if (c->lo_phase) {
    // complex64 phase: stop at the single-precision residual floor, estimated
    // as eps32 (max |k|^2/2 + max V + |lambda|) max|phi|, or on a stall near it
    const double floor_est = (c->floor_coef + 5.96e-8 * fabs(c->lam)) * c->phimax;
    const double thr = c->switch_res > 0.0 ? c->switch_res : c->switch_fac * floor_est;
    if (c->res_inf <= 0.5 * c->anchor_res) { c->anchor_res = c->res_inf; c->anchor_iter = c->iter; }
    const bool stalled = c->iter - c->anchor_iter >= c->stall_window && c->res_inf < 3.0 * thr;
    if (c->res_inf < thr || stalled || nphase >= c->max_iter_phase) {
      c->switch_req = 1; c->status = ST_NOT_CONVERGED; c->done = 1;
    }
  } else if (c->stall_switch) {
    // refinement phase: its step moments are single precision; if ||r||_inf
    // has not halved for 4 stall_window iterations, finish in FP64 (after the
    // beta restart ||r||_inf first grows ~10x; on the 256^2 and 128^3 bench
    // problems the longest gap between halvings is ~1500 iterations)
    if (c->res_inf <= 0.5 * c->anchor_res) { c->anchor_res = c->res_inf; c->anchor_iter = c->iter; }
    if (c->iter - c->anchor_iter >= 4 * c->stall_window) {
      c->switch_req = 1; c->status = ST_NOT_CONVERGED; c->done = 1;
    }
  }
}

// After C3: Polak-Ribiere beta+ (eq. CG:PR), gamma = Re<d, phi>, and the
// descent check of Section 5.2 (Re<grad E, p> >= 0 -> gradient step).
// tot: 0 <r,Pr>, 1 Re<r - r_prev, Pr>, 2 Re<Pr,phi>, 3 Re<p_prev,phi>,
//      4 Re<r,p_prev>, 5 Re<r,phi>
static __device__ void finalize_C3(Ctl* c, const Fin& a, const double (&tot)[6], bool writer) {
  const double w = a.weight;
  const double rPr = w * tot[0];
  double beta = 0.0;
  if (!c->restart && c->cg)
    beta = c->beta_rule == 1 ? rPr / c->rPr_prev                  // Fletcher-Reeves (eq. CG:FR)
                             : fmax(w * tot[1] / c->rPr_prev, 0.0);  // Polak-Ribiere beta+
  const double Prphi = w * tot[2], pphi = w * tot[3], rp = w * tot[4], rphi = w * tot[5];
  double gamma = -Prphi + beta * pphi;
  // Re<H phi, p> = Re<r, d> - gamma Re<r, phi> + lambda gamma (1 - ||phi||^2)
  const double desc = -rPr + beta * rp - gamma * rphi + c->lam * gamma * (1.0 - c->norm2);
  c->fallback = 0;
  if (desc >= 0.0) {
    c->fallback = 1; c->fallbacks += 1;
    beta = 0.0; gamma = -Prphi;
  }
  c->beta = beta; c->gamma = gamma; c->rPr = rPr;
  c->rPr_prev = rPr;
  double* row = log_row(c, writer);
  if (row) { row[7] = beta; row[10] = c->fallback; }
}

// sin and cos of a step angle.  Steps are usually tiny, so for |t| < 0.05
// the Maclaurin series (truncation below 1e-18 there: t^9/9! and t^10/10!)
// replaces the general FP64 sincos, which is long on GB300's FP64 pipe.
__device__ __forceinline__ void step_sincos(double t, double* s, double* c) {
  if (fabs(t) < 0.05) {
    const double t2 = t * t;
    *s = t * (1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880)))));
    *c = 1.0 + t2 * (-0.5 + t2 * (1.0 / 24 + t2 * (-1.0 / 720 + t2 * (1.0 / 40320 + t2 * (-1.0 / 3628800)))));
  } else {
    sincos(t, s, c);
  }
}

// Energy change along the geodesic, exact trigonometric polynomial (reading R6),
// for s = sin(theta), c = cos(theta).
__device__ __forceinline__ double delta_E(double s, double cth, double R, double aqq, double lam, double eta,
                                          double U0, double U1, double V2, double UW, double VW, double W2) {
  const double s2 = s * s, c2 = cth * cth;
  return 2.0 * cth * s * R + s2 * (aqq - lam) +
         0.5 * eta * (s2 * s2 * (U0 + W2) + c2 * s2 * (4.0 * V2 + 2.0 * UW) + 4.0 * cth * s * s2 * (VW - U1));
}

// After the last A pass: step size by the model minimiser (eq. theta_opt,
// reading R4) with energy-decrease backtracking (Section 5.1), then the
// retraction scalars for the next H pass.
// asum[0]: 0 Re<H phi,p>, 1 <p,A_x p>+<p,V p>, 2 |p|^2, 3 u v, 4 v^2, 5 u w,
//          6 v w, 7 w^2, 8 v    (u = |phi|^2, v = Re(conj(phi) p), w = |p|^2)
// asum[ax>0][1]: <p, A_ax p>
// Newton's method on d/dt of the step polynomial delta_E (closed-form first
// and second derivatives, with A = aqq - lam, B = eta/2 (U0 + W2),
// C = eta/2 (4 V2 + 2 UW), D = 2 eta (VW - U1)) from the model step t0; t0 is
// kept when the curvature is not positive or the iterate leaves (0, pi/2].
static __device__ double exact_step(double t0, double R, double aqq, double lam, double eta, double U0, double U1,
                                    double V2, double UW, double VW, double W2) {
  const double A = aqq - lam, B = 0.5 * eta * (U0 + W2), C = 0.5 * eta * (4.0 * V2 + 2.0 * UW);
  const double D = 2.0 * eta * (VW - U1);
  double t = t0;
  for (int it = 0; it < 30; ++it) {
    double s, c, s2, c2, s4, c4;
    sincos(t, &s, &c);
    sincos(2.0 * t, &s2, &c2);
    sincos(4.0 * t, &s4, &c4);
    const double d1 = 2.0 * R * c2 + A * s2 + 4.0 * B * s * s * s * c + 0.5 * C * s4 + D * (3.0 * c * c * s * s - s * s * s * s);
    const double d2 = -4.0 * R * s2 + 2.0 * A * c2 + 4.0 * B * (3.0 * s * s * c * c - s * s * s * s) + 2.0 * C * c4 +
                      D * (6.0 * c * s * (c * c - s * s) - 4.0 * s * s * s * c);
    if (!(d2 > 0.0)) return t0;
    const double dt = d1 / d2;
    t -= dt;
    if (!(t > 0.0 && t <= 1.5707963267948966)) return t0;
    if (fabs(dt) <= 1e-15 * fabs(t)) break;
  }
  return t;
}

static __device__ void finalize_A(Ctl* c, const Fin& a, bool writer) {
  const double w = a.weight;
  const double* s0 = c->asum[0];
  const double W1 = w * s0[2];
  const double inv = 1.0 / sqrt(W1);
  double app = s0[1];
  for (int ax = 1; ax < a.dim; ++ax) app += c->asum[ax][1];
  const double R = w * s0[0] * inv;
  const double aqq = w * app * inv * inv;
  const double U1 = w * s0[3] * inv, V2 = w * s0[4] * inv * inv, UW = w * s0[5] * inv * inv;
  const double VW = w * s0[6] * inv * inv * inv, W2 = w * s0[7] * inv * inv * inv * inv;
  const double rho = w * s0[8] * inv;
  const double eta = a.eta, lam = c->lam, U0 = c->U0;
  const double curv = aqq + eta * UW + 2.0 * eta * V2 - lam;
  double th = (curv > 0.0) ? -R / curv : c->theta_default;
  if (c->line_search == 1) th = exact_step(th, R, aqq, lam, eta, U0, U1, V2, UW, VW, W2);
  double sn, cs;
  step_sincos(th, &sn, &cs);
  double dE = delta_E(sn, cs, R, aqq, lam, eta, U0, U1, V2, UW, VW, W2);
  int bt = 0;
  while (!(dE < 0.0) && bt < c->max_backtracks) {
    th *= 0.5; ++bt;
    step_sincos(th, &sn, &cs);
    dE = delta_E(sn, cs, R, aqq, lam, eta, U0, U1, V2, UW, VW, W2);
  }
  const double nrm2 = cs * cs * c->norm2 + 2.0 * cs * sn * rho + sn * sn;
  c->theta = th; c->c = cs; c->s = sn; c->inv_np = inv; c->inv_nrm = 1.0 / sqrt(nrm2);
  c->dE = dE; c->backtracks = bt; c->backtracks_total += bt;
  double* row = log_row(c, writer);
  if (row) { row[8] = th; row[9] = dE; row[11] = bt; }
  c->retract = 1;
  c->restart = 0;
  c->iter += 1;
  if (c->tol_dE > 0.0 && fabs(dE) <= c->tol_dE) c->stop_dE = 1;
  if (!isfinite(dE) || !isfinite(th)) { c->status = ST_NONFINITE; c->done = 1; }
}

__device__ __forceinline__ void set_loop_condition(const PassArgs& a, int keep_going) {
  if (a.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, keep_going ? 1u : 0u);
}

// Scalars a pass body reads (copied from the control block at entry).
struct Scal {
  int retract;
  int pc;  // preconditioner kind (Ctl::pc_kind; API calls: 0, P_C)
  double c, s, inv_np, inv_nrm, lam, alpha, beta, gamma;
};

// The preconditioners of Section 5.4 as P_V^a P_Delta^b P_V^c around the
// Fourier core: exponents of P_V before (pre) and after (post) the core,
// coded 0 (none), 1 (P_V^{1/2}), 2 (P_V), and whether the core divides by
// alpha + |k|^2/2 (P_Delta, eq. PDelta) or is the identity.
//   P_C  = P_V^{1/2} P_Delta P_V^{1/2} (eq. combinedP_12): 1, Delta, 1
//   P_Delta (eq. PDelta): 0, Delta, 0      P_V (eq. PV): 2, identity, 0
//   P_C1 = P_V P_Delta (eq. combinedP): 0, Delta, 2  (P_Delta first)
//   P_C2 = P_Delta P_V (eq. combinedP): 2, Delta, 0  (P_V first)
//   none: 0, identity, 0
__device__ __forceinline__ int pc_pre(int k) { return k == 0 ? 1 : (k == 2 || k == 4) ? 2 : 0; }
__device__ __forceinline__ int pc_post(int k) { return k == 0 ? 1 : k == 3 ? 2 : 0; }
__device__ __forceinline__ bool pc_core(int k) { return !(k == 2 || k == 5); }
template <typename T> __device__ __forceinline__ T pv_factor(T den, int code) {
  return code == 0 ? T(1) : (code == 2 ? T(1) / den : T(1) / sqrt(den));
}

__device__ __forceinline__ Scal scal_of(const Ctl* c, const PassArgs& a) {
  Scal S;
  S.retract = a.solver ? c->retract : 0;
  S.pc = a.solver ? c->pc_kind : 0;
  S.c = c->c; S.s = c->s; S.inv_np = c->inv_np; S.inv_nrm = c->inv_nrm;
  S.lam = a.solver ? c->lam : 0.0;
  S.alpha = a.solver ? c->alpha : (a.api_alpha > 0 ? a.api_alpha : c->alpha);
  S.beta = c->beta; S.gamma = c->gamma;
  return S;
}

// Reduction slots per pass and which of them are maxima.
template <int ROLE> struct Moments { static constexpr int K = 0; static constexpr unsigned MAX = 0u; };
template <> struct Moments<P_HX> { static constexpr int K = 6; static constexpr unsigned MAX = 32u; };
template <> struct Moments<P_HMID> { static constexpr int K = 2; static constexpr unsigned MAX = 0u; };
template <> struct Moments<P_C1> { static constexpr int K = 3; static constexpr unsigned MAX = 1u; };
template <> struct Moments<P_C3> { static constexpr int K = 6; static constexpr unsigned MAX = 0u; };
template <> struct Moments<P_AX> { static constexpr int K = 9; static constexpr unsigned MAX = 0u; };
template <> struct Moments<P_AMID> { static constexpr int K = 1; static constexpr unsigned MAX = 0u; };

// ---------------------------------------------------------------------------
// Multipliers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ const T* tab(const void* p) { return static_cast<const T*>(p); }

// ---------------------------------------------------------------------------
// Contiguous (x) passes.  Block = lpb lines x Tl threads; tid = t + Tl*l.
//
// Three element types: TF for the line transform, TS for the state fields
// (phi, H phi, r_{n-1}, V) and TD for the direction fields (P_C workspace s,
// P r, p).  TF = TS = TD gives the plain complex64 or complex128 passes; the
// refinement passes use TS = double with TF = TD = float for the direction
// (P_C r and the moments of A p), and TF = TS = double, TD = float for H phi.
// ---------------------------------------------------------------------------
// Max threads per block: 512 with single-precision transforms, 256 with double.
template <typename T> struct MaxThreads { static constexpr int value = sizeof(T) == 8 ? 256 : 512; };

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename To, typename From>
__device__ __forceinline__ cplx<To> cconv(From v) { return cmk<cplx<To>>((To)v.x, (To)v.y); }

// One unit of a contiguous pass: lines unit*lpb .. unit*lpb + lpb - 1 (the
// block has lpb * M/8 threads).  Adds this thread's reduction terms to acc[]
// (Moments<ROLE>: sums, or maxima for the slots flagged in MAX).
template <typename TF, typename TS, typename TD, int M, int ROLE, int EV = 8>
__device__ __forceinline__ void xunit(const PassArgs& a, const Scal& S, long long unit, unsigned char* smraw,
                                      Acc* acc) {
  using CF = cplx<TF>;
  using CS = cplx<TS>;
  using CD = cplx<TD>;
  constexpr int E = LineCfg<M, EV>::E, Tl = LineCfg<M, EV>::Tl;
  constexpr int LS = M + M / 16;  // padded line stride in shared memory
  // lines of at most 32 threads lie inside one warp (tid = t + Tl l) and own
  // their shared-memory rows: their transforms need only warp barriers
  constexpr bool W = Tl <= 32;
  CF* sm = reinterpret_cast<CF*>(smraw);

  const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
  const long long line = unit * a.lpb + l;
  const long long base = line * M;
  const int iy = (int)((a.row0 + line) % a.ny);  // row0: global row of local line 0 (cluster slices)
  const CF* __restrict__ tw = static_cast<const CF*>(a.tw);
  const TF* __restrict__ xi = tab<TF>(a.xi[0]);
  const TS* __restrict__ V = tab<TS>(a.V);
  auto si = [l](int pos) { return l * LS + pos + (pos >> 4); };
  const TF invM = TF(1) / TF(M);

  CF v[E];
  if constexpr (ROLE == P_HX) {
    // ---- H_phi f, x part, plus the real-space terms (TF == TS) --------------------
    static_assert(sizeof(TF) == sizeof(TS), "H passes transform the state precision");
    const CS* __restrict__ phi = static_cast<const CS*>(a.phi);
    const CS* __restrict__ f = static_cast<const CS*>(a.f ? a.f : a.phi);
    if (a.pf > 0 && unit + a.pf < a.nblocks) {
      // fields larger than L2: the block about one wave later reads the rows of
      // unit + pf; start bringing them (phi, f, V) into L2 now, 128-byte lines
      const long long e0 = (unit + a.pf) * a.lpb * M;
      const int nb = a.lpb * M * (int)sizeof(CS);
      for (int off = threadIdx.x * 128; off < nb; off += blockDim.x * 128) {
        prefetch_l2(reinterpret_cast<const char*>(phi + e0) + off);
        if (a.f && a.f != a.phi) prefetch_l2(reinterpret_cast<const char*>(f + e0) + off);
      }
      const int nv = a.lpb * M * (int)sizeof(TS);
      for (int off = threadIdx.x * 128; off < nv; off += blockDim.x * 128)
        prefetch_l2(reinterpret_cast<const char*>(V + e0) + off);
    }
    CS ph[E];
    TS vv[E];
    const bool retract = S.retract;
    const TS cc = TS(retract ? S.c * S.inv_nrm : 1.0);
    const TS ss = TS(retract ? S.s * S.inv_np * S.inv_nrm : 0.0);
    const CD* __restrict__ p = static_cast<const CD*>(a.p);
    CS* __restrict__ phi_out = static_cast<CS*>(a.phi_out);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      CS x = phi[g];
      if (retract) {
        const CS pq = cconv<TS>(p[g]);
        x = cmk<CS>(cc * x.x + ss * pq.x, cc * x.y + ss * pq.y);
        phi_out[g] = x;
      }
      ph[q] = x;
      vv[q] = V[g];
      v[q] = cconv<TF>((a.f && !a.solver) ? f[g] : x);
    }
    line_dft<M, E, -1, W>(v, sm, si, t, tw);
    const TF y = tab<TF>(a.xc[1])[iy];
    const TF om = TF(a.omega);
    TF akin = 0, arot = 0;  // arot: the rotation symbol without omega (omega is applied in finalize_H)
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const TF k = xi[t + q * Tl];
      const TF mk = TF(0.5) * k * k, kr = y * k;
      const TF a2 = v[q].x * v[q].x + v[q].y * v[q].y;
      akin += mk * a2; arot += kr * a2;
      v[q] = cscale(v[q], (mk + om * kr) * invM);
    }
    line_dft<M, E, +1, W>(v, sm, si, t, tw);
    CS* __restrict__ tout = static_cast<CS*>(a.t);
    const TS eta = TS(a.eta);
    TS apot = 0, au2 = 0, an2 = 0, umax = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      const TS u = ph[q].x * ph[q].x + ph[q].y * ph[q].y;
      const TS m = vv[q] + eta * u;
      const CS fq = (a.f && !a.solver) ? f[g] : ph[q];  // the operand f (re-read in API mode)
      tout[g] = cmk<CS>(TS(v[q].x) + m * fq.x, TS(v[q].y) + m * fq.y);
      apot += vv[q] * u; au2 += u * u; an2 += u; umax = fmax(umax, u);
    }
    acc[0] = acc_add(acc[0], acc_from(akin * invM));
    acc[1] = acc_add(acc[1], acc_from(arot * invM));
    acc[2] = acc_add(acc[2], acc_from(apot));
    acc[3] = acc_add(acc[3], acc_from(au2));
    acc[4] = acc_add(acc[4], acc_from(an2));
    acc[5] = acc_max(acc[5], acc_from(umax));
  } else if constexpr (ROLE == P_C1) {
    // ---- s = FFT_x[P_V^{1/2} r], r = H phi - lambda phi (solver) or r_in (API) ----
    const CS* __restrict__ phi = static_cast<const CS*>(a.phi);
    const CS* __restrict__ rin = static_cast<const CS*>(a.solver ? a.t : a.r_in);
    const TS lam = TS(S.lam);
    const TS alpha = TS(S.alpha);
    const TS eta = TS(a.eta);
    TS rmax = 0, r2 = 0, bad = 0;
    const int pre = pc_pre(S.pc);
    const bool uses_pv = pre != 0 || pc_post(S.pc) != 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      const CS ph = phi[g];
      CS r = rin[g];
      if (a.solver) r = cmk<CS>(r.x - lam * ph.x, r.y - lam * ph.y);
      const TS den = alpha + V[g] + eta * (ph.x * ph.x + ph.y * ph.y);
      bad += (den > TS(0) || !uses_pv) ? TS(0) : TS(1);
      const TS a2 = r.x * r.x + r.y * r.y;
      rmax = fmax(rmax, a2); r2 += a2;
      v[q] = cconv<TF>(cscale(r, pv_factor(den, pre)));
    }
    line_dft<M, E, -1, W>(v, sm, si, t, tw);
    CD* __restrict__ sout = static_cast<CD*>(a.s);
#pragma unroll
    for (int q = 0; q < E; ++q) sout[base + t + q * Tl] = cconv<TD>(v[q]);
    acc[0] = acc_max(acc[0], acc_from(rmax));
    acc[1] = acc_add(acc[1], acc_from(r2));
    acc[2] = acc_add(acc[2], acc_from(bad));
  } else if constexpr (ROLE == P_C3) {
    // ---- Pr = P_V^{1/2} IFFT_x[s] (the 1/N is applied in the core pass) ----
    const CS* __restrict__ phi = static_cast<const CS*>(a.phi);
    CD* __restrict__ sbuf = static_cast<CD*>(a.s);
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = cconv<TF>(sbuf[base + t + q * Tl]);
    const TS alpha = TS(S.alpha);
    const TS eta = TS(a.eta);
    if (!a.solver) {
      line_dft<M, E, +1, W>(v, sm, si, t, tw);
      CD* __restrict__ out = static_cast<CD*>(a.out);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const long long g = base + t + q * Tl;
        const CS ph = phi[g];
        const TS den = alpha + V[g] + eta * (ph.x * ph.x + ph.y * ph.y);
        out[g] = cconv<TD>(cscale(cconv<TS>(v[q]), pv_factor(den, pc_post(S.pc))));
      }
      return;
    }
    // every operand of the epilogue is loaded before the transform, so the
    // loads overlap it instead of waiting behind its barriers
    const CS* __restrict__ Hphi = static_cast<const CS*>(a.t);
    CS* __restrict__ rprev = static_cast<CS*>(a.r_prev);
    const CD* __restrict__ pprev = static_cast<const CD*>(a.p);
    CS ph[E], hq[E], ro[E];
    CD pp[E];
    TS vv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      ph[q] = phi[g];
      hq[q] = Hphi[g];
      ro[q] = rprev[g];
      pp[q] = pprev[g];
      vv[q] = V[g];
    }
    line_dft<M, E, +1, W>(v, sm, si, t, tw);
    const TS lam = TS(S.lam);
    const int post = pc_post(S.pc);
    TS a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      const TS den = alpha + vv[q] + eta * (ph[q].x * ph[q].x + ph[q].y * ph[q].y);
      const CD Prd = cconv<TD>(cscale(cconv<TS>(v[q]), pv_factor(den, post)));
      sbuf[g] = Prd;
      const CS Pr = cconv<TS>(Prd);  // the stored direction, as later passes see it
      const CS r = cmk<CS>(hq[q].x - lam * ph[q].x, hq[q].y - lam * ph[q].y);
      const CS pq = cconv<TS>(pp[q]);
      a0 += r.x * Pr.x + r.y * Pr.y;
      a1 += (r.x - ro[q].x) * Pr.x + (r.y - ro[q].y) * Pr.y;
      a2 += Pr.x * ph[q].x + Pr.y * ph[q].y;
      a3 += pq.x * ph[q].x + pq.y * ph[q].y;
      a4 += r.x * pq.x + r.y * pq.y;
      a5 += r.x * ph[q].x + r.y * ph[q].y;
      rprev[g] = r;
    }
    acc[0] = acc_add(acc[0], acc_from(a0)); acc[1] = acc_add(acc[1], acc_from(a1));
    acc[2] = acc_add(acc[2], acc_from(a2)); acc[3] = acc_add(acc[3], acc_from(a3));
    acc[4] = acc_add(acc[4], acc_from(a4)); acc[5] = acc_add(acc[5], acc_from(a5));
  } else if constexpr (ROLE == P_AX) {
    // ---- p = -Pr + beta p_prev - gamma phi ; moments for the step size ----
    const CS* __restrict__ phi = static_cast<const CS*>(a.phi);
    const CD* __restrict__ Pr = static_cast<const CD*>(a.s);
    const CS* __restrict__ Hphi = static_cast<const CS*>(a.t);
    CD* __restrict__ pbuf = static_cast<CD*>(a.p);
    const TS beta = TS(S.beta), gamma = TS(S.gamma);
    TS aR = 0, aV = 0, aW1 = 0, aUV = 0, aV2 = 0, aUW = 0, aVW = 0, aW2 = 0, aRho = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const long long g = base + t + q * Tl;
      const CS ph = phi[g], h = Hphi[g];
      const CS pr = cconv<TS>(Pr[g]), pp = cconv<TS>(pbuf[g]);
      const CD pnd = cconv<TD>(cmk<CS>(-pr.x + beta * pp.x - gamma * ph.x, -pr.y + beta * pp.y - gamma * ph.y));
      pbuf[g] = pnd;
      const CS pn = cconv<TS>(pnd);  // moments of the stored p
      v[q] = cconv<TF>(pnd);
      const TS u = ph.x * ph.x + ph.y * ph.y;
      const TS vr = ph.x * pn.x + ph.y * pn.y;
      const TS wq = pn.x * pn.x + pn.y * pn.y;
      aR += h.x * pn.x + h.y * pn.y;
      aV += V[g] * wq;
      aW1 += wq; aUV += u * vr; aV2 += vr * vr; aUW += u * wq; aVW += vr * wq; aW2 += wq * wq; aRho += vr;
    }
    line_dft<M, E, -1, W>(v, sm, si, t, tw);
    const TF y = tab<TF>(a.xc[1])[iy];
    const TF om = TF(a.omega);
    TF akr = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const TF k = xi[t + q * Tl];
      akr += (TF(0.5) * k * k + om * y * k) * (v[q].x * v[q].x + v[q].y * v[q].y);
    }
    acc[0] = acc_add(acc[0], acc_from(aR));
    acc[1] = acc_add(acc_add(acc[1], acc_from(aV)), acc_from(akr * invM));
    acc[2] = acc_add(acc[2], acc_from(aW1)); acc[3] = acc_add(acc[3], acc_from(aUV));
    acc[4] = acc_add(acc[4], acc_from(aV2)); acc[5] = acc_add(acc[5], acc_from(aUW));
    acc[6] = acc_add(acc[6], acc_from(aVW)); acc[7] = acc_add(acc[7], acc_from(aW2));
    acc[8] = acc_add(acc[8], acc_from(aRho));
  }
}

// ---------------------------------------------------------------------------
// Strided (y, z) passes.  Block = tx columns x Tl threads; tid = c + tx*t.
// ---------------------------------------------------------------------------
// One unit of a strided pass: the tile of tx adjacent x-columns number unit
// (block = tx * M/8 threads).  Reduction terms are added to acc[].
template <typename T, int M, int ROLE, int EV = 8>
__device__ __forceinline__ void sunit(const PassArgs& a, const Scal& S, long long unit, unsigned char* smraw,
                                      Acc* acc) {
  using C = cplx<T>;
  constexpr int E = LineCfg<M, EV>::E, Tl = LineCfg<M, EV>::Tl;
  C* sm = reinterpret_cast<C*>(smraw);
  const int tx = a.tx;
  const int c = threadIdx.x % tx, t = threadIdx.x / tx;
  const int xt = (int)(unit % a.ntx);
  const long long outer = unit / a.ntx;
  const int ix = xt * tx + c;
  const long long base = outer * a.outer_stride + ix;
  const long long st = a.stride;
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  auto si = [tx, c](int pos) { return pos * tx + c; };
  const T* __restrict__ xia = tab<T>(a.xi[a.axis]);
  const T invM = T(1) / T(M);

  C v[E];
  if constexpr (ROLE == P_HMID) {
    const C* __restrict__ f = static_cast<const C*>((a.f && !a.solver) ? a.f : a.phi);
    const C* tb = static_cast<const C*>(a.t);
    C tv[E];  // the accumulated t, loaded before the transforms so the loads overlap them
#pragma unroll
    for (int q = 0; q < E; ++q) {
      v[q] = f[base + (t + q * Tl) * st];
      tv[q] = tb[base + (t + q * Tl) * st];
    }
    line_dft<M, E, -1>(v, sm, si, t, tw);
    const T om = T(a.omega);
    const T x = (a.axis == 1) ? tab<T>(a.xc[0])[ix] : T(0);
    const T rx = (a.axis == 1) ? -x : T(0);  // rotation symbol -omega x mu (y), omega applied below; none for z
    T akin = 0, arot = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xia[t + q * Tl];
      const T mk = T(0.5) * k * k, kr = rx * k;
      const T a2 = v[q].x * v[q].x + v[q].y * v[q].y;
      akin += mk * a2; arot += kr * a2;
      v[q] = cscale(v[q], (mk + om * kr) * invM);
    }
    line_dft<M, E, +1>(v, sm, si, t, tw);
    C* __restrict__ dst = static_cast<C*>(a.out ? a.out : a.t);  // API: final pass writes the caller's buffer
#pragma unroll
    for (int q = 0; q < E; ++q) dst[base + (t + q * Tl) * st] = cadd(tv[q], v[q]);
    acc[0] = acc_add(acc[0], acc_from(akin * invM));
    acc[1] = acc_add(acc[1], acc_from(arot * invM));
  } else if constexpr (ROLE == P_CFWD || ROLE == P_CINV || ROLE == P_CCORE) {
    C* __restrict__ sb = static_cast<C*>(a.s);
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sb[base + (t + q * Tl) * st];
    if constexpr (ROLE == P_CINV) {
      line_dft<M, E, +1>(v, sm, si, t, tw);
    } else {
      line_dft<M, E, -1>(v, sm, si, t, tw);
    }
    if constexpr (ROLE == P_CCORE) {
      // (alpha + |k|^2 / 2)^{-1} / N on the full frequency grid (eq. PDelta)
      const T alpha = T(S.alpha);
      const T invN = T(1.0 / ((double)a.nx * a.ny * (a.dim == 3 ? a.nz : 1)));
      const T kx = tab<T>(a.xi[0])[ix];
      T kother = 0;
      if (a.dim == 3) {
        // axis == 2 (z) here; y index is the outer index
        const T ky = tab<T>(a.xi[1])[outer];
        kother = ky * ky;
      }
#pragma unroll
      const bool core = pc_core(S.pc);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const T k = xia[t + q * Tl];
        const T den = alpha + T(0.5) * (kx * kx + kother + k * k);
        v[q] = cscale(v[q], core ? invN / den : invN);
      }
      line_dft<M, E, +1>(v, sm, si, t, tw);
    }
#pragma unroll
    for (int q = 0; q < E; ++q) sb[base + (t + q * Tl) * st] = v[q];
  } else if constexpr (ROLE == P_AMID) {
    const C* __restrict__ pb = static_cast<const C*>(a.p);
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = pb[base + (t + q * Tl) * st];
    line_dft<M, E, -1>(v, sm, si, t, tw);
    const T om = T(a.omega);
    const T x = (a.axis == 1) ? tab<T>(a.xc[0])[ix] : T(0);
    const T rs = (a.axis == 1) ? -om * x : T(0);
    T akr = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xia[t + q * Tl];
      akr += (T(0.5) * k * k + rs * k) * (v[q].x * v[q].x + v[q].y * v[q].y);
    }
    acc[0] = acc_add(acc[0], acc_from(akr * invM));
  }
}


// ---------------------------------------------------------------------------
// Standalone pass kernels (one unit per block): used by the API entry points,
// the graph-captured solve and the host-loop solve.  The last block to finish
// sums the per-block partials in a fixed order and runs the scalar step.
// ---------------------------------------------------------------------------
template <int ROLE, int K>
__device__ __forceinline__ void store_sums(const PassArgs& a, const double (&tot)[K]) {
  Ctl* ctl = a.ctl;
  const Fin F = fin_of(a);
  if constexpr (ROLE == P_HX) {
    for (int k = 0; k < K; ++k) ctl->hsum[0][k] = tot[k];
  } else if constexpr (ROLE == P_HMID) {
    ctl->hsum[a.axis][0] = tot[0];
    ctl->hsum[a.axis][1] = tot[1];
    if (a.last_axis) finalize_H(ctl, F, true);
  } else if constexpr (ROLE == P_C1) {
    finalize_C1(ctl, F, tot, true);
  } else if constexpr (ROLE == P_C3) {
    finalize_C3(ctl, F, tot, true);
  } else if constexpr (ROLE == P_AX) {
    for (int k = 0; k < K; ++k) ctl->asum[0][k] = tot[k];
  } else if constexpr (ROLE == P_AMID) {
    ctl->asum[a.axis][1] = tot[0];
    if (a.last_axis) {
      finalize_A(ctl, F, true);
      set_loop_condition(a, ctl->done ? 0 : 1);
    }
  }
}

template <int ROLE>
__device__ __forceinline__ void reduce_and_finish(const PassArgs& a, const Acc* acc) {
  constexpr int K = Moments<ROLE>::K;
  if (a.nomoments) return;  // uniform over the launch
  if constexpr (K > 0) {
    // the P_C passes reduce only inside a solve
    if ((ROLE == P_C1 || ROLE == P_C3) && !a.solver) return;
    Acc v[K];
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = acc[k];
    if (grid_reduce<K, Moments<ROLE>::MAX>(v, a, tot) && threadIdx.x == 0) store_sums<ROLE, K>(a, tot);
  }
}

template <typename TF, typename TS, typename TD, int M, int ROLE, int EV>
__global__ void __launch_bounds__(MaxThreads<TF>::value < MaxThreads<TS>::value ? MaxThreads<TF>::value : MaxThreads<TS>::value) pass_x(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.solver && a.ctl->done) return;
  const Scal S = scal_of(a.ctl, a);
  Acc acc[kMaxMoments];
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  xunit<TF, TS, TD, M, ROLE, EV>(a, S, blockIdx.x, smraw, acc);
  reduce_and_finish<ROLE>(a, acc);
}

template <typename T, int M, int ROLE, int EV>
__global__ void __launch_bounds__(MaxThreads<T>::value) pass_s(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.solver && a.ctl->done) {
    if (ROLE == P_AMID && a.last_axis && blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(a, 0);
    return;
  }
  const Scal S = scal_of(a.ctl, a);
  Acc acc[kMaxMoments];
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  sunit<T, M, ROLE, EV>(a, S, blockIdx.x, smraw, acc);
  reduce_and_finish<ROLE>(a, acc);
}

// ---------------------------------------------------------------------------
// Host-side dispatch over M
// ---------------------------------------------------------------------------
// Precision modes of a launch: 0 complex64, 1 complex128, 2 refinement split:
// the state (phi, H phi, r_{n-1}, V) and the H phi transforms in double-single
// (dsf, ~48 bits on the FP32 pipe), the direction (P_C workspace, p) in FP32.
template <int MODE, int ROLE> struct ModeTypes;
template <int ROLE> struct ModeTypes<0, ROLE> { using TF = float; using TS = float; using TD = float; };
template <int ROLE> struct ModeTypes<1, ROLE> { using TF = double; using TS = double; using TD = double; };
template <int ROLE> struct ModeTypes<2, ROLE> {
  static constexpr bool h = (ROLE == P_HX || ROLE == P_HMID);
  static constexpr bool state = (ROLE == P_C1 || ROLE == P_C3 || ROLE == P_AX);
  using TF = typename std::conditional<h, dsf, float>::type;
  using TS = typename std::conditional<h || state, dsf, float>::type;
  using TD = float;
};

template <int MODE, int M, int ROLE, int EV>
cudaError_t launch_one(const PassArgs& a, cudaStream_t st) {
  using MT = ModeTypes<MODE, ROLE>;
  using TF = typename MT::TF;
  using C = cplx<TF>;
  constexpr int Tl = LineCfg<M, EV>::Tl;
  constexpr bool contig = (ROLE == P_HX || ROLE == P_C1 || ROLE == P_C3 || ROLE == P_AX);
  int threads, smem;
  if constexpr (contig) {
    threads = Tl * a.lpb;
    smem = a.lpb * (M + M / 16) * (int)sizeof(C);
  } else {
    threads = Tl * a.tx;
    smem = M * a.tx * (int)sizeof(C);
  }
  void (*kern)(PassArgs);
  if constexpr (contig) kern = pass_x<TF, typename MT::TS, typename MT::TD, M, ROLE, EV>;
  else kern = pass_s<TF, M, ROLE, EV>;
  static DeviceOnce attr;
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.set(dev);
  }
  kern<<<a.nblocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// E = 8 for every M; E = 4 (plans chosen by the tuner) for M >= 32, in
// their own translation units (gpe_k_e4_*.cu).
template <int MODE, int ROLE, int EV = 8>
cudaError_t launch_role(const PassArgs& a, cudaStream_t st) {
  if constexpr (EV == 8) {
    switch (a.M) {
      case 8: return launch_one<MODE, 8, ROLE, 8>(a, st);
      case 16: return launch_one<MODE, 16, ROLE, 8>(a, st);
      case 32: return launch_one<MODE, 32, ROLE, 8>(a, st);
      case 64: return launch_one<MODE, 64, ROLE, 8>(a, st);
      case 128: return launch_one<MODE, 128, ROLE, 8>(a, st);
      case 256: return launch_one<MODE, 256, ROLE, 8>(a, st);
      case 512: return launch_one<MODE, 512, ROLE, 8>(a, st);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (a.M) {
      case 32: return launch_one<MODE, 32, ROLE, EV>(a, st);
      case 64: return launch_one<MODE, 64, ROLE, EV>(a, st);
      case 128: return launch_one<MODE, 128, ROLE, EV>(a, st);
      case 256: return launch_one<MODE, 256, ROLE, EV>(a, st);
      case 512: return launch_one<MODE, 512, ROLE, EV>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
}

}  // namespace gpe
