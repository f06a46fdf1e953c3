// gpe_adjoint.cu -- pointwise and reduction kernels of the tangent-space
// adjoint solve (gpe_tangent_solve): the projected conjugate gradient method
// for K z = P g on {z : <phi, z> = 0}, with
//   K f = H_phi f + eta |phi|^2 f + eta phi^2 conj(f) - lambda f
// (the operator of 1/2 grad^2 E(phi)[f, f] - lambda ||f||^2, Section 2) and
// P h = h - <phi, h> phi (the tangent projector M_phi of Section 2 with the
// phase direction i phi removed too).  H_phi f and the preconditioner P_C are
// the pass kernels of the solver; this file adds the fused epilogues, the
// inner products (FP64 sums, fixed order) and the scalar steps, which run on
// the device so that the host reads scalars only at convergence checks.
#include "gpe_internal.h"

namespace gpe {

namespace {

constexpr int kDotThreads = 256;

template <typename C> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

__device__ __forceinline__ double2 dconj_mul(double ax, double ay, double bx, double by) {
  // conj(a) * b
  return make_double2(ax * bx + ay * by, ax * by - ay * bx);
}

// Block sum of NV doubles (shuffle tree within warps, then warp 0 over the
// warp results; fixed order), written to partials[blockIdx.x * NV + j].
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ partials) {
  __shared__ double sm[kDotThreads / 32][NV];
#pragma unroll
  for (int j = 0; j < NV; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sm[warp][j] = v[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double x = lane < kDotThreads / 32 ? sm[lane][j] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) partials[(size_t)blockIdx.x * NV + j] = x;
    }
  }
}

// Up to three complex inner products sum conj(x_j) y_j (x_j null: skipped).
template <typename C>
__global__ void __launch_bounds__(kDotThreads) k_dots(const C* __restrict__ x0, const C* __restrict__ y0,
                                                      const C* __restrict__ x1, const C* __restrict__ y1,
                                                      const C* __restrict__ x2, const C* __restrict__ y2, long long n,
                                                      double* __restrict__ partials) {
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (x0) { const C a = x0[i], b = y0[i]; const double2 d = dconj_mul(a.x, a.y, b.x, b.y); v[0] += d.x; v[1] += d.y; }
    if (x1) { const C a = x1[i], b = y1[i]; const double2 d = dconj_mul(a.x, a.y, b.x, b.y); v[2] += d.x; v[3] += d.y; }
    if (x2) { const C a = x2[i], b = y2[i]; const double2 d = dconj_mul(a.x, a.y, b.x, b.y); v[4] += d.x; v[5] += d.y; }
  }
  block_sum_store<6>(v, partials);
}

// q <- q + eta |phi|^2 p + eta phi^2 conj(p) - lam p  (q holds H_phi p on entry),
// then the sums <phi, q>, <p, q>, <p, phi>.
template <typename C>
__global__ void __launch_bounds__(kDotThreads) k_hess_epi(const C* __restrict__ phi, const C* __restrict__ p,
                                                          C* __restrict__ q, long long n, double eta, double lam,
                                                          double* __restrict__ partials) {
  using R = typename Real<C>::type;
  const R e = R(eta), l = R(lam);
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C f = phi[i], d = p[i];
    C h = q[i];
    const R u = f.x * f.x + f.y * f.y;
    const R s2x = f.x * f.x - f.y * f.y, s2y = R(2) * f.x * f.y;  // phi^2
    // phi^2 conj(p) = (s2x + i s2y)(d.x - i d.y)
    const R cx = s2x * d.x + s2y * d.y, cy = s2y * d.x - s2x * d.y;
    h.x += e * (u * d.x + cx) - l * d.x;
    h.y += e * (u * d.y + cy) - l * d.y;
    q[i] = h;
    double2 t = dconj_mul(f.x, f.y, h.x, h.y); v[0] += t.x; v[1] += t.y;
    t = dconj_mul(d.x, d.y, h.x, h.y); v[2] += t.x; v[3] += t.y;
    t = dconj_mul(d.x, d.y, f.x, f.y); v[4] += t.x; v[5] += t.y;
  }
  block_sum_store<6>(v, partials);
}

// z += a p; r -= a (q - c phi); and the sum |r|^2.
template <typename C>
__global__ void __launch_bounds__(kDotThreads) k_step(C* __restrict__ z, C* __restrict__ r, const C* __restrict__ p,
                                                      const C* __restrict__ q, const C* __restrict__ phi, long long n,
                                                      const AdjScalars* __restrict__ S, double* __restrict__ partials) {
  using R = typename Real<C>::type;
  if (S->stop) return;  // converged or broken down: leave z and r as they are
  const R a = R(S->a), cr = R(S->c_re), ci = R(S->c_im);
  double v[2] = {0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C d = p[i], h = q[i], f = phi[i];
    C zz = z[i], rr = r[i];
    const R qx = h.x - (cr * f.x - ci * f.y), qy = h.y - (cr * f.y + ci * f.x);
    zz.x += a * d.x; zz.y += a * d.y;
    rr.x -= a * qx; rr.y -= a * qy;
    z[i] = zz; r[i] = rr;
    v[0] += (double)rr.x * rr.x + (double)rr.y * rr.y;
  }
  block_sum_store<2>(v, partials);
}

// h_out = h_in - c phi (c complex from S), h_out may alias h_in.
template <typename C>
__global__ void k_proj(const C* __restrict__ h_in, C* __restrict__ h_out, const C* __restrict__ phi, long long n,
                       const AdjScalars* __restrict__ S) {
  using R = typename Real<C>::type;
  const R cr = R(S->c_re), ci = R(S->c_im);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C h = h_in[i], f = phi[i];
    C o;
    o.x = h.x - (cr * f.x - ci * f.y);
    o.y = h.y - (cr * f.y + ci * f.x);
    h_out[i] = o;
  }
}

// p = (y - c phi) + beta p (beta = 0: p is not read).
template <typename C>
__global__ void k_dir(C* __restrict__ p, const C* __restrict__ y, const C* __restrict__ phi, long long n,
                      const AdjScalars* __restrict__ S) {
  using R = typename Real<C>::type;
  if (S->stop) return;
  const R cr = R(S->c_re), ci = R(S->c_im), b = R(S->beta);
  const bool keep = S->beta != 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C h = y[i], f = phi[i];
    C o;
    o.x = h.x - (cr * f.x - ci * f.y);
    o.y = h.y - (cr * f.y + ci * f.x);
    if (keep) { const C q = p[i]; o.x += b * q.x; o.y += b * q.y; }
    p[i] = o;
  }
}

// Fixed-order sum of the block partials (NV per block), then the scalar step.
__global__ void k_finish(const double* __restrict__ partials, int nblk, int nv, double weight, int stage,
                         AdjScalars* __restrict__ S) {
  __shared__ double sm[32][6];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int j = 0; j < nv; ++j) v[j] += partials[(size_t)b * nv + j];
  for (int j = 0; j < 6; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int j = 0; j < 6; ++j) sm[warp][j] = v[j];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t[6] = {0, 0, 0, 0, 0, 0};
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
    for (int j = 0; j < 6; ++j) t[j] += sm[w][j];
  for (int j = 0; j < 6; ++j) t[j] *= weight;  // weighted inner products
  if (S->stop) return;  // the solve has ended; later kernels of the last round change nothing
  switch (stage) {
    case ADJ_PROJ:  // t = <phi, h>
      S->c_re = t[0]; S->c_im = t[1];
      break;
    case ADJ_BB:  // t = ||r0||^2
      S->bb = t[0]; S->rr = t[0];
      if (!isfinite(t[0])) { S->bad = 3; S->stop = 1; }
      else if (t[0] == 0.0) S->stop = 1;  // P g = 0: z = 0
      break;
    case ADJ_PQ: {  // t = <phi, q>, <p, q>, <p, phi>;  Re<p, q - c phi>
      S->c_re = t[0]; S->c_im = t[1];
      // <p, c phi> = c <p, phi>
      const double cpr = t[0] * t[4] - t[1] * t[5];
      S->pq = t[2] - cpr;
      if (!(S->pq > 0.0) || !isfinite(S->pq)) { S->bad = 1; S->stop = 1; }  // K not positive on the tangent space
      else S->a = S->ry / S->pq;
      break;
    }
    case ADJ_RR:  // t = ||r||^2
      S->rr = t[0];
      S->iters += 1;
      if (!isfinite(t[0])) { S->bad = 3; S->stop = 1; }
      else if (t[0] <= S->tol2 * S->bb) S->stop = 1;  // ||r|| <= tol ||P g||
      break;
    case ADJ_RY:        // t = <phi, y>, <r, y>, <r, phi>;  Re<r, y - c phi>
    case ADJ_RY_FIRST: {
      S->c_re = t[0]; S->c_im = t[1];
      const double crp = t[0] * t[4] - t[1] * t[5];
      const double ry = t[2] - crp;
      S->beta = (stage == ADJ_RY_FIRST) ? 0.0 : ry / S->ry;
      if (!(ry > 0.0) || !isfinite(ry)) { S->bad = 2; S->stop = 1; }  // preconditioner not positive
      S->ry = ry;
      break;
    }
    default:
      break;
  }
}

// rhs = s g_rho phi (s = 2 / h^d: the weighted gradient of a loss of the
// density |phi|^2 whose coefficient gradient is g_rho).
template <typename C>
__global__ void k_density_rhs(const C* __restrict__ phi, const double* __restrict__ g_rho, C* __restrict__ rhs,
                              long long n, double s) {
  using R = typename Real<C>::type;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C f = phi[i];
    const R k = R(s * g_rho[i]);
    C o;
    o.x = k * f.x;
    o.y = k * f.y;
    rhs[i] = o;
  }
}

// grad_V = -h^d Re(conj(z) phi)
template <typename C>
__global__ void k_dV_from_z(const C* __restrict__ phi, const C* __restrict__ z, double* __restrict__ gV, long long n,
                            double weight) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C f = phi[i], q = z[i];
    gV[i] = -weight * ((double)q.x * f.x + (double)q.y * f.y);
  }
}

int grid_of(long long n, int max_blocks) {
  long long g = (n + 4LL * kDotThreads - 1) / (4LL * kDotThreads);
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

}  // namespace

cudaError_t adj_dots(int prec, const void* x0, const void* y0, const void* x1, const void* y1, const void* x2,
                     const void* y2, long long n, double weight, int stage, AdjScalars* S, double* partials,
                     int max_blocks, cudaStream_t st) {
  const int g = grid_of(n, max_blocks);
  if (prec == 1)
    k_dots<double2><<<g, kDotThreads, 0, st>>>((const double2*)x0, (const double2*)y0, (const double2*)x1,
                                               (const double2*)y1, (const double2*)x2, (const double2*)y2, n, partials);
  else
    k_dots<float2><<<g, kDotThreads, 0, st>>>((const float2*)x0, (const float2*)y0, (const float2*)x1,
                                              (const float2*)y1, (const float2*)x2, (const float2*)y2, n, partials);
  k_finish<<<1, 1024, 0, st>>>(partials, g, 6, weight, stage, S);
  return cudaGetLastError();
}

cudaError_t adj_hess_epi(int prec, const void* phi, const void* p, void* q, long long n, double eta, double lam,
                         double weight, AdjScalars* S, double* partials, int max_blocks, cudaStream_t st) {
  const int g = grid_of(n, max_blocks);
  if (prec == 1)
    k_hess_epi<double2><<<g, kDotThreads, 0, st>>>((const double2*)phi, (const double2*)p, (double2*)q, n, eta, lam,
                                                   partials);
  else
    k_hess_epi<float2><<<g, kDotThreads, 0, st>>>((const float2*)phi, (const float2*)p, (float2*)q, n, eta, lam,
                                                  partials);
  k_finish<<<1, 1024, 0, st>>>(partials, g, 6, weight, ADJ_PQ, S);
  return cudaGetLastError();
}

cudaError_t adj_step(int prec, void* z, void* r, const void* p, const void* q, const void* phi, long long n,
                     double weight, AdjScalars* S, double* partials, int max_blocks, cudaStream_t st) {
  const int g = grid_of(n, max_blocks);
  if (prec == 1)
    k_step<double2><<<g, kDotThreads, 0, st>>>((double2*)z, (double2*)r, (const double2*)p, (const double2*)q,
                                               (const double2*)phi, n, S, partials);
  else
    k_step<float2><<<g, kDotThreads, 0, st>>>((float2*)z, (float2*)r, (const float2*)p, (const float2*)q,
                                              (const float2*)phi, n, S, partials);
  k_finish<<<1, 1024, 0, st>>>(partials, g, 2, weight, ADJ_RR, S);
  return cudaGetLastError();
}

cudaError_t adj_proj(int prec, const void* h_in, void* h_out, const void* phi, long long n, const AdjScalars* S,
                     cudaStream_t st) {
  const int g = grid_of(n, 4096);
  if (prec == 1) k_proj<double2><<<g, kDotThreads, 0, st>>>((const double2*)h_in, (double2*)h_out, (const double2*)phi, n, S);
  else k_proj<float2><<<g, kDotThreads, 0, st>>>((const float2*)h_in, (float2*)h_out, (const float2*)phi, n, S);
  return cudaGetLastError();
}

cudaError_t adj_dir(int prec, void* p, const void* y, const void* phi, long long n, const AdjScalars* S, cudaStream_t st) {
  const int g = grid_of(n, 4096);
  if (prec == 1) k_dir<double2><<<g, kDotThreads, 0, st>>>((double2*)p, (const double2*)y, (const double2*)phi, n, S);
  else k_dir<float2><<<g, kDotThreads, 0, st>>>((float2*)p, (const float2*)y, (const float2*)phi, n, S);
  return cudaGetLastError();
}

cudaError_t adj_density_rhs(int prec, const void* phi, const double* g_rho, void* rhs, long long n, double s,
                            cudaStream_t st) {
  const int g = grid_of(n, 4096);
  if (prec == 1) k_density_rhs<double2><<<g, kDotThreads, 0, st>>>((const double2*)phi, g_rho, (double2*)rhs, n, s);
  else k_density_rhs<float2><<<g, kDotThreads, 0, st>>>((const float2*)phi, g_rho, (float2*)rhs, n, s);
  return cudaGetLastError();
}

cudaError_t adj_dV_from_z(int prec, const void* phi, const void* z, double* gV, long long n, double weight,
                          cudaStream_t st) {
  const int g = grid_of(n, 4096);
  if (prec == 1) k_dV_from_z<double2><<<g, kDotThreads, 0, st>>>((const double2*)phi, (const double2*)z, gV, n, weight);
  else k_dV_from_z<float2><<<g, kDotThreads, 0, st>>>((const float2*)phi, (const float2*)z, gV, n, weight);
  return cudaGetLastError();
}

}  // namespace gpe
