// gpe_misc.cu -- pass dispatch and the small elementwise kernels around a
// solve (precision conversion, initial normalisation).
#include "gpe_internal.h"
#include "gpe_ds.cuh"

namespace gpe {

static cudaError_t launch_pass_f32(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: case P_HMID: return launch_group_f32_h(pass, a, st);
    case P_AX: case P_AMID: return launch_group_f32_a(pass, a, st);
    default: return launch_group_f32_c(pass, a, st);
  }
}

static cudaError_t launch_pass_f64(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: case P_HMID: return launch_group_f64_h(pass, a, st);
    case P_AX: case P_AMID: return launch_group_f64_a(pass, a, st);
    default: return launch_group_f64_c(pass, a, st);
  }
}

static cudaError_t launch_pass_f32_e4(Pass pass, const PassArgs& a, cudaStream_t st) {
  switch (pass) {
    case P_HX: case P_HMID: return launch_group_f32_h_e4(pass, a, st);
    case P_AX: case P_AMID: return launch_group_f32_a_e4(pass, a, st);
    default: return launch_group_f32_c_e4(pass, a, st);
  }
}

static cudaError_t launch_pass_e4(int mode, Pass pass, const PassArgs& a, cudaStream_t st) {
  if (mode == 0) return launch_pass_f32_e4(pass, a, st);
  if (mode == 1) {
    switch (pass) {
      case P_HX: case P_HMID: return launch_group_f64_h_e4(pass, a, st);
      case P_AX: case P_AMID: return launch_group_f64_a_e4(pass, a, st);
      default: return launch_group_f64_c_e4(pass, a, st);
    }
  }
  switch (pass) {
    case P_HX: case P_HMID: case P_C1: case P_C3: case P_AX: return launch_group_split_e4(pass, a, st);
    default: return launch_pass_f32_e4(pass, a, st);
  }
}

cudaError_t launch_pass(int mode, Pass pass, const PassArgs& a, cudaStream_t st) {
  if (a.E == 4) return launch_pass_e4(mode, pass, a, st);
  // complex64 passes through the TMA pipelines where the plan and the fields allow:
  // the x passes (H phi; in a solve also C1, C3 and AX) and every strided pass (also
  // the single-precision strided passes of the refinement phase, mode 2)
  const bool strided = pass == P_HMID || pass == P_CFWD || pass == P_CCORE || pass == P_CINV || pass == P_AMID;
  const bool xc = pass == P_C1 || pass == P_C3 || pass == P_AX;
  if ((mode == 0 && (strided || pass == P_HX || xc)) || (mode == 2 && strided && pass != P_HMID)) {
    bool used = false;
    const cudaError_t e = pass == P_HX ? launch_hx_bulk(a, st, &used)
                          : xc        ? launch_xc_bulk(pass, a, st, &used)
                                      : launch_strided_tma(pass, a, st, &used);
    if (e != cudaSuccess || used) return e;
  }
  if (mode == 0) return launch_pass_f32(pass, a, st);
  if (mode == 1) return launch_pass_f64(pass, a, st);
  // refinement split: H phi and the state in double-single, the strided
  // direction passes are plain complex64.
  switch (pass) {
    case P_HX: case P_HMID: case P_C1: case P_C3: case P_AX: return launch_group_split(pass, a, st);
    default: return launch_pass_f32(pass, a, st);
  }
}

__global__ void k_c128_to_c64(const double2* __restrict__ s, float2* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = s[i];
    d[i] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void k_c64_to_c128(const float2* __restrict__ s, double2* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = s[i];
    d[i] = make_double2((double)v.x, (double)v.y);
  }
}
__global__ void k_d2f(const double* __restrict__ s, float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

// double-single <-> complex64 / complex128 (the refinement state)
__global__ void k_c64_to_ds(const float2* __restrict__ s, dsc* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = s[i];
    dsc o;
    o.x = dsf(v.x);
    o.y = dsf(v.y);
    d[i] = o;
  }
}
__global__ void k_ds_to_c128(const dsc* __restrict__ s, double2* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dsc v = s[i];
    d[i] = make_double2((double)v.x, (double)v.y);
  }
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

cudaError_t launch_convert_c128_to_c64(const void* src, void* dst, long long n, cudaStream_t st) {
  k_c128_to_c64<<<grid_for(n), 256, 0, st>>>((const double2*)src, (float2*)dst, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_c64_to_c128(const void* src, void* dst, long long n, cudaStream_t st) {
  k_c64_to_c128<<<grid_for(n), 256, 0, st>>>((const float2*)src, (double2*)dst, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_c64_to_ds(const void* src, void* dst, long long n, cudaStream_t st) {
  k_c64_to_ds<<<grid_for(n), 256, 0, st>>>((const float2*)src, (dsc*)dst, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_ds_to_c128(const void* src, void* dst, long long n, cudaStream_t st) {
  k_ds_to_c128<<<grid_for(n), 256, 0, st>>>((const dsc*)src, (double2*)dst, n);
  return cudaGetLastError();
}
__global__ void k_d2ds(const double* __restrict__ s, dsf* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = dsf(s[i]);
}
cudaError_t launch_d2ds(const double* src, void* dst, long long n, cudaStream_t st) {
  k_d2ds<<<grid_for(n), 256, 0, st>>>(src, (dsf*)dst, n);
  return cudaGetLastError();
}
cudaError_t launch_d2f(const double* src, float* dst, long long n, cudaStream_t st) {
  k_d2f<<<grid_for(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// One bisection step for the Thomas-Fermi chemical potential (eq. TF_App with
// mu fixed by the normalisation ||phi^TF|| = 1): S(mid) = h^d sum max(mid - V, 0) / eta
// with mid = (lo + hi) / 2; the last block to finish replaces lo (S < 1) or hi.
constexpr int kTfThreads = 256;
__global__ void __launch_bounds__(kTfThreads) k_tf_bisect(const double* __restrict__ V, long long n, double weight,
                                                         double eta, double* state, double* __restrict__ partials,
                                                         unsigned* ticket) {
  __shared__ double sm[kTfThreads / 32];
  __shared__ int s_last;
  const double mid = 0.5 * (__ldcg(state) + __ldcg(state + 1));  // written by the previous launch
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += fmax(mid - V[i], 0.0);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kTfThreads / 32; ++w) b += sm[w];
    partials[blockIdx.x] = b;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(partials + b);
  if (weight * tot / eta < 1.0) state[0] = mid;
  else state[1] = mid;
  *ticket = 0u;
}
cudaError_t launch_tf_bisect(const double* V, long long n, double weight, double eta, double* state,
                             double* partials, unsigned* ticket, cudaStream_t st) {
  long long g = (n + 8LL * kTfThreads - 1) / (8LL * kTfThreads);
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  k_tf_bisect<<<(int)g, kTfThreads, 0, st>>>(V, n, weight, eta, state, partials, ticket);
  return cudaGetLastError();
}

__global__ void k_tf_fill(const double* __restrict__ V, long long n, double eta, const double* state,
                          double2* __restrict__ phi) {
  const double mu = 0.5 * (__ldcg(state) + __ldcg(state + 1));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    phi[i] = make_double2(sqrt(fmax(mu - V[i], 0.0) / eta), 0.0);
}
cudaError_t launch_tf_fill(const double* V, long long n, double eta, const double* state, void* phi128,
                           cudaStream_t st) {
  k_tf_fill<<<grid_for(n), 256, 0, st>>>(V, n, eta, state, (double2*)phi128);
  return cudaGetLastError();
}

// Epilogue of gpe_energy_grad: grad_phi <- 2 h^d H_phi phi in place (Section 2,
// nabla E = 2 H_phi phi, h^d converting to the coefficient vector) and
// grad_V = h^d |phi|^2.  Either output may be null.
template <typename C>
__global__ void k_grad_epilogue(const C* __restrict__ phi, C* __restrict__ gphi, double* __restrict__ gV, long long n,
                                double weight) {
  using R = decltype(C::x);
  const R two_w = R(2.0 * weight);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (gphi) {
      const C h = gphi[i];
      C g;
      g.x = two_w * h.x;
      g.y = two_w * h.y;
      gphi[i] = g;
    }
    if (gV) {
      const C v = phi[i];
      const double re = (double)v.x, im = (double)v.y;
      gV[i] = weight * (re * re + im * im);
    }
  }
}
cudaError_t launch_grad_epilogue(int prec, const void* phi, void* gphi, double* gV, long long n, double weight,
                                 cudaStream_t st) {
  if (prec == 1)
    k_grad_epilogue<double2><<<grid_for(n), 256, 0, st>>>((const double2*)phi, (double2*)gphi, gV, n, weight);
  else
    k_grad_epilogue<float2><<<grid_for(n), 256, 0, st>>>((const float2*)phi, (float2*)gphi, gV, n, weight);
  return cudaGetLastError();
}

__device__ __forceinline__ bool phase_failed(int status) { return status == 4 || status == 5; }  // non-finite, P_V

__global__ void k_batch_between(const float2* __restrict__ s, double2* __restrict__ d128, dsc* __restrict__ dds,
                                long long n, const Ctl* __restrict__ ctl) {
  if (phase_failed(ctl->status)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = s[i];
    d128[i] = make_double2((double)v.x, (double)v.y);
    dsc w;
    w.x = dsf(v.x);
    w.y = dsf(v.y);
    dds[i] = w;
  }
}
cudaError_t launch_batch_between(const void* phi64, void* phi128, void* phids, long long n, const Ctl* ctl,
                                 cudaStream_t st) {
  k_batch_between<<<grid_for(n), 256, 0, st>>>((const float2*)phi64, (double2*)phi128, (dsc*)phids, n, ctl);
  return cudaGetLastError();
}

__global__ void k_batch_gate(Ctl* ctl, cudaGraphConditionalHandle cond) {
  Ctl& c = *ctl;
  c.iters_lo = c.iter;
  const bool go_on = (c.switch_req || c.status == 0) && !phase_failed(c.status);
  unsigned refine = 0;
  if (go_on && c.iter < c.max_iter) {
    c.done = 0; c.status = 0; c.switch_req = 0; c.lo_phase = 0; c.phase = 1; c.restart = 1; c.stop_dE = 0;
    c.iter_phase0 = c.iter; c.max_iter_phase = c.max_iter;
    c.stall_switch = 1; c.anchor_res = 1e300; c.anchor_iter = c.iter;
    refine = 1;
  }
  cudaGraphSetConditional(cond, refine);
}

__global__ void k_batch_gate64(Ctl* ctl, cudaGraphConditionalHandle cond) {
  Ctl& c = *ctl;
  unsigned run = 0;
  if (c.phase == 1 && c.lo_phase == 0 && c.stall_switch && c.switch_req && c.iter < c.max_iter) {
    c.iters_hi = c.iter;
    c.done = 0; c.status = 0; c.switch_req = 0; c.phase = 2; c.restart = 1; c.stop_dE = 0;
    c.iter_phase0 = c.iter; c.max_iter_phase = c.max_iter; c.stall_switch = 0;
    run = 1;
  }
  cudaGraphSetConditional(cond, run);
}
cudaError_t launch_batch_gate64(Ctl* ctl, unsigned long long cond, cudaStream_t st) {
  k_batch_gate64<<<1, 1, 0, st>>>(ctl, (cudaGraphConditionalHandle)cond);
  return cudaGetLastError();
}
cudaError_t launch_batch_gate(Ctl* ctl, unsigned long long cond, cudaStream_t st) {
  k_batch_gate<<<1, 1, 0, st>>>(ctl, (cudaGraphConditionalHandle)cond);
  return cudaGetLastError();
}

__global__ void k_batch_final(const dsc* __restrict__ s, double2* __restrict__ d, long long n, const Ctl* __restrict__ ctl) {
  if (ctl->phase != 1 || ctl->lo_phase != 0 || phase_failed(ctl->status)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const dsc v = s[i];
    d[i] = make_double2((double)v.x, (double)v.y);
  }
}
cudaError_t launch_batch_final(const void* phids, void* phi128, long long n, const Ctl* ctl, cudaStream_t st) {
  k_batch_final<<<grid_for(n), 256, 0, st>>>((const dsc*)phids, (double2*)phi128, n, ctl);
  return cudaGetLastError();
}

// Fixed-order FP64 sum of |phi|^2 over all blocks (runs once per solve
// phase): per-block partials, the last block to finish sums them in block
// order and arms the control block: c = 1, s = 0, inv_nrm = 1 / ||phi||,
// retract = 1, so that the next H pass normalises phi in place.
constexpr int kNormThreads = 256;
template <typename C>
__global__ void __launch_bounds__(kNormThreads) k_init_norm(const C* __restrict__ phi, long long n, double weight,
                                                            Ctl* ctl, double* __restrict__ partials,
                                                            unsigned* ticket) {
  __shared__ double sm[kNormThreads / 32];
  __shared__ int s_last;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C v = phi[i];
    const double re = (double)v.x, im = (double)v.y;
    acc += re * re + im * im;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kNormThreads / 32; ++w) b += sm[w];
    partials[blockIdx.x] = b;
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(partials + b);
  ctl->c = 1.0;
  ctl->s = 0.0;
  ctl->inv_np = 0.0;
  ctl->inv_nrm = 1.0 / sqrt(weight * tot);
  ctl->retract = 1;
  *ticket = 0u;  // ready for the next reduction
}

cudaError_t launch_init_norm(int prec, const void* phi, long long n, double weight, Ctl* ctl, double* partials,
                             unsigned* ticket, cudaStream_t st) {
  long long g = (n + 8LL * kNormThreads - 1) / (8LL * kNormThreads);
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  const int grid = (int)g;
  if (prec == 1) k_init_norm<double2><<<grid, kNormThreads, 0, st>>>((const double2*)phi, n, weight, ctl, partials, ticket);
  else if (prec == 2) k_init_norm<dsc><<<grid, kNormThreads, 0, st>>>((const dsc*)phi, n, weight, ctl, partials, ticket);
  else k_init_norm<float2><<<grid, kNormThreads, 0, st>>>((const float2*)phi, n, weight, ctl, partials, ticket);
  return cudaGetLastError();
}

}  // namespace gpe
