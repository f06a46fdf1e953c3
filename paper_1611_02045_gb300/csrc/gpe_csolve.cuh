// gpe_csolve.cuh -- the complex64 phase of PCG_C (arXiv:1611.02045,
// Algorithm 2 with the descent check of Section 5.2 and the step-size rule of
// Section 5.1) for one 2D instance held entirely in a thread-block cluster's
// distributed shared memory.
//
// A cluster of C = M/16 CTAs solves one M x M problem (M in [32, 256]).  CTA
// r keeps rows 16r .. 16r+15 of every iteration field in its shared memory:
// phi_n, t = H phi_n, s (P_C workspace, then P r_n), p and r_{n-1}.  The x
// passes run on those rows with the same unit bodies as the global-memory
// passes (pointed at shared memory); the y passes gather their 16 columns from
// the whole cluster through distributed shared memory.  Each reduction writes
// one partial per CTA into CTA 0's shared memory, meets at a hardware cluster
// barrier, and every CTA sums the C partials in the same order and runs the
// scalar step on its own copy of the control block, so no global memory is
// touched inside the loop except the potential V (read-only, L2-resident) and
// the per-iteration log.
#pragma once
#include <cooperative_groups.h>

#include "gpe_passes.cuh"

namespace gpe {

namespace cgc = cooperative_groups;

struct ClusterSolveArgs {
  PassArgs base;     // geometry, physics and tables (float); field pointers are set per CTA
  float2* phi;       // [M][M] complex64 phi, in: phi_0, out: the last iterate
  const float* V;    // [M][M] potential (float)
  Ctl* ctl;          // control block (in: options and retraction scalars; out: final state)
};

constexpr int kCSRows = 16;

// One y pass over this CTA's 16 columns; rows gathered from the cluster.
//   P_HMID : t += (1/2 mu^2 - omega x mu) phi  (+ Parseval kinetic/rotation sums)
//   P_CCORE: s  = IFFT_y[ FFT_y(s) / (alpha + |k|^2/2) ] / N
//   P_AMID : Parseval sum of <p, (1/2 mu^2 - omega x mu) p>
template <int M, int ROLE>
__device__ __forceinline__ void cs_yunit(const cgc::cluster_group& cl, int rank, float2* fld, float2* tacc,
                                         float2* xs, const PassArgs& a, const Scal& S, Acc* acc) {
  constexpr int E = 8, Tl = M / 8, R = kCSRows;
  const int c = threadIdx.x % R, t = threadIdx.x / R;
  const int x = rank * R + c;
  const float2* __restrict__ tw = static_cast<const float2*>(a.tw);
  const float* __restrict__ xiy = static_cast<const float*>(a.xi[1]);
  const float invM = 1.0f / float(M);
  float2 w[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int y = t + q * Tl;
    const float2* src = cl.map_shared_rank(fld, (unsigned)(y / R));
    w[q] = src[(y % R) * M + x];
  }
  auto si = [c](int pos) { return pos * R + c; };
  // the last users of xs were the x unit before the reduction's cluster barrier
  line_dft<M, E, -1, false, false>(w, xs, si, t, tw);
  if constexpr (ROLE == P_HMID || ROLE == P_AMID) {
    const float om = float(a.omega);
    const float rx = -static_cast<const float*>(a.xc[0])[x];
    float akin = 0.f, arot = 0.f;  // arot: rotation symbol with omega (A p) or without it (H phi, finalize_H applies it)
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const float k = xiy[t + q * Tl];
      const float mk = 0.5f * k * k, kr = rx * k, mr = om * kr;
      const float a2 = w[q].x * w[q].x + w[q].y * w[q].y;
      akin += mk * a2;
      arot += (ROLE == P_AMID ? mr : kr) * a2;
      w[q] = cscale(w[q], (mk + mr) * invM);
    }
    if constexpr (ROLE == P_AMID) {
      acc[0] = acc_add(acc[0], acc_from((akin + arot) * invM));
      return;
    } else {
      acc[0] = acc_add(acc[0], acc_from(akin * invM));
      acc[1] = acc_add(acc[1], acc_from(arot * invM));
      line_dft<M, E, +1>(w, xs, si, t, tw);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int y = t + q * Tl;
        float2* dst = cl.map_shared_rank(tacc, (unsigned)(y / R));
        float2* e = dst + (y % R) * M + x;
        *e = cadd(*e, w[q]);  // one writer per element in the cluster
      }
    }
  } else {
    static_assert(ROLE == P_CCORE, "y roles: HMID, CCORE, AMID");
    const float alpha = float(S.alpha);
    const float invN = 1.0f / float(M * M);
    const float kx = static_cast<const float*>(a.xi[0])[x];
    const bool core = pc_core(S.pc);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const float k = xiy[t + q * Tl];
      w[q] = cscale(w[q], core ? invN / (alpha + 0.5f * (kx * kx + k * k)) : invN);
    }
    line_dft<M, E, +1>(w, xs, si, t, tw);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int y = t + q * Tl;
      float2* dst = cl.map_shared_rank(fld, (unsigned)(y / R));
      dst[(y % R) * M + x] = w[q];
    }
  }
}

// Cluster-wide fixed-order sum of the CTAs' block totals (tot[] in FP64,
// valid in thread 0 of every CTA on return: only thread 0 runs the scalar
// steps).  part[2][C][kMaxMoments] lives in CTA 0's shared memory and red_sm
// holds two block buffers; parity alternates between reductions, so a slow
// reader never sees the next reduction's partials, and the cluster barrier of
// the reduction in between orders a buffer's readers before its next writers:
// no block barrier before the block sum and none after the cluster sum.
template <int K, unsigned MAXMASK>
__device__ __forceinline__ void cs_reduce(const cgc::cluster_group& cl, int rank, int csize, const Acc* acc,
                                          Acc* part, int& parity, Acc* red_sm, double* tot) {
  Acc v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = acc[k];
  block_reduce<K, MAXMASK, false>(v, red_sm + parity * 32 * kMaxMoments);
  Acc* p0 = cl.map_shared_rank(part, 0u) + (size_t)parity * kCSRows * kMaxMoments;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) p0[rank * kMaxMoments + k] = v[k];
  }
  cl.sync();
  if (threadIdx.x < 32) {
    // lane r takes CTA r's partials; fixed-order shuffle tree across the lanes
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = lane < csize ? p0[lane * kMaxMoments + k] : Acc{0.0f, 0.0f};
    warp_tree<K, MAXMASK>(v);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] = acc_to_double(v[k]);
    }
  }
  parity ^= 1;
}

template <int M>
__global__ void __launch_bounds__((M / 8) * kCSRows) cluster_solve(ClusterSolveArgs P) {
  constexpr int R = kCSRows, LS = M + M / 16;
  cgc::cluster_group cl = cgc::this_cluster();
  const int rank = (int)cl.block_rank();
  const int csize = (int)cl.num_blocks();
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* phi_s = reinterpret_cast<float2*>(smraw);
  float2* t_s = phi_s + R * M;
  float2* s_s = t_s + R * M;
  float2* p_s = s_s + R * M;
  float2* r_s = p_s + R * M;
  float2* xs = r_s + R * M;  // exchange scratch, R * LS elements
  __shared__ Ctl S;
  __shared__ Acc part[2 * kCSRows * kMaxMoments];
  __shared__ Acc red_sm[2 * 32 * kMaxMoments];  // two buffers, alternating with the reductions
  __shared__ double tot[kMaxMoments];

  const int row0 = rank * R;
  // load this CTA's rows of phi_0; p_{-1} = r_{-1} = 0
  for (int i = threadIdx.x; i < R * M; i += blockDim.x) {
    phi_s[i] = P.phi[(size_t)row0 * M + i];
    p_s[i] = make_float2(0.f, 0.f);
    r_s[i] = make_float2(0.f, 0.f);
  }
  if (threadIdx.x == 0) S = *P.ctl;
  cl.sync();

  // x-unit arguments: the same unit bodies as the global passes, on shared rows
  __shared__ PassArgs ax_s;
  if (threadIdx.x == 0) {
    ax_s = P.base;
    ax_s.lpb = R;
    ax_s.row0 = row0;
    ax_s.solver = 1;
    ax_s.phi = phi_s;
    ax_s.phi_out = phi_s;
    ax_s.f = nullptr;
    ax_s.t = t_s;
    ax_s.s = s_s;
    ax_s.p = p_s;
    ax_s.r_prev = r_s;
    ax_s.V = P.V + (size_t)row0 * M;
  }
  __syncthreads();
  const PassArgs& ax = ax_s;
  const Fin F = fin_of(ax);
  const bool writer = rank == 0;
  unsigned char* xsb = reinterpret_cast<unsigned char*>(xs);
  int parity = 0;
  Acc acc[kMaxMoments];
  auto zero = [&]() {
#pragma unroll
    for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.f, 0.f};
  };

  while (!S.done) {
    // ---- H phi_n (x pass folds in the retraction to phi_n) ----
    Scal sc = scal_of(&S, ax);
    zero();
    xunit<float, float, float, M, P_HX>(ax, sc, 0, xsb, acc);
    cs_reduce<6, 32u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0)
      for (int k = 0; k < 6; ++k) S.hsum[0][k] = tot[k];
    zero();
    cs_yunit<M, P_HMID>(cl, rank, phi_s, t_s, xs, ax, sc, acc);
    cs_reduce<2, 0u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0) {
      S.hsum[1][0] = tot[0];
      S.hsum[1][1] = tot[1];
      finalize_H(&S, F, writer);
    }
    __syncthreads();
    // ---- residual, stopping rule, P_C r_n ----
    sc = scal_of(&S, ax);
    zero();
    xunit<float, float, float, M, P_C1>(ax, sc, 0, xsb, acc);
    cs_reduce<3, 1u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0) {
      const double t3[3] = {tot[0], tot[1], tot[2]};
      finalize_C1(&S, F, t3, writer);
    }
    __syncthreads();
    if (S.done) break;
    cs_yunit<M, P_CCORE>(cl, rank, s_s, nullptr, xs, ax, sc, acc);
    cl.sync();
    zero();
    xunit<float, float, float, M, P_C3>(ax, sc, 0, xsb, acc);
    cs_reduce<6, 0u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0) {
      const double t6[6] = {tot[0], tot[1], tot[2], tot[3], tot[4], tot[5]};
      finalize_C3(&S, F, t6, writer);
    }
    __syncthreads();
    // ---- p_n and the step size ----
    sc = scal_of(&S, ax);
    zero();
    xunit<float, float, float, M, P_AX>(ax, sc, 0, xsb, acc);
    cs_reduce<9, 0u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0)
      for (int k = 0; k < 9; ++k) S.asum[0][k] = tot[k];
    zero();
    cs_yunit<M, P_AMID>(cl, rank, p_s, nullptr, xs, ax, sc, acc);
    cs_reduce<1, 0u>(cl, rank, csize, acc, part, parity, red_sm, tot);
    if (threadIdx.x == 0) {
      S.asum[1][1] = tot[0];
      finalize_A(&S, F, writer);
    }
    __syncthreads();
  }
  // write back this CTA's rows of the last iterate and (rank 0) the control block
  for (int i = threadIdx.x; i < R * M; i += blockDim.x) P.phi[(size_t)row0 * M + i] = phi_s[i];
  if (writer && threadIdx.x == 0) *P.ctl = S;
  cl.sync();  // no CTA leaves while others may still address its shared memory
}

template <int M>
constexpr size_t cluster_solve_smem() {
  return (size_t)(5 * kCSRows * M + kCSRows * (M + M / 16)) * sizeof(float2);
}

// Kernel attributes (dynamic shared memory, non-portable cluster size), set
// once per device; call before any stream capture that launches the kernel.
template <int M>
cudaError_t cluster_solve_attrs() {
  static DeviceOnce attr;
  const int dev = DeviceOnce::device();
  if (attr.done(dev)) return cudaSuccess;
  auto kern = cluster_solve<M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cluster_solve_smem<M>());
  if (e != cudaSuccess) return e;
  if (M / kCSRows > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  attr.set(dev);
  return cudaSuccess;
}

template <int M>
cudaError_t launch_cluster_solve_one(const ClusterSolveArgs& P, cudaStream_t st) {
  constexpr int R = kCSRows;
  const int csize = M / R;
  const int threads = (M / 8) * R;
  const size_t smem = cluster_solve_smem<M>();
  auto kern = cluster_solve<M>;
  cudaError_t e = cluster_solve_attrs<M>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

}  // namespace gpe
