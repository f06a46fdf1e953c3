// gpe_cluster.cuh -- H_phi f on 2D fields held in a thread-block cluster's
// distributed shared memory (arXiv:1611.02045, Section 2 operator with the
// discretisation of eq. FFTdiscret, Section 3).
//
// One cluster of C = M/16 CTAs transforms one M x M field (M in [32, 256]).
// CTA r owns rows 16r .. 16r+15.  The x part of H is applied row by row in
// the owning CTA (line DFT, multiplier 1/2 xi^2 + omega y xi, inverse DFT,
// plus the real-space term (V + eta|phi|^2) f); the result t stays in shared
// memory.  After a cluster barrier, CTA r takes the 16 columns 16r .. 16r+15:
// it gathers them from every CTA's copy of f through distributed shared memory,
// applies the y part (1/2 mu^2 - omega x mu) and adds it into the owners' t.
// After a second barrier each CTA writes its rows of t = H_phi f.  Global
// memory is touched once per point: read f (and phi when it differs), read
// V, write the result -- the algorithmic traffic of H phi.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "gpe_fft.cuh"
#include "gpe_internal.h"

namespace gpe {

namespace cg = cooperative_groups;

constexpr int kClusterRows = 16;  // rows (and columns) per CTA

struct ClusterHArgs {
  int M;             // nx == ny
  int nbatch;        // fields
  long long stride;  // elements between consecutive fields
  double eta, omega;
  const void* xi;    // x frequencies, kernel precision
  const void* xiy;   // y frequencies
  const void* xc;    // x coordinates
  const void* yc;    // y coordinates
  const void* tw;    // twiddles e^{-2 pi i m/M}
  const void* V;     // potential, one M x M array shared by all fields
  const void* phi;   // density fields
  const void* f;     // operands (may equal phi)
  void* out;         // results
};

// Two CTAs per SM in single precision (two fields in flight per SM group).
template <typename T> struct ClusterMinBlocks { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

template <typename T, int M>
__global__ void __launch_bounds__((M / 8) * kClusterRows, ClusterMinBlocks<T>::value) cluster_apply_H(ClusterHArgs a) {
  using C = cplx<T>;
  constexpr int E = 8, Tl = M / 8, R = kClusterRows;
  constexpr int LS = M + M / 16;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int csize = (int)cl.num_blocks();
  const long long field = blockIdx.x / csize;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* fs = reinterpret_cast<C*>(smraw);  // [R][M] operand rows of this CTA
  C* ts = fs + R * M;                     // [R][M] accumulator rows of this CTA
  C* xs = ts + R * M;                     // exchange scratch: [R][LS] (x) or [M][R] (y)
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const T* __restrict__ xi = static_cast<const T*>(a.xi);
  const T invM = T(1) / T(M);
  const T om = T(a.omega);
  const long long fb = field * a.stride;

  // ---- x part, rows of this CTA -------------------------------------------------
  {
    const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
    const int y = rank * R + l;
    const C* __restrict__ f = static_cast<const C*>(a.f);
    const C* __restrict__ phi = static_cast<const C*>(a.phi);
    const T* __restrict__ V = static_cast<const T*>(a.V);
    const bool same = (a.f == a.phi);
    C w[E];
    T m[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * Tl;
      const long long g = fb + (long long)y * M + x;
      w[q] = f[g];
      const C ph = same ? w[q] : phi[g];
      m[q] = V[(long long)y * M + x] + T(a.eta) * (ph.x * ph.x + ph.y * ph.y);
      fs[l * M + x] = w[q];
    }
    auto si = [l](int pos) { return l * LS + pos + (pos >> 4); };
    line_dft<M, E, -1>(w, xs, si, t, tw);
    const T yy = static_cast<const T*>(a.yc)[y];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xi[t + q * Tl];
      w[q] = cscale(w[q], (T(0.5) * k * k + om * yy * k) * invM);
    }
    line_dft<M, E, +1>(w, xs, si, t, tw);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const C v = fs[l * M + t + q * Tl];  // the operand, kept in shared memory
      ts[l * M + t + q * Tl] = cmk<C>(w[q].x + m[q] * v.x, w[q].y + m[q] * v.y);
    }
  }
  cl.sync();  // every CTA's rows of f and t are complete and visible

  // ---- y part, columns of this CTA, rows gathered from the whole cluster ------
  {
    const int c = threadIdx.x % R, t = threadIdx.x / R;
    const int x = rank * R + c;
    C w[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int y = t + q * Tl;
      const C* src = cl.map_shared_rank(fs, (unsigned)(y / R));
      w[q] = src[(y % R) * M + x];
    }
    __syncthreads();  // the x part's readers of xs are done (line_dft syncs again before writing)
    auto si = [c](int pos) { return pos * R + c; };
    line_dft<M, E, -1>(w, xs, si, t, tw);
    const T xx = static_cast<const T*>(a.xc)[x];
    const T* __restrict__ xiy = static_cast<const T*>(a.xiy);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xiy[t + q * Tl];
      w[q] = cscale(w[q], (T(0.5) * k * k - om * xx * k) * invM);
    }
    line_dft<M, E, +1>(w, xs, si, t, tw);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int y = t + q * Tl;
      C* dst = cl.map_shared_rank(ts, (unsigned)(y / R));
      C* e = dst + (y % R) * M + x;
      *e = cadd(*e, w[q]);  // each element of t has exactly one writer in the cluster
    }
  }
  cl.sync();  // all additions into this CTA's t are done; nobody reads our smem after this

  // ---- write rows ---------------------------------------------------------------
  {
    const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
    const int y = rank * R + l;
    C* __restrict__ out = static_cast<C*>(a.out);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int x = t + q * Tl;
      out[fb + (long long)y * M + x] = ts[l * M + x];
    }
  }
}

template <typename T, int M>
cudaError_t launch_cluster_apply_H_one(const ClusterHArgs& a, cudaStream_t st) {
  using C = cplx<T>;
  constexpr int R = kClusterRows;
  const int csize = M / R;
  const int threads = (M / 8) * R;
  const size_t smem = (size_t)(2 * R * M + R * (M + M / 16)) * sizeof(C);
  auto kern = cluster_apply_H<T, M>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nbatch * csize));
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
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace gpe
