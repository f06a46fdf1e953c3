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
  int E;             // values per thread: 16 (single precision, M >= 64) or 8 (also when 0)
  int rows;          // streaming form (E = 16): rows per CTA, 16 (also when 0) or 32
  int* flow_ctr;     // dataflow form (gpe_hflow.cu): zeroed counters, at least nbatch + 2 ints (or null)
  int flow_cap;      // ints in flow_ctr
  int* status;       // device int set to GPE_ERR_TIMEOUT when a bounded wait gives up (or null)
};

// The dataflow form of the batched H phi for 256 x 256 complex64 fields with
// f == phi (gpe_hflow.cu); *used = false when the call does not qualify (the
// caller then launches a cluster form).
cudaError_t launch_h_batch_flow(const ClusterHArgs& a, int* ctr, int ctr_cap, int* status, cudaStream_t st,
                                bool* used);
size_t h_batch_flow_counters(int nbatch);

// Two CTAs per SM in single precision (two fields in flight per SM group).
template <typename T> struct ClusterMinBlocks { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

// Shared memory per CTA: operand rows, accumulator rows, and the exchange
// buffer (rows of the x part or columns of the y part, padded).
template <typename T, int M> struct ClusterHSmem {
  static constexpr int LS = M + M / 16;  // padded line stride
  static constexpr size_t bytes = (size_t)(2 * kClusterRows * M + kClusterRows * LS) * sizeof(cplx<T>);
};

// EV values per thread: 8 (radix-8 then 8/4/2 Stockham stages, two exchanges
// per 256-point transform) or 16 (radix-16 stages: one exchange, half the
// shared-memory traffic, half the threads).
template <typename T, int M, int EV>
__global__ void __launch_bounds__((M / EV) * kClusterRows, ClusterMinBlocks<T>::value) cluster_apply_H(ClusterHArgs a) {
  using C = cplx<T>;
  constexpr int E = EV, Tl = M / EV, R = kClusterRows;
  constexpr int LS = ClusterHSmem<T, M>::LS;
  static_assert(Tl <= 32 && (32 % Tl) == 0, "a row's threads lie inside one warp");
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

  // ---- x part, rows of this CTA: row l is transformed by the Tl threads
  //      t + Tl l, inside one warp, in its own exchange row (warp barriers) ----
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
    line_dft<M, E, -1, true>(w, xs, si, t, tw);
    const T yy = static_cast<const T*>(a.yc)[y];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xi[t + q * Tl];
      w[q] = cscale(w[q], (T(0.5) * k * k + om * yy * k) * invM);
    }
    line_dft<M, E, +1, true>(w, xs, si, t, tw);
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
    auto si = [c](int pos) { return pos * R + c; };
    line_dft<M, E, -1>(w, xs, si, t, tw);  // its first barrier also retires the x part's use of xs
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

// 16-byte asynchronous copy global -> shared (cached in L2 only) and its group
// control (cp.async, sm_80 and later).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Streaming form of the batched H phi: each resident cluster loops over the
// fields cluster_id, cluster_id + #clusters, ...; while the columns of field k
// are transformed, the rows of field k + #clusters are already being copied
// into the second row buffer.  The x part stores t = A_x f + (V + eta|phi|^2) f
// straight to out; the y part adds its columns' A_y f into out (the lines are
// still in L2), so no accumulator rows are kept and one cluster barrier per
// field suffices:
//   wait rows(k) -> x part(k) -> cluster barrier -> prefetch rows(k+1)
//   -> y part(k) [gathers rows(k) from the cluster]
// After the barrier of field k every CTA has finished the y part of field
// k - 1, so the buffer that held rows(k - 1) is free for rows(k + 1).
// Requires f (and phi) 16-byte aligned.
// Rows per CTA RR: 16 (clusters of M/16 CTAs, two CTAs per SM) or 32 (clusters
// of M/32 CTAs, one 512-thread CTA per SM at M = 256 with E = 16).
template <typename T, int RR> struct StreamMinBlocks { static constexpr int value = RR == 16 ? ClusterMinBlocks<T>::value : 1; };

// Exchange layout of the x part: row l, position p at l * XLS + p + XP * (p / 16).
// At M = 256 with E = 16 the pad is 2 per 16 (16-byte aligned runs of 16 for
// the vector stores of dft256x16), else 1 per 16.  (Column transforms kept
// inside one warp -- two columns per warp, padded row buffers -- were measured
// 2x slower: their cluster gathers and output stores touch 16 rows per warp
// instruction instead of two contiguous 128-byte segments.)
template <int M, int EV> struct StreamX {
  static constexpr bool fast = (M == 256 && EV == 16);
  static constexpr int XP = fast ? 2 : 1;
  static constexpr int XLS = M + XP * (M / 16);
  static constexpr int RS = M;
};
template <typename T, int M, int EV, int RR> struct StreamSmem {
  using C = cplx<T>;
  static constexpr size_t rows = (size_t)2 * RR * StreamX<M, EV>::RS * sizeof(C);
  static constexpr size_t xs = (size_t)RR * StreamX<M, EV>::XLS * sizeof(C);  // >= M * RR (y part)
  static constexpr size_t tws = StreamX<M, EV>::fast ? (size_t)16 * kTw256Stride * sizeof(float4) : 0;
  static constexpr size_t bytes = rows + xs + tws;
};

template <typename T, int M, int EV, int RR>
__global__ void __launch_bounds__((M / EV) * RR, StreamMinBlocks<T, RR>::value)
    cluster_apply_H_stream(ClusterHArgs a) {
  using C = cplx<T>;
  constexpr int E = EV, Tl = M / EV, R = RR;
  constexpr bool FAST = StreamX<M, EV>::fast;
  constexpr int XP = StreamX<M, EV>::XP, XLS = StreamX<M, EV>::XLS, RS = StreamX<M, EV>::RS;
  constexpr int NT = Tl * R;  // threads per CTA
  static_assert(Tl <= 32 && (32 % Tl) == 0, "a row's threads lie inside one warp");
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int csize = (int)cl.num_blocks();
  const long long cid = blockIdx.x / csize, ncl = gridDim.x / csize;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* rows = reinterpret_cast<C*>(smraw);  // [2][R][RS] row buffers
  C* xs = rows + 2 * R * RS;               // [R][XLS] (x), [M][R] or [R][XLS] (y) exchange
  float4* tws = reinterpret_cast<float4*>(smraw + StreamSmem<T, M, EV, RR>::rows + StreamSmem<T, M, EV, RR>::xs);
  const C* __restrict__ f = static_cast<const C*>(a.f);
  const C* __restrict__ phi = static_cast<const C*>(a.phi);
  const T* __restrict__ V = static_cast<const T*>(a.V);
  C* out = static_cast<C*>(a.out);
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const T* __restrict__ xi = static_cast<const T*>(a.xi);
  const T* __restrict__ xiy = static_cast<const T*>(a.xiy);
  const T invM = T(1) / T(M);
  const T om = T(a.omega), eta = T(a.eta);
  const bool same = (a.f == a.phi);
  if constexpr (FAST) dft256_twiddles(tws, reinterpret_cast<const float2*>(tw));  // read after the first barrier

  // rows R rank .. R rank + R - 1 of field fld (R M contiguous elements) into rows of stride RS
  auto fetch = [&](long long fld, C* dst) {
    const char* src = reinterpret_cast<const char*>(f + fld * a.stride + (long long)rank * R * M);
    char* d = reinterpret_cast<char*>(dst);
    constexpr int per_row = M * (int)sizeof(C) / 16, chunks = R * per_row;
    for (int i = threadIdx.x; i < chunks; i += NT) {
      const int r = i / per_row, j = i - r * per_row;
      cp_async16(d + (size_t)r * RS * sizeof(C) + 16 * j, src + 16 * (long long)i);
    }
    cp_async_commit();
  };
  if (cid < a.nbatch) fetch(cid, rows);
  int k = 0;
  for (long long fld = cid; fld < a.nbatch; fld += ncl, ++k) {
    C* fs = rows + (k & 1) * R * RS;
    C* fn = rows + ((k & 1) ^ 1) * R * RS;
    cp_async_wait_all();
    __syncthreads();  // rows(k) complete in fs; every warp is done with xs (y part of k - 1)
    const long long fb = fld * a.stride;

    // ---- x part: row l by the Tl threads t + Tl l (one warp, warp barriers) ----
    {
      const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
      const int y = rank * R + l;
      // row bases once: the per-q offsets q Tl below are compile-time constants
      const C* frow = fs + l * RS + t;
      const T* Vrow = V + y * M + t;
      C* orow = out + fb + (long long)y * M + t;
      C w[E];
      T m[E];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        w[q] = frow[q * Tl];
        const C ph = same ? w[q] : phi[fb + (long long)y * M + t + q * Tl];
        m[q] = Vrow[q * Tl] + eta * (ph.x * ph.x + ph.y * ph.y);
      }
      auto si = [l](int pos) { return l * XLS + pos + XP * (pos >> 4); };
      if constexpr (FAST) dft256x16<-1, true, true>(w, xs, si, t, tws);
      else line_dft<M, E, -1, true>(w, xs, si, t, tw);
      const T yy = static_cast<const T*>(a.yc)[y];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const T kx = xi[t + q * Tl];
        w[q] = cscale(w[q], (T(0.5) * kx * kx + om * yy * kx) * invM);
      }
      if constexpr (FAST) dft256x16<+1, true, true>(w, xs, si, t, tws);
      else line_dft<M, E, +1, true>(w, xs, si, t, tw);
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const C v = frow[q * Tl];
        orow[q * Tl] = cmk<C>(w[q].x + m[q] * v.x, w[q].y + m[q] * v.y);
      }
    }
    cl.sync();  // rows(k) of every CTA visible; t rows stored; y parts of k - 1 finished
    if (fld + ncl < a.nbatch) fetch(fld + ncl, fn);

    // ---- y part: columns R rank .. R rank + R - 1, rows gathered from the cluster ----
    {
      const int c = threadIdx.x % R, t = threadIdx.x / R;
      const int x = rank * R + c;
      C* ocol = out + fb + (long long)t * M + x;
      // row y = t + q Tl lives in CTA y / R at local row y % R
      C w[E], tv[E];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int y = t + q * Tl;
        const C* src = cl.map_shared_rank(fs, (unsigned)(y / R));
        w[q] = src[(y % R) * RS + x];
      }
      // t = A_x f + (V + eta|phi|^2) f of these columns, stored by the rows' owners before
      // the barrier: loaded now so that the loads overlap the transforms
#pragma unroll
      for (int q = 0; q < E; ++q) tv[q] = __ldcg(ocol + q * Tl * M);
      auto si = [c](int pos) { return pos * R + c; };
      // the first barrier of the transform retires the x part's use of xs
      if constexpr (FAST) dft256x16<-1, false, false>(w, xs, si, t, tws);
      else line_dft<M, E, -1>(w, xs, si, t, tw);
      const T xx = static_cast<const T*>(a.xc)[x];
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const T ky = xiy[t + q * Tl];
        w[q] = cscale(w[q], (T(0.5) * ky * ky - om * xx * ky) * invM);
      }
      if constexpr (FAST) dft256x16<+1, false, false>(w, xs, si, t, tws);
      else line_dft<M, E, +1>(w, xs, si, t, tw);
#pragma unroll
      for (int q = 0; q < E; ++q) ocol[q * Tl * M] = cadd(tv[q], w[q]);
    }
  }
  cl.sync();  // no CTA leaves while others may still gather from its rows
}

template <typename T, int M, int EV>
cudaError_t launch_cluster_apply_H_one(const ClusterHArgs& a, cudaStream_t st) {
  constexpr int R = kClusterRows;
  const int csize = M / R;
  const int threads = (M / EV) * R;
  const size_t smem = ClusterHSmem<T, M>::bytes;
  auto kern = cluster_apply_H<T, M, EV>;
  static DeviceOnce attr;
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr.set(dev);
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

// Streaming launcher: as many clusters as can be resident (at most one per
// field); false in *ok when the kernel cannot be used (f or phi not 16-byte
// aligned), so the caller launches the one-field-per-cluster form.
template <typename T, int M, int EV, int RR>
cudaError_t launch_cluster_apply_H_stream(const ClusterHArgs& a, cudaStream_t st, bool* ok) {
  *ok = false;
  if ((reinterpret_cast<uintptr_t>(a.f) & 15u) != 0 || (reinterpret_cast<uintptr_t>(a.phi) & 15u) != 0) return cudaSuccess;
  constexpr int R = RR;
  const int csize = M / R;
  const int threads = (M / EV) * R;
  const size_t smem = StreamSmem<T, M, EV, RR>::bytes;
  auto kern = cluster_apply_H_stream<T, M, EV, RR>;
  static std::atomic<int> max_clusters_dev[64];  // per device; 0 = not yet queried
  const int dev = DeviceOnce::device();
  int max_clusters = (dev >= 0 && dev < 64) ? max_clusters_dev[dev].load() : 0;
  cudaLaunchConfig_t cfg = {};
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
  if (max_clusters <= 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    int n = 0;
    cfg.gridDim = dim3((unsigned)csize);
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess || n < 1) { cudaGetLastError(); n = 1; }
    max_clusters = n;
    if (dev >= 0 && dev < 64) max_clusters_dev[dev].store(n);
  }
  const int ncl = a.nbatch < max_clusters ? a.nbatch : max_clusters;
  cfg.gridDim = dim3((unsigned)(ncl * csize));
  *ok = true;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace gpe
