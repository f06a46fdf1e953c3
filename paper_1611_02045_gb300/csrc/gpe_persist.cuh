// gpe_persist.cuh -- the whole PCG_C loop (arXiv:1611.02045, Algorithm 2) as
// one persistent cooperative kernel.
//
// Every pass of an iteration becomes a phase of the kernel: the blocks stride
// over the pass's work units (the same unit bodies as the standalone pass
// kernels), then meet at a grid barrier.  Reductions go through per-block
// partials that every block sums in the same fixed order, so every block
// holds bit-identical totals and runs the scalar step (lambda, convergence,
// beta, step size) on its own shared-memory copy of the control block; block
// 0 also writes the log and, at the end, the control block.  No kernel is
// launched and nothing returns to the host until the loop ends.
//
// Grid barriers spin on a generation counter with an iteration limit: a wait
// that gives up sets the error flag, the kernel leaves its loop and reports
// GPE_ERR_TIMEOUT instead of hanging.  Co-residency of all blocks is
// guaranteed by the cooperative launch.
#pragma once
#include "gpe_passes.cuh"

namespace gpe {

struct PersistArgs {
  PassArgs hx, hy, hz, c1, cfwd, ccore, cinv, c3, ax, ay, az;
  Ctl* ctl;
  double* partials;  // [2][gridDim.x][kMaxMoments]
  unsigned* bar;     // [0] arrivals, [1] generation (zero before launch)
  int* err;          // 1 when a barrier wait gave up (zero before launch)
  long long units;   // work units per pass (equal for every pass: square/cubic grids)
  long long spin_limit;  // polls of one barrier wait before it gives up (kSpinLimit by default)
};

// ~2^26 polls of >= 32 ns: seconds, far beyond any legitimate wait.
constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ bool grid_sync(const PersistArgs& P) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = P.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(P.bar, 1u) == gridDim.x - 1) {
      atomicExch(P.bar, 0u);
      __threadfence();
      atomicAdd(P.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        // give up after spin_limit polls, or at once when another block already gave up
        if (++spins > P.spin_limit || *(volatile int*)P.err) {
          ok = 0;
          atomicExch(P.err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok && (*(volatile int*)P.err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Block partials -> barrier -> fixed-order total in every block (tot[] in
// shared memory, FP64, valid in all threads on return).
template <int K, unsigned MAXMASK>
__device__ __forceinline__ bool all_reduce(const PersistArgs& P, const Acc* acc, int& parity, double* tot) {
  __shared__ Acc red_sm[32 * kMaxMoments];
  Acc v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = acc[k];
  block_reduce<K, MAXMASK>(v, red_sm);
  Acc* part = acc_slots(P.partials) + (size_t)parity * gridDim.x * kMaxMoments;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[(size_t)blockIdx.x * kMaxMoments + k] = v[k];
  }
  if (!grid_sync(P)) return false;
  Acc w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = Acc{0.0f, 0.0f};
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
  }
  __syncthreads();
  parity ^= 1;
  return true;
}

template <int MODE, int ROLE> using TFof = typename ModeTypes<MODE, ROLE>::TF;
template <int MODE, int ROLE> using TSof = typename ModeTypes<MODE, ROLE>::TS;
template <int MODE, int ROLE> using TDof = typename ModeTypes<MODE, ROLE>::TD;

template <int MODE, int M, int ROLE>
__device__ __forceinline__ void x_phase(const PassArgs& a, const Scal& S, long long units, unsigned char* sm,
                                        Acc* acc) {
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  for (long long u = blockIdx.x; u < units; u += gridDim.x)
    xunit<TFof<MODE, ROLE>, TSof<MODE, ROLE>, TDof<MODE, ROLE>, M, ROLE>(a, S, u, sm, acc);
}

template <int MODE, int M, int ROLE>
__device__ __forceinline__ void s_phase(const PassArgs& a, const Scal& S, long long units, unsigned char* sm,
                                        Acc* acc) {
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  for (long long u = blockIdx.x; u < units; u += gridDim.x) sunit<TFof<MODE, ROLE>, M, ROLE>(a, S, u, sm, acc);
}

template <int MODE, int M, int DIM>
__global__ void __launch_bounds__(256) persist_solve(PersistArgs P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ Ctl S;
  __shared__ double tot[kMaxMoments];
  if (threadIdx.x == 0) S = *P.ctl;
  __syncthreads();
  const bool writer = blockIdx.x == 0;
  const Fin F = fin_of(P.hx);
  const long long U = P.units;
  int parity = 0;
  bool ok = true;
  Acc acc[kMaxMoments];

  while (!S.done) {
    // ---- H phi_n (x pass folds in the retraction to phi_n) ----
    Scal sc = scal_of(&S, P.hx);
    x_phase<MODE, M, P_HX>(P.hx, sc, U, smraw, acc);
    if (!(ok = all_reduce<6, 32u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0)
      for (int k = 0; k < 6; ++k) S.hsum[0][k] = tot[k];
    s_phase<MODE, M, P_HMID>(P.hy, sc, U, smraw, acc);
    if (!(ok = all_reduce<2, 0u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0) {
      S.hsum[1][0] = tot[0];
      S.hsum[1][1] = tot[1];
      if (DIM == 2) finalize_H(&S, F, writer);
    }
    if constexpr (DIM == 3) {
      s_phase<MODE, M, P_HMID>(P.hz, sc, U, smraw, acc);
      if (!(ok = all_reduce<2, 0u>(P, acc, parity, tot))) break;
      if (threadIdx.x == 0) {
        S.hsum[2][0] = tot[0];
        S.hsum[2][1] = tot[1];
        finalize_H(&S, F, writer);
      }
    }
    __syncthreads();
    // ---- residual, stopping rule, P_C r_n ----
    sc = scal_of(&S, P.c1);
    x_phase<MODE, M, P_C1>(P.c1, sc, U, smraw, acc);
    if (!(ok = all_reduce<3, 1u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0) {
      const double t3[3] = {tot[0], tot[1], tot[2]};
      finalize_C1(&S, F, t3, writer);
    }
    __syncthreads();
    if (S.done) break;
    if constexpr (DIM == 3) {
      s_phase<MODE, M, P_CFWD>(P.cfwd, sc, U, smraw, acc);
      if (!(ok = grid_sync(P))) break;
    }
    s_phase<MODE, M, P_CCORE>(P.ccore, sc, U, smraw, acc);
    if (!(ok = grid_sync(P))) break;
    if constexpr (DIM == 3) {
      s_phase<MODE, M, P_CINV>(P.cinv, sc, U, smraw, acc);
      if (!(ok = grid_sync(P))) break;
    }
    x_phase<MODE, M, P_C3>(P.c3, sc, U, smraw, acc);
    if (!(ok = all_reduce<6, 0u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0) {
      const double t6[6] = {tot[0], tot[1], tot[2], tot[3], tot[4], tot[5]};
      finalize_C3(&S, F, t6, writer);
    }
    __syncthreads();
    // ---- p_n and the step size ----
    sc = scal_of(&S, P.ax);
    x_phase<MODE, M, P_AX>(P.ax, sc, U, smraw, acc);
    if (!(ok = all_reduce<9, 0u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0)
      for (int k = 0; k < 9; ++k) S.asum[0][k] = tot[k];
    s_phase<MODE, M, P_AMID>(P.ay, sc, U, smraw, acc);
    if (!(ok = all_reduce<1, 0u>(P, acc, parity, tot))) break;
    if (threadIdx.x == 0) {
      S.asum[1][1] = tot[0];
      if (DIM == 2) finalize_A(&S, F, writer);
    }
    if constexpr (DIM == 3) {
      s_phase<MODE, M, P_AMID>(P.az, sc, U, smraw, acc);
      if (!(ok = all_reduce<1, 0u>(P, acc, parity, tot))) break;
      if (threadIdx.x == 0) {
        S.asum[2][1] = tot[0];
        finalize_A(&S, F, writer);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!ok) {
      S.status = 6;  // GPE_ERR_TIMEOUT
      S.done = 1;
    }
    if (writer) *P.ctl = S;
  }
}

// Host launcher for one mode (gpe_p_m<mode>.cu).  Returns
// cudaErrorInvalidValue when (M, dim) has no persistent kernel.
cudaError_t launch_persist_m0(int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                              cudaStream_t st, int* max_blocks_per_sm);
cudaError_t launch_persist_m1(int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                              cudaStream_t st, int* max_blocks_per_sm);
cudaError_t launch_persist_m2(int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                              cudaStream_t st, int* max_blocks_per_sm);

// Occupancy query (grid == 0) or cooperative launch of persist_solve<MODE, M, DIM>.
template <int MODE, int M, int DIM>
cudaError_t launch_persist_one(const PersistArgs& P, int grid, int block, size_t smem, cudaStream_t st,
                               int* max_blocks_per_sm) {
  auto kern = persist_solve<MODE, M, DIM>;
  if (max_blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, kern, block, smem);
    if (e != cudaSuccess || grid == 0) return e;
  }
  PersistArgs copy = P;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(block), args, smem, st);
}

template <int MODE>
cudaError_t launch_persist_mode(int M, int dim, const PersistArgs& P, int grid, int block, size_t smem,
                                cudaStream_t st, int* mb) {
  if (dim == 2) {
    switch (M) {
      case 64: return launch_persist_one<MODE, 64, 2>(P, grid, block, smem, st, mb);
      case 128: return launch_persist_one<MODE, 128, 2>(P, grid, block, smem, st, mb);
      case 256: return launch_persist_one<MODE, 256, 2>(P, grid, block, smem, st, mb);
      case 512: return launch_persist_one<MODE, 512, 2>(P, grid, block, smem, st, mb);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (M) {
    case 64: return launch_persist_one<MODE, 64, 3>(P, grid, block, smem, st, mb);
    case 128: return launch_persist_one<MODE, 128, 3>(P, grid, block, smem, st, mb);
    case 256: return launch_persist_one<MODE, 256, 3>(P, grid, block, smem, st, mb);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpe
