// gpe_peaks.cu -- arithmetic-pipe rates of this GPU, for the rooflines of the
// kernels that are not bound by memory: the FP64 passes (GPE_FP64 mode) run on
// the FP64 pipe, the double-single and single-precision transforms on the FP32
// pipe.  Each thread runs independent chains of fused multiply-adds in
// registers (no memory traffic inside the loop), so the measured rate is the
// pipe's sustainable issue rate at the clocks of the moment.
#include <cuda_runtime.h>

#include <cstring>

#include "gpe.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (covers the pipe latency)

// a <- a * b + c with b slightly below 1 and c small: the values stay bounded
// and normal for any iteration count.
template <int KIND>
__global__ void __launch_bounds__(256) fma_rate_kernel(double* sink, long long iters, float seed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (KIND == 0) {
    double a[kChains];
    const double b = 0.999999 + 1e-9 * seed, c = 1e-7 * (1.0 + seed);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k + tid * 1e-6;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[tid] = s;
  } else if constexpr (KIND == 1) {
    float a[kChains];
    const float b = 0.9999f + 1e-6f * seed, c = 1e-5f * (1.0f + seed);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k + tid * 1e-6f;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    sink[tid] = s;
  } else {
    // packed two-wide FP32: fma.rn.f32x2 on 64-bit register pairs
    unsigned long long a[kChains], b, c;
    const float bb = 0.9999f + 1e-6f * seed, cc = 1e-5f * (1.0f + seed);
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(bb), "f"(bb));
    asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(cc), "f"(cc));
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const float x = seed + k + tid * 1e-6f, y = x + 0.5f;
      asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x), "f"(y));
    }
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(b), "l"(c));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float x, y;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
      s += x + y;
    }
    sink[tid] = s;
  }
}

template <int KIND>
cudaError_t launch_rate(int grid, double* sink, long long iters, cudaStream_t st) {
  fma_rate_kernel<KIND><<<grid, 256, 0, st>>>(sink, iters, 0.25f);
  return cudaGetLastError();
}

}  // namespace

extern "C" gpe_status gpe_alu_peak(int kind, void* stream, double* gflops) {
  if (!gflops || kind < 0 || kind > 2) return GPE_ERR_ARG;
  *gflops = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GPE_ERR_CUDA;
  const int grid = 8 * nsm;  // 8 blocks of 8 warps per SM: 64 warps, the SM's limit
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 256 * (size_t)grid) != cudaSuccess) return GPE_ERR_CUDA;
  // iterations for roughly 50 ms at the nominal rates (FP64 ~1.2 TFLOP/s, FP32 ~75 TFLOP/s)
  const long long iters = (kind == 0) ? 15000 : 500000;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gpe_status s = GPE_OK;
  float best = 0.0f;
  auto launch = [&]() {
    return kind == 0 ? launch_rate<0>(grid, sink, iters, st)
                     : kind == 1 ? launch_rate<1>(grid, sink, iters, st) : launch_rate<2>(grid, sink, iters, st);
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = GPE_ERR_CUDA;
  if (s == GPE_OK && launch() != cudaSuccess) s = GPE_ERR_CUDA;  // warm-up (clocks, module load)
  for (int rep = 0; rep < 3 && s == GPE_OK; ++rep) {
    float ms = 0.0f;
    if (cudaEventRecord(e0, st) != cudaSuccess || launch() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      s = GPE_ERR_CUDA;
      break;
    }
    if (rep == 0 || ms < best) best = ms;
  }
  if (s == GPE_OK && best > 0.0f) {
    // flops per FMA: 2 (scalar) or 4 (two-wide)
    const double per_fma = kind == 2 ? 4.0 : 2.0;
    const double flops = per_fma * kChains * (double)iters * 256.0 * grid;
    *gflops = flops / (best * 1e-3) / 1e9;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return s;
}
