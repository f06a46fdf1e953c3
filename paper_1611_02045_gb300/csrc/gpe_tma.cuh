// gpe_tma.cuh -- Tensor Memory Accelerator and mbarrier primitives shared by
// the TMA-fed kernels (inline PTX, sm_90 and later; this build targets sm_103a).
//
//  * mbarriers in shared memory: init, arrive with an expected transaction
//    byte count, plain arrive, and a BOUNDED parity wait (a wait that gives up
//    returns false; no kernel of this library spins without a limit);
//  * copies that complete on an mbarrier: 1D bulk global -> shared
//    (cp.async.bulk) and 3D tiles through a tensor map (cp.async.bulk.tensor);
//  * a 3D tile reduce-add shared -> global through a tensor map (the TMA adds
//    each float of the tile into global memory, rounding as one FP32 add);
//  * an acquire load at GPU scope for flags written by other thread blocks.
// Tensor maps are encoded on the host through the driver's
// cuTensorMapEncodeTiled, obtained with cudaGetDriverEntryPointByVersion
// (encode_fn; nullptr when the driver does not provide it).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace gpe {

// try_wait polls before a wait gives up (each poll may suspend briefly): seconds.
constexpr long long kTmaWaitLimit = 1ll << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One arrival that also expects `bytes` of copies to complete on bar.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// true when the phase with the given parity has completed; false after the bound.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (long long n = 0; n < kTmaWaitLimit; ++n) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 3D tile load global -> shared through the tensor map, completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(smem_u32(bar))
      : "memory");
}

// Contiguous global -> shared bulk copy (16-byte aligned, size a multiple of 16),
// completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// global[tile at (c0, c1, c2)] += shared tile (FP32 elements of the tensor map),
// as one bulk async-group of the calling thread.  The writers of the shared
// tile order their stores before it with fence.proxy.async.shared::cta; the
// caller commits the group and waits (cp.async.bulk.wait_group[.read]) before
// it reuses the tile.
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];"
      ::"l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The driver's tensor-map encoder (host), nullptr when unavailable.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn();

}  // namespace gpe
