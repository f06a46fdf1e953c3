// gpe_hflow.cu -- H_phi f on a batch of 256 x 256 complex64 fields
// (arXiv:1611.02045, Section 2 operator with the discretisation of
// eq. FFTdiscret, Section 3) as a dataflow of independent work units.
//
// H_phi f = A_x f + A_y f + (V + eta|phi|^2) f with the per-axis spectral parts
//   A_x f = IFFT_x[ (1/2 xi^2 + omega y xi) FFT_x f ]   (row lines)
//   A_y f = IFFT_y[ (1/2 mu^2 - omega x mu) FFT_y f ]   (column lines).
// Each field is split into 16 x units (16 rows each) and 16 y units (16
// columns each).  An x unit stores t = A_x f + (V + eta|f|^2) f to its rows of
// out; a y unit adds A_y f into its columns of out, which is only allowed once
// the field's 16 x units have stored their rows.  Units come from one ticket
// counter in an order that puts every x unit of a field `lag` fields ahead of
// the field's y units; a y unit that finds its field incomplete waits (bounded)
// on the field's x-unit counter.  Persistent blocks (two per SM, all SMs) walk
// the tickets with two shared-memory stages: while one unit is transformed,
// the TMA copies the next unit's input into the other stage
//   x unit: 16 contiguous rows of f (32 KB) and of V (16 KB), 1D bulk copies;
//   y unit: the 256 x 16 column tile of f (32 KB), a 3D tensor-map box with
//           the 128-byte swizzle (conflict-free column access);
// and a y unit's result tile is added into out by a TMA reduce-add.  Every
// line is transformed by 16 threads of one warp (two lines per warp), with
// shared-memory exchanges inside the warp, so the only block barrier is the
// one at the end of each unit.
//
// Global traffic per point: read f (x unit) and write out once (16 bytes);
// the y unit's re-read of f and the read-modify-write of out hit L2 while the
// field is in flight (lag fields ~ 32 MB).  The same arithmetic in 16-CTA
// clusters (gpe_cluster.cuh) leaves SM slots empty: clusters of 16 pack into
// 14 x 16 = 224 of the 304 CTA slots of the GPU, and every field waits for its
// slowest CTA; here all slots are busy and no unit waits for another block
// except through the x-unit counters.
//
// Counters (ctr, owned by the context, zero between launches): ctr[0] ticket,
// ctr[1] blocks finished, ctr[2 + b] x units of field b done.  The last block
// to finish zeroes them, so no separate reset runs before the next launch.
#include <cuda_runtime.h>

#include <atomic>

#include "gpe_cluster.cuh"
#include "gpe_fft.cuh"
#include "gpe_internal.h"
#include "gpe_tma.cuh"

namespace gpe {

namespace {

constexpr int kFM = 256;                                    // grid side
constexpr size_t kFlowStage = 48 * 1024;                    // bytes per stage
constexpr size_t kFlowTws = 16 * kTw256Stride * sizeof(float4);
constexpr size_t kFlowKt = 2 * kFM * sizeof(float2);          // multiplier tables (x, y)
constexpr size_t kFlowSmem = 2 * kFlowStage + kFlowTws + kFlowKt + 32;  // + 2 mbarriers, 2 unit ids
constexpr int kFlowLag = 32;                                // fields between a field's x and y units

struct FlowArgs {
  int nbatch, lag;
  long long stride;  // elements between consecutive fields
  float eta, omega;
  const float *xi, *xiy, *xc, *yc, *V;
  const float2* tw;  // e^{-2 pi i m/256}
  const float2* f;   // operand (= phi)
  float2* out;
  int* ctr;          // [0] ticket, [1] blocks finished, [2 + b] x units done of field b
  int* status;       // set to GPE_ERR_TIMEOUT (6) when a bounded wait gives up (may be null)
};

// Ticket u -> (type 0 = x unit / 1 = y unit, field, block of 16 lines).
// Order: the x units of fields 0 .. D-1; then, for j = 0, 1, ...: the y units
// of field j followed by the x units of field D + j; then the remaining y
// units.  Every x unit of a field comes before its y units.
__host__ __device__ inline void flow_unit(long long u, int B, int D, int* type, int* fld, int* blk) {
  const long long head = 16LL * D;
  if (u < head) { *type = 0; *fld = (int)(u / 16); *blk = (int)(u % 16); return; }
  long long k = u - head;
  const long long P = (long long)B - D;
  if (k < 32 * P) {
    const long long pair = k / 32, w = k % 32;
    if (w < 16) { *type = 1; *fld = (int)pair; *blk = (int)w; }
    else { *type = 0; *fld = (int)(D + pair); *blk = (int)(w - 16); }
    return;
  }
  k -= 32 * P;
  *type = 1; *fld = (int)(P + k / 16); *blk = (int)(k % 16);
}

// A 256-point row line held by 16 threads of a warp (v[q] = position t + 16q),
// transformed in place in the line's own 256 slots: the stage-1 results of
// thread t (positions 16t .. 16t+15) go out as eight 16-byte chunks with the
// chunk index XOR (t mod 8), so the vector stores and the stage-2 loads are
// free of bank conflicts without padding.  Twiddles from the per-thread table
// of dft256_twiddles.  Same arithmetic as dft256x16.
template <int DIR>
__device__ __forceinline__ void dft256_row(float2 (&v)[16], float2* row, int t, const float4* tws) {
  dft16<DIR>(v);
  __syncwarp();
  {
    float4* d = reinterpret_cast<float4*>(row + 16 * t);
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i ^ (t & 7)] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = row[16 * q + 2 * ((t >> 1) ^ (q & 7)) + (t & 1)];
  const float4* w = tws + t * kTw256Stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 p = w[i];
    if (i > 0) v[2 * i] = ctw<DIR>(v[2 * i], make_float2(p.x, p.y));
    v[2 * i + 1] = ctw<DIR>(v[2 * i + 1], make_float2(p.z, p.w));
  }
  dft16<DIR>(v);
}

// Element (row y, column 2 wp + j) of a [256][16] complex64 tile written by the
// TMA with the 128-byte swizzle: 16-byte chunk wp of row y sits at chunk
// wp ^ (y mod 8) of that 128-byte row.  Index in float2 units.
__device__ __forceinline__ int tile_cell(int y, int wp, int j) { return y * 16 + 2 * (wp ^ (y & 7)) + j; }

// A 256-point column line of the swizzled tile (column 2 wp + j) held by 16
// threads of a warp; the exchange stores position p in row pi(p) = p ^ ((p >> 4) & 7)
// (a permutation), which keeps the stage-1 stores and stage-2 loads
// conflict-free and inside the warp's own cells of the tile.
template <int DIR>
__device__ __forceinline__ void dft256_col(float2 (&v)[16], float2* tile, int t, int wp, int j, const float4* tws) {
  dft16<DIR>(v);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = 16 * t + r;
    tile[tile_cell(p ^ ((p >> 4) & 7), wp, j)] = v[r];
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p = t + 16 * q;
    v[q] = tile[tile_cell(p ^ ((p >> 4) & 7), wp, j)];
  }
  const float4* w = tws + t * kTw256Stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 p = w[i];
    if (i > 0) v[2 * i] = ctw<DIR>(v[2 * i], make_float2(p.x, p.y));
    v[2 * i + 1] = ctw<DIR>(v[2 * i + 1], make_float2(p.z, p.w));
  }
  dft16<DIR>(v);
}

__global__ void __launch_bounds__(256, 2)
    h_batch_flow(FlowArgs a, const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmO) {
  using C = float2;
  extern __shared__ __align__(1024) unsigned char flow_sm[];
  float4* tws = reinterpret_cast<float4*>(flow_sm + 2 * kFlowStage);
  // kt[axis][p] = (k_p, k_p^2 / (2M)): the Fourier multiplier of a line is (k^2/2 + c k)/M
  // = fma(c/M, k, k^2/(2M)) with c = omega y (x lines) or -omega x (y lines); 1/M is exact
  float2* kt = reinterpret_cast<float2*>(flow_sm + 2 * kFlowStage + kFlowTws);
  unsigned char* ctl_sm = flow_sm + 2 * kFlowStage + kFlowTws + kFlowKt;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(ctl_sm);
  volatile int* uid = reinterpret_cast<volatile int*>(ctl_sm + 16);
  volatile int* last_block = reinterpret_cast<volatile int*>(ctl_sm + 24);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int t = lane & 15, j = lane >> 4;  // thread of its line, line of the warp
  const long long total = 32LL * a.nbatch;
  const float invM = 1.0f / kFM, om = a.omega, eta = a.eta;
  auto stage = [&](int s) { return reinterpret_cast<C*>(flow_sm + s * kFlowStage); };
  bool ok = (smem_u32(flow_sm) & 1023u) == 0;  // the swizzled tiles need 1024-byte alignment

  // thread 0: the ticket taken one refill ahead, and the x-unit count of the
  // next unit's field read one unit ahead (when that unit is a y unit)
  int tk_next = 0, early = 0;
  // thread 0: start the copies of the next ticket's unit into stage s
  auto grab_issue = [&](int s) {
    const long long u = tk_next;
    tk_next = atomicAdd(a.ctr, 1);
    if (u >= total || !ok) { uid[s] = -1; return; }
    uid[s] = (int)u;
    int type, fld, blk;
    flow_unit(u, a.nbatch, a.lag, &type, &fld, &blk);
    C* d = stage(s);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses of the stage
    if (type == 0) {
      mbar_expect_tx(&full[s], 48 * 1024);
      bulk_load(d, a.f + fld * a.stride + (long long)blk * 16 * kFM, 32 * 1024, &full[s]);
      bulk_load(reinterpret_cast<unsigned char*>(d) + 32 * 1024, a.V + blk * 16 * kFM, 16 * 1024, &full[s]);
    } else {
      mbar_expect_tx(&full[s], 32 * 1024);
      tma_load_3d(d, &tmF, 32 * blk, 0, fld, &full[s]);
    }
  };
  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  dft256_twiddles(tws, a.tw);
  for (int i = tid; i < 2 * kFM; i += blockDim.x) {
    const float k = (i < kFM ? a.xi : a.xiy)[i & (kFM - 1)];
    kt[i] = make_float2(k, 0.5f * k * k * invM);
  }
  __syncthreads();
  if (tid == 0) {
    tk_next = atomicAdd(a.ctr, 1);
    grab_issue(0);
    grab_issue(1);
  }
  __syncthreads();

  unsigned par = 0u;  // bit s: phase parity of stage s
  int s = 0;
  for (;;) {
    const int u = uid[s];
    if (u < 0) break;
    int type, fld, blk;
    flow_unit(u, a.nbatch, a.lag, &type, &fld, &blk);
    if (!mbar_wait(&full[s], (par >> s) & 1u)) ok = false;
    par ^= 1u << s;
    C* st = stage(s);
    if (type == 0) {
      // ---- x unit: row 16 blk + l, l = 2 wp + j ----
      const int l = 2 * wp + j;
      C* row = st + l * kFM;
      const float* Vr = reinterpret_cast<const float*>(st + 16 * kFM) + l * kFM;
      C w[16], sr[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        w[q] = row[t + 16 * q];
        const float m = Vr[t + 16 * q] + eta * (w[q].x * w[q].x + w[q].y * w[q].y);
        sr[q] = make_float2(m * w[q].x, m * w[q].y);
      }
      dft256_row<-1>(w, row, t, tws);
      const float cy = om * a.yc[16 * blk + l] * invM;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float2 k = kt[t + 16 * q];
        w[q] = cscale(w[q], fmaf(cy, k.x, k.y));
      }
      dft256_row<+1>(w, row, t, tws);
      C* orow = a.out + fld * a.stride + (long long)(16 * blk + l) * kFM + t;
#pragma unroll
      for (int q = 0; q < 16; ++q) orow[16 * q] = cadd(w[q], sr[q]);
    } else {
      // ---- y unit: column 16 blk + 2 wp + j; A_y f written back into the tile ----
      C w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) w[q] = st[tile_cell(t + 16 * q, wp, j)];
      dft256_col<-1>(w, st, t, wp, j, tws);
      const float cx = -om * a.xc[16 * blk + 2 * wp + j] * invM;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float2 k = kt[kFM + t + 16 * q];
        w[q] = cscale(w[q], fmaf(cx, k.x, k.y));
      }
      dft256_col<+1>(w, st, t, wp, j, tws);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 16; ++q) st[tile_cell(t + 16 * q, wp, j)] = w[q];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // tile stores -> the TMA's reads
    }
    __syncthreads();  // the stage is consumed (y: rewritten); this unit's stores are issued
    if (type == 0 && tid == 32) {
      // the x unit's rows are stored: count it (the fence waits in warp 1, off thread 0's path)
      __threadfence();
      atomicAdd(a.ctr + 2 + fld, 1);
    }
    if (tid == 0) {
      if (type == 1) {
        // the field's x units must have stored t before the TMA adds A_y f to it
        long long n = 0;
        if (early < 16)
          while (ld_acquire_gpu(a.ctr + 2 + fld) < 16 && n < kTmaWaitLimit) ++n;
        if (n >= kTmaWaitLimit) ok = false;
        asm volatile("fence.proxy.async;" ::: "memory");  // generic stores of out -> the TMA's adds
        tma_reduce_add_3d(&tmO, st, 32 * blk, 0, fld);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // tile read before the refill
      }
      grab_issue(s);
      early = 0;
      const int un = uid[s ^ 1];
      if (un >= 0) {
        int ty, fl, bl;
        flow_unit(un, a.nbatch, a.lag, &ty, &fl, &bl);
        if (ty == 1) early = ld_acquire_gpu(a.ctr + 2 + fl);
      }
    }
    s ^= 1;
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (!ok && a.status) atomicExch(a.status, 6);  // GPE_ERR_TIMEOUT
  // the last block to finish returns the counters to zero for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *last_block = atomicAdd(a.ctr + 1, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (*last_block) {
    __threadfence();
    for (int i = tid; i < a.nbatch; i += blockDim.x) a.ctr[2 + i] = 0;
    if (tid == 0) { a.ctr[0] = 0; a.ctr[1] = 0; }
  }
}

// FP32 view [B][256][512] of complex64 fields, boxes of 16 complex columns x 256 rows, 128-byte swizzle.
bool encode_flow_map(CUtensorMap* m, const void* base, int nbatch, long long stride) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {2 * kFM, kFM, (cuuint64_t)nbatch};
  const cuuint64_t strides[2] = {(cuuint64_t)kFM * 8, (cuuint64_t)stride * 8};
  const cuuint32_t box[3] = {32, kFM, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t h_batch_flow_counters(int nbatch) { return (size_t)nbatch + 2; }

cudaError_t launch_h_batch_flow(const ClusterHArgs& a, int* ctr, int ctr_cap, int* status, cudaStream_t st,
                                bool* used) {
  *used = false;
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (a.M != kFM || a.nbatch < 1 || a.f != a.phi || !ctr || (size_t)ctr_cap < h_batch_flow_counters(a.nbatch) ||
      !al16(a.f) || !al16(a.out) || !al16(a.V) || (a.stride & 1))
    return cudaSuccess;
  CUtensorMap tmF, tmO;
  if (!encode_flow_map(&tmF, a.f, a.nbatch, a.stride) || !encode_flow_map(&tmO, a.out, a.nbatch, a.stride)) {
    cudaGetLastError();
    return cudaSuccess;
  }
  static std::atomic<int> grid_dev[64];  // resident blocks per device; 0 = not yet queried
  const int dev = DeviceOnce::device();
  int grid = (dev >= 0 && dev < 64) ? grid_dev[dev].load() : 0;
  if (grid <= 0) {
    cudaError_t e = cudaFuncSetAttribute(h_batch_flow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFlowSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, nsm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h_batch_flow, 256, kFlowSmem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaSuccess;
    grid = per_sm * nsm;
    if (dev >= 0 && dev < 64) grid_dev[dev].store(grid);
  }
  const long long units = 32LL * a.nbatch;
  if (units < grid) grid = (int)units;
  FlowArgs fa;
  fa.nbatch = a.nbatch;
  fa.lag = a.nbatch < kFlowLag ? a.nbatch : kFlowLag;
  fa.stride = a.stride;
  fa.eta = (float)a.eta;
  fa.omega = (float)a.omega;
  fa.xi = static_cast<const float*>(a.xi);
  fa.xiy = static_cast<const float*>(a.xiy);
  fa.xc = static_cast<const float*>(a.xc);
  fa.yc = static_cast<const float*>(a.yc);
  fa.V = static_cast<const float*>(a.V);
  fa.tw = static_cast<const float2*>(a.tw);
  fa.f = static_cast<const float2*>(a.f);
  fa.out = static_cast<float2*>(a.out);
  fa.ctr = ctr;
  fa.status = status;
  h_batch_flow<<<grid, 256, kFlowSmem, st>>>(fa, tmF, tmO);
  *used = true;
  return cudaGetLastError();
}

}  // namespace gpe
