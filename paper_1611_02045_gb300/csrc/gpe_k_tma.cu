// gpe_k_tma.cu -- the passes of H_phi f (Section 2 operator, eq. FFTdiscret of
// Section 3) in complex64 fed by the Tensor Memory Accelerator:
//  * y / z passes (roles P_HMID: t += IFFT_axis[ (1/2 k^2 - omega x k) FFT_axis f ];
//    P_CFWD, P_CCORE, P_CINV: the Fourier core of P_C; P_AMID: the A p moments),
//    the arithmetic of pass_s<float, M, ROLE>, column tiles through 3D
//    tensor-map boxes;
//  * x (role P_HX): t = IFFT_x[ (1/2 xi^2 + omega y xi) FFT_x f ] + (V + eta|phi|^2) f
//    with the solver's retraction folded in, the arithmetic of
//    pass_x<float, float, float, M, P_HX>, rows through 1D bulk copies.
//
// A strided pass touches a tile of tx adjacent x-columns along the whole
// transformed axis (rows of tx * 8 bytes, a field row apart).  Here each block
// is persistent: it walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...,
// and while it transforms one tile, the TMA unit copies the next tile's f and
// t columns (3D tensor-map boxes, at most 256 rows per box) into the other of
// two shared-memory stages, completing on that stage's mbarrier.  The loads
// therefore overlap the transforms, which the one-tile-per-block kernel
// cannot do.  Every mbarrier wait is bounded: a wait that gives up marks the
// solve (or API call) GPE_ERR_TIMEOUT in the control block, waits (bounded)
// for the block's copy still in flight, and the block joins the reduction
// with what it has, so that no kernel hangs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gpe_passes.cuh"
#include "gpe_tma.cuh"

namespace gpe {

namespace {

// Input tiles per unit of a strided role: f and t (H), s (the P_C passes), p (A p moments).
template <int ROLE> struct STiles { static constexpr int value = ROLE == P_HMID ? 2 : 1; };

template <int M, int EV, int ROLE>
__global__ void __launch_bounds__(512) pass_s_tma(PassArgs a, const __grid_constant__ CUtensorMap tm0,
                                                   const __grid_constant__ CUtensorMap tm1) {
  using T = float;
  using C = float2;
  constexpr int E = LineCfg<M, EV>::E, Tl = LineCfg<M, EV>::Tl;
  constexpr int BOX = M < 256 ? M : 256;  // rows per tensor-map box
  constexpr int NBOX = M / BOX;
  constexpr int NT = STiles<ROLE>::value;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  if (a.solver && a.ctl->done) {
    if (ROLE == P_AMID && a.last_axis && blockIdx.x == 0 && threadIdx.x == 0) set_loop_condition(a, 0);
    return;
  }
  const Scal S = scal_of(a.ctl, a);
  const int tx = a.tx;
  const int tile = M * tx;  // elements of one column tile
  C* stage = reinterpret_cast<C*>(smraw);  // [2 stages][NT tiles]
  C* ex = stage + 2 * NT * tile;           // transform exchange [M][tx]
  const int c = threadIdx.x % tx, t = threadIdx.x / tx;
  const long long units = a.nblocks;
  const unsigned bytes = (unsigned)NT * (unsigned)tile * (unsigned)sizeof(C);

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // input columns of tile u into stage s (one thread)
  auto issue = [&](long long u, int s) {
    const int xt = (int)(u % a.ntx);
    const int outer = (int)(u / a.ntx);
    C* d0 = stage + (NT * s) * tile;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stage's earlier generic reads
    mbar_expect_tx(&bar[s], bytes);
#pragma unroll
    for (int b = 0; b < NBOX; ++b) {
      const int x0 = xt * tx;
      const int y0 = a.axis == 1 ? b * BOX : outer;
      const int z0 = a.axis == 1 ? outer : b * BOX;
      tma_load_3d(d0 + b * BOX * tx, &tm0, x0, y0, z0, &bar[s]);
      if constexpr (NT == 2) tma_load_3d(d0 + tile + b * BOX * tx, &tm1, x0, y0, z0, &bar[s]);
    }
  };

  Acc acc[kMaxMoments];
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const T* __restrict__ xia = tab<T>(a.xi[a.axis]);
  const T invM = T(1) / T(M);
  const T om = T(a.omega);
  auto si = [tx, c](int pos) { return pos * tx + c; };

  if (threadIdx.x == 0 && (long long)blockIdx.x < units) issue(blockIdx.x, 0);
  int i = 0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x, ++i) {
    const int s = i & 1;
    const bool next = u + gridDim.x < units;
    if (threadIdx.x == 0 && next) issue(u + gridDim.x, s ^ 1);
    const bool ok = mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      // give up: report, wait (bounded) for this block's copies still in flight, and
      // join the reduction with what the block has
      if (threadIdx.x == 0) {
        atomicExch(&a.ctl->status, 6);  // GPE_ERR_TIMEOUT
        atomicExch(&a.ctl->done, 1);
        mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
        if (next) mbar_wait(&bar[s ^ 1], (unsigned)(((i + 1) >> 1) & 1));
      }
      __syncthreads();
      break;
    }
    const C* in0 = stage + (NT * s) * tile;
    const int xt = (int)(u % a.ntx);
    const long long outer = u / a.ntx;
    const int ix = xt * tx + c;
    const long long base = outer * a.outer_stride + ix;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = in0[(t + q * Tl) * tx + c];
    if constexpr (ROLE == P_HMID) {
      // t += (1/2 mu^2 - omega x mu) f (y) or 1/2 zeta^2 f (z), the operand tile, then t
      C tv[E];
#pragma unroll
      for (int q = 0; q < E; ++q) tv[q] = in0[tile + (t + q * Tl) * tx + c];
      line_dft<M, E, -1>(v, ex, si, t, tw);
      const T x = (a.axis == 1) ? tab<T>(a.xc[0])[ix] : T(0);
      const T rx = (a.axis == 1) ? -x : T(0);  // rotation symbol -omega x mu (y); none for z
      T akin = 0, arot = 0;
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const T k = xia[t + q * Tl];
        const T mk = T(0.5) * k * k, kr = rx * k;
        const T a2 = v[q].x * v[q].x + v[q].y * v[q].y;
        akin += mk * a2;
        arot += kr * a2;
        v[q] = cscale(v[q], (mk + om * kr) * invM);
      }
      line_dft<M, E, +1>(v, ex, si, t, tw);
      C* __restrict__ dst = static_cast<C*>(a.out ? a.out : a.t);  // API: the final pass writes the caller's buffer
#pragma unroll
      for (int q = 0; q < E; ++q) dst[base + (t + q * Tl) * a.stride] = cadd(tv[q], v[q]);
      acc[0] = acc_add(acc[0], acc_from(akin * invM));
      acc[1] = acc_add(acc[1], acc_from(arot * invM));
    } else if constexpr (ROLE == P_CFWD || ROLE == P_CINV || ROLE == P_CCORE) {
      if constexpr (ROLE == P_CINV) {
        line_dft<M, E, +1>(v, ex, si, t, tw);
      } else {
        line_dft<M, E, -1>(v, ex, si, t, tw);
      }
      if constexpr (ROLE == P_CCORE) {
        // (alpha + |k|^2 / 2)^{-1} / N on the full frequency grid (eq. PDelta)
        const T alpha = T(S.alpha);
        const T invN = T(1.0 / ((double)a.nx * a.ny * (a.dim == 3 ? a.nz : 1)));
        const T kx = tab<T>(a.xi[0])[ix];
        T kother = 0;
        if (a.dim == 3) {
          const T ky = tab<T>(a.xi[1])[outer];  // axis 2 (z): the y index is the outer index
          kother = ky * ky;
        }
        const bool core = pc_core(S.pc);
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const T k = xia[t + q * Tl];
          const T den = alpha + T(0.5) * (kx * kx + kother + k * k);
          v[q] = cscale(v[q], core ? invN / den : invN);
        }
        line_dft<M, E, +1>(v, ex, si, t, tw);
      }
      C* __restrict__ sb = static_cast<C*>(a.s);
#pragma unroll
      for (int q = 0; q < E; ++q) sb[base + (t + q * Tl) * a.stride] = v[q];
    } else {
      static_assert(ROLE == P_AMID, "strided roles: HMID, CFWD, CCORE, CINV, AMID");
      line_dft<M, E, -1>(v, ex, si, t, tw);
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
    __syncthreads();  // stage s is read by every thread before it is refilled
  }
  reduce_and_finish<ROLE>(a, acc);
}

// x pass of H phi: blocks of lpb whole lines (rows), persistent over the units
// blockIdx.x, blockIdx.x + gridDim.x, ...; stage s holds the unit's phi rows,
// its second operand (f in an API call with f != phi, p in a solve with the
// retraction) and its V rows, copied in by one thread while the previous unit
// is transformed.
template <int M, int EV>
__global__ void __launch_bounds__(512) pass_hx_bulk(PassArgs a, int second) {
  using T = float;
  using C = float2;
  constexpr int E = LineCfg<M, EV>::E, Tl = LineCfg<M, EV>::Tl;
  constexpr int LS = M + M / 16;
  constexpr bool W = Tl <= 32;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  if (a.solver && a.ctl->done) return;
  const Scal S = scal_of(a.ctl, a);
  const int lpb = a.lpb;
  const int rows = lpb * M;  // elements of one unit
  const size_t cbytes = (size_t)rows * sizeof(C), vbytes = (size_t)rows * sizeof(T);
  const size_t sbytes = 2 * cbytes + vbytes;  // one stage
  unsigned char* stage0 = smraw;
  C* sm = reinterpret_cast<C*>(smraw + 2 * sbytes);  // transform exchange [lpb][LS]
  const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
  const long long units = a.nblocks;
  const C* __restrict__ phi = static_cast<const C*>(a.phi);
  const C* __restrict__ sec = static_cast<const C*>(second == 1 ? a.f : a.p);  // 0: no second operand
  const T* __restrict__ V = tab<T>(a.V);
  const unsigned bytes = (unsigned)((second ? 2 : 1) * cbytes + vbytes);

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](long long u, int s) {
    unsigned char* d = stage0 + s * sbytes;
    const long long e0 = u * rows;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], bytes);
    bulk_load(d, phi + e0, (unsigned)cbytes, &bar[s]);
    if (second) bulk_load(d + cbytes, sec + e0, (unsigned)cbytes, &bar[s]);
    bulk_load(d + 2 * cbytes, V + e0, (unsigned)vbytes, &bar[s]);
  };

  Acc acc[kMaxMoments];
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  const C* __restrict__ tw = static_cast<const C*>(a.tw);
  const T* __restrict__ xi = tab<T>(a.xi[0]);
  const T invM = T(1) / T(M);
  const T om = T(a.omega), eta = T(a.eta);
  auto si = [l](int pos) { return l * LS + pos + (pos >> 4); };
  const bool retract = a.solver && S.retract;
  const T cc = T(retract ? S.c * S.inv_nrm : 1.0);
  const T ss = T(retract ? S.s * S.inv_np * S.inv_nrm : 0.0);
  C* __restrict__ phi_out = static_cast<C*>(a.phi_out);
  C* __restrict__ tout = static_cast<C*>(a.t);

  if (threadIdx.x == 0 && (long long)blockIdx.x < units) issue(blockIdx.x, 0);
  int i = 0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x, ++i) {
    const int s = i & 1;
    const bool next = u + gridDim.x < units;
    if (threadIdx.x == 0 && next) issue(u + gridDim.x, s ^ 1);
    const bool ok = mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(&a.ctl->status, 6);  // GPE_ERR_TIMEOUT
        atomicExch(&a.ctl->done, 1);
        mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
        if (next) mbar_wait(&bar[s ^ 1], (unsigned)(((i + 1) >> 1) & 1));
      }
      __syncthreads();
      break;
    }
    const unsigned char* d = stage0 + s * sbytes;
    const C* phs = reinterpret_cast<const C*>(d) + l * M + t;
    const C* secs = reinterpret_cast<const C*>(d + cbytes) + l * M + t;
    const T* vs = reinterpret_cast<const T*>(d + 2 * cbytes) + l * M + t;
    const long long line = u * lpb + l;
    const long long base = line * M + t;
    const int iy = (int)((a.row0 + line) % a.ny);
    C ph[E], v[E];
    T vv[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      C x = phs[q * Tl];
      if (retract) {
        const C pq = secs[q * Tl];
        x = make_float2(cc * x.x + ss * pq.x, cc * x.y + ss * pq.y);
        phi_out[base + q * Tl] = x;
      }
      ph[q] = x;
      vv[q] = vs[q * Tl];
      v[q] = (second == 1) ? secs[q * Tl] : x;
    }
    line_dft<M, E, -1, W>(v, sm, si, t, tw);
    const T y = tab<T>(a.xc[1])[iy];
    T akin = 0, arot = 0;  // arot: the rotation symbol without omega (omega is applied in finalize_H)
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T k = xi[t + q * Tl];
      const T mk = T(0.5) * k * k, kr = y * k;
      const T a2 = v[q].x * v[q].x + v[q].y * v[q].y;
      akin += mk * a2;
      arot += kr * a2;
      v[q] = cscale(v[q], (mk + om * kr) * invM);
    }
    line_dft<M, E, +1, W>(v, sm, si, t, tw);
    T apot = 0, au2 = 0, an2 = 0, umax = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const T uu = ph[q].x * ph[q].x + ph[q].y * ph[q].y;
      const T m = vv[q] + eta * uu;
      const C fq = (second == 1) ? secs[q * Tl] : ph[q];  // the operand f (API call with f != phi)
      tout[base + q * Tl] = make_float2(v[q].x + m * fq.x, v[q].y + m * fq.y);
      apot += vv[q] * uu;
      au2 += uu * uu;
      an2 += uu;
      umax = fmaxf(umax, uu);
    }
    acc[0] = acc_add(acc[0], acc_from(akin * invM));
    acc[1] = acc_add(acc[1], acc_from(arot * invM));
    acc[2] = acc_add(acc[2], acc_from(apot));
    acc[3] = acc_add(acc[3], acc_from(au2));
    acc[4] = acc_add(acc[4], acc_from(an2));
    acc[5] = acc_max(acc[5], acc_from(umax));
    __syncthreads();  // stage s is read by every thread before it is refilled
  }
  reduce_and_finish<P_HX>(a, acc);
}

// Input fields of a bulk-staged x pass of P_C or A p (solver, complex64), in
// their order in a stage; V follows them.  The outputs are written by the
// unit body into stage regions and stored back by bulk copies:
//   C1: reads phi, t (H phi); writes s_hat over the t region -> s
//   C3: reads s_hat, phi, t, r_{n-1}, p; writes P r over s_hat -> s and r_n over r_{n-1} -> r_prev
//   AX: reads phi, s (P r), t, p; writes p_n over p -> p
template <int ROLE> struct XcFields;
template <> struct XcFields<P_C1> { static constexpr int n = 2; };
template <> struct XcFields<P_C3> { static constexpr int n = 5; };
template <> struct XcFields<P_AX> { static constexpr int n = 4; };

// Global field k of role ROLE (input order above).
template <int ROLE>
__device__ __forceinline__ void* xc_field(const PassArgs& a, int k) {
  if constexpr (ROLE == P_C1) return k == 0 ? const_cast<void*>(a.phi) : a.t;
  else if constexpr (ROLE == P_C3) {
    void* f[5] = {a.s, const_cast<void*>(a.phi), a.t, a.r_prev, a.p};
    return f[k];
  } else {
    void* f[4] = {const_cast<void*>(a.phi), a.s, a.t, a.p};
    return f[k];
  }
}

// The x passes C1, C3 and AX of a complex64 solve through the bulk-copy
// pipeline: persistent blocks walk units of lpb rows with two shared-memory
// stages (the next unit's input rows land by 1D bulk copies while the current
// one runs the unit body of the global-memory pass, pointed at the stage);
// written fields go back by bulk copies.  Same arithmetic and reductions as
// pass_x<float, float, float, M, ROLE, EV>.
template <int M, int EV, int ROLE>
__global__ void __launch_bounds__(512) pass_xc_bulk(PassArgs a) {
  using C = float2;
  constexpr int NF = XcFields<ROLE>::n;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ PassArgs sa[2];  // the unit body's arguments, pointed at stage s
  if (a.solver && a.ctl->done) return;
  const Scal S = scal_of(a.ctl, a);
  const int lpb = a.lpb;
  const int rows = lpb * M;
  const size_t cb = (size_t)rows * sizeof(C), vb = (size_t)rows * sizeof(float);
  const size_t sbytes = NF * cb + vb;
  unsigned char* stage0 = smraw;
  unsigned char* ex = smraw + 2 * sbytes;  // transform exchange [lpb][M + M/16]
  const long long units = a.nblocks;
  const unsigned bytes = (unsigned)sbytes;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < 2; ++s) {
      PassArgs b = a;
      unsigned char* d = stage0 + s * sbytes;
      C* reg[NF];
      for (int k = 0; k < NF; ++k) reg[k] = reinterpret_cast<C*>(d + k * cb);
      b.V = d + NF * cb;
      if constexpr (ROLE == P_C1) { b.phi = reg[0]; b.t = reg[1]; b.s = reg[1]; }
      else if constexpr (ROLE == P_C3) { b.s = reg[0]; b.phi = reg[1]; b.t = reg[2]; b.r_prev = reg[3]; b.p = reg[4]; }
      else { b.phi = reg[0]; b.s = reg[1]; b.t = reg[2]; b.p = reg[3]; }
      sa[s] = b;
    }
  }
  __syncthreads();
  // one thread: input rows of unit u into stage s
  auto issue = [&](long long u, int s) {
    unsigned char* d = stage0 + s * sbytes;
    const long long e0 = u * rows;
    sa[s].row0 = a.row0 + (int)(u * lpb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], bytes);
    for (int k = 0; k < NF; ++k)
      bulk_load(d + k * cb, static_cast<const C*>(xc_field<ROLE>(a, k)) + e0, (unsigned)cb, &bar[s]);
    bulk_load(d + NF * cb, static_cast<const float*>(a.V) + e0, (unsigned)vb, &bar[s]);
  };
  // one thread: written regions of unit u in stage s back to global memory
  auto store = [&](long long u, int s) {
    unsigned char* d = stage0 + s * sbytes;
    const long long e0 = u * rows;
    auto put = [&](void* dst, int k) {
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                   ::"l"(static_cast<C*>(dst) + e0), "r"(smem_u32(d + k * cb)), "r"((unsigned)cb) : "memory");
    };
    if constexpr (ROLE == P_C1) put(a.s, 1);
    else if constexpr (ROLE == P_C3) { put(a.s, 0); put(a.r_prev, 3); }
    else put(a.p, 3);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  };

  Acc acc[kMaxMoments];
#pragma unroll
  for (int k = 0; k < kMaxMoments; ++k) acc[k] = Acc{0.0f, 0.0f};
  if (threadIdx.x == 0 && (long long)blockIdx.x < units) issue(blockIdx.x, 0);
  int i = 0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x, ++i) {
    const int s = i & 1;
    const bool next = u + gridDim.x < units;
    if (threadIdx.x == 0 && next) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // stage s^1 stored back (unit i-1)
      issue(u + gridDim.x, s ^ 1);
    }
    const bool ok = mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(&a.ctl->status, 6);  // GPE_ERR_TIMEOUT
        atomicExch(&a.ctl->done, 1);
        mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
        if (next) mbar_wait(&bar[s ^ 1], (unsigned)(((i + 1) >> 1) & 1));
      }
      __syncthreads();
      break;
    }
    xunit<float, float, float, M, ROLE, EV>(sa[s], S, 0, ex, acc);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // stage writes before the bulk stores
    __syncthreads();
    if (threadIdx.x == 0) store(u, s);
  }
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  reduce_and_finish<ROLE>(a, acc);
}
// Tensor map over a complex64 field [nz][ny][nx] (8-byte elements), boxes of
// tx x-columns along the pass axis (BOX rows).
bool encode_field(CUtensorMap* m, const void* base, const PassArgs& a, int box) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)a.nx * 8, (cuuint64_t)a.nx * a.ny * 8};
  const cuuint32_t boxd[3] = {(cuuint32_t)a.tx, (cuuint32_t)(a.axis == 1 ? box : 1), (cuuint32_t)(a.axis == 1 ? 1 : box)};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, boxd, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int M, int EV, int ROLE>
cudaError_t launch_tma_one(const PassArgs& a0, cudaStream_t st, bool* used) {
  constexpr int Tl = LineCfg<M, EV>::Tl;
  constexpr int NT = STiles<ROLE>::value;
  PassArgs a = a0;
  // tiles of at least 8 columns (64-byte row segments per box row) where the grid and
  // the thread cap allow: narrower plans (tuned for the one-tile-per-block kernel)
  // are widened; the tile count follows
  if (a.tx < 8 && a.nx % 8 == 0 && Tl * 8 <= 512) {
    const long long outer = a.nblocks / a.ntx;
    a.tx = 8;
    a.ntx = a.nx / 8;
    a.nblocks = (int)(a.ntx * outer);
  }
  const int threads = Tl * a.tx;
  if (threads > 512 || a.tx < 2 || (a.tx & 1)) return cudaSuccess;  // 16-byte rows: tx even
  const size_t smem = (size_t)(2 * NT + 1) * M * a.tx * sizeof(float2);
  if (smem > 200 * 1024) return cudaSuccess;
  const void* src0 = ROLE == P_HMID ? ((a.f && !a.solver) ? a.f : a.phi) : (ROLE == P_AMID ? a.p : a.s);
  const void* src1 = ROLE == P_HMID ? a.t : src0;
  if ((reinterpret_cast<uintptr_t>(src0) & 15u) || (reinterpret_cast<uintptr_t>(src1) & 15u)) return cudaSuccess;
  CUtensorMap tm0, tm1;
  constexpr int BOX = M < 256 ? M : 256;
  if (!encode_field(&tm0, src0, a, BOX)) return cudaSuccess;
  if (NT == 2 && !encode_field(&tm1, src1, a, BOX)) return cudaSuccess;
  if (NT == 1) tm1 = tm0;
  auto kern = pass_s_tma<M, EV, ROLE>;
  static DeviceOnce attr;
  static std::atomic<int> occ_dev[64][8];  // blocks per SM, per device and tile width (log2 tx; 0 = unknown)
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.set(dev);
  }
  int cls = 0;
  while ((2 << cls) <= a.tx && cls < 7) ++cls;
  int occ = (dev >= 0 && dev < 64) ? occ_dev[dev][cls].load() : 0;
  if (occ <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess || occ < 1) { cudaGetLastError(); return cudaSuccess; }
    if (dev >= 0 && dev < 64) occ_dev[dev][cls].store(occ);
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaGetLastError();
  const long long grid = (long long)occ * nsm;
  // the pipeline pays when every block has at least two tiles to overlap; smaller
  // fields (L2-resident 2D grids) keep the tuned one-tile-per-block kernel
  if (a.nblocks < 2 * grid) return cudaSuccess;
  *used = true;
  kern<<<(unsigned)grid, threads, smem, st>>>(a, tm0, tm1);
  return cudaGetLastError();
}

template <int ROLE>
cudaError_t launch_s_role(const PassArgs& a, cudaStream_t st, bool* used) {
  switch (a.M) {
    case 64: return launch_tma_one<64, 8, ROLE>(a, st, used);
    case 128: return launch_tma_one<128, 8, ROLE>(a, st, used);
    case 256: return launch_tma_one<256, 8, ROLE>(a, st, used);
    case 512: return launch_tma_one<512, 8, ROLE>(a, st, used);
    default: return cudaSuccess;
  }
}

template <int M, int EV>
cudaError_t launch_hx_one(const PassArgs& a0, cudaStream_t st, bool* used) {
  constexpr int Tl = LineCfg<M, EV>::Tl;
  PassArgs a = a0;
  // 256 threads per block: lpb = 256 / Tl whole lines per unit
  const long long nlines = (long long)a.ny * a.nz;
  int lpb = 256 / Tl;
  while (lpb > 1 && nlines % lpb) lpb >>= 1;
  if (lpb < 1 || nlines / lpb < 1) return cudaSuccess;
  a.lpb = lpb;
  a.nblocks = (int)(nlines / lpb);
  const int threads = Tl * lpb;
  // second operand: f (API call with f != phi: 1) or p (solve with the retraction: 2)
  const int second = (!a.solver && a.f && a.f != a.phi) ? 1 : (a.solver ? 2 : 0);
  const size_t cb = (size_t)lpb * M * sizeof(float2), vb = (size_t)lpb * M * sizeof(float);
  const size_t smem = 2 * (2 * cb + vb) + (size_t)lpb * (M + M / 16) * sizeof(float2);
  if (smem > 200 * 1024 || (cb & 15) || (vb & 15)) return cudaSuccess;
  const void* ptrs[3] = {a.phi, second == 1 ? a.f : (second == 2 ? a.p : a.phi), a.V};
  for (const void* q : ptrs)
    if (reinterpret_cast<uintptr_t>(q) & 15u) return cudaSuccess;
  auto kern = pass_hx_bulk<M, EV>;
  static DeviceOnce attr;
  static std::atomic<int> occ_dev[64];
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.set(dev);
  }
  int occ = (dev >= 0 && dev < 64) ? occ_dev[dev].load() : 0;
  if (occ <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess || occ < 1) { cudaGetLastError(); return cudaSuccess; }
    if (dev >= 0 && dev < 64) occ_dev[dev].store(occ);
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaGetLastError();
  const long long grid = (long long)occ * nsm;
  if (a.nblocks < 2 * grid) return cudaSuccess;  // at least two units per block, as for the strided passes
  *used = true;
  kern<<<(unsigned)grid, threads, smem, st>>>(a, second);
  return cudaGetLastError();
}

template <int M, int EV, int ROLE>
cudaError_t launch_xc_one(const PassArgs& a0, cudaStream_t st, bool* used) {
  constexpr int Tl = LineCfg<M, EV>::Tl;
  constexpr int NF = XcFields<ROLE>::n;
  PassArgs a = a0;
  // up to 256 threads per block, units of lpb whole lines; fewer lines when the
  // two stages would not leave room for two blocks per SM
  const long long nlines = (long long)a.ny * a.nz;
  int lpb = 256 / Tl;
  auto smem_of = [&](int l) {
    return 2 * ((size_t)l * M * (NF * sizeof(float2) + sizeof(float))) + (size_t)l * (M + M / 16) * sizeof(float2);
  };
  while (lpb > 1 && (nlines % lpb || smem_of(lpb) > 110 * 1024)) lpb >>= 1;
  if (nlines % lpb || smem_of(lpb) > 200 * 1024) return cudaSuccess;
  a.lpb = lpb;
  a.nblocks = (int)(nlines / lpb);
  const int threads = Tl * lpb;
  const size_t cb = (size_t)lpb * M * sizeof(float2), vb = (size_t)lpb * M * sizeof(float);
  if ((cb & 15) || (vb & 15)) return cudaSuccess;
  const void* ptrs[6] = {a.phi, a.t, a.s, a.r_prev, a.p, a.V};
  for (const void* q : ptrs)
    if (reinterpret_cast<uintptr_t>(q) & 15u) return cudaSuccess;
  const size_t smem = smem_of(lpb);
  auto kern = pass_xc_bulk<M, EV, ROLE>;
  static DeviceOnce attr;
  static std::atomic<int> occ_dev[64][8];  // [device][log2 lpb]
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.set(dev);
  }
  int lg = 0;
  while ((1 << lg) < lpb && lg < 7) ++lg;
  int occ = (dev >= 0 && dev < 64) ? occ_dev[dev][lg].load() : 0;
  if (occ <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess || occ < 1) { cudaGetLastError(); return cudaSuccess; }
    if (dev >= 0 && dev < 64) occ_dev[dev][lg].store(occ);
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaGetLastError();
  const long long grid = (long long)occ * nsm;
  // at least two units per block, and no more blocks than the plan's (the reduction partials hold those)
  if (a.nblocks < 2 * grid || grid > a0.nblocks) return cudaSuccess;
  *used = true;
  kern<<<(unsigned)grid, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int ROLE>
cudaError_t launch_xc_role(const PassArgs& a, cudaStream_t st, bool* used) {
  switch (a.M) {
    case 64: return launch_xc_one<64, 8, ROLE>(a, st, used);
    case 128: return launch_xc_one<128, 8, ROLE>(a, st, used);
    case 256: return launch_xc_one<256, 8, ROLE>(a, st, used);
    case 512: return launch_xc_one<512, 8, ROLE>(a, st, used);
    default: return cudaSuccess;
  }
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}


// x pass of H phi in complex64 through the bulk-copy pipeline (M in 64 .. 512,
// 16-byte aligned phi, f or p and V, E = 8); *used = false otherwise.
cudaError_t launch_hx_bulk(const PassArgs& a, cudaStream_t st, bool* used) {
  *used = false;
  if (a.E != 0 && a.E != 8) return cudaSuccess;
  if (a.row0 != 0) return cudaSuccess;
  switch (a.M) {
    case 64: return launch_hx_one<64, 8>(a, st, used);
    case 128: return launch_hx_one<128, 8>(a, st, used);
    case 256: return launch_hx_one<256, 8>(a, st, used);
    case 512: return launch_hx_one<512, 8>(a, st, used);
    default: return cudaSuccess;
  }
}

// A strided pass (y or z) in complex64 through the TMA pipeline when the plan
// and the fields allow it (E = 8, even tile width, 16-byte aligned inputs,
// M in {64, 128, 256, 512}); roles P_HMID, P_CFWD, P_CCORE, P_CINV, P_AMID;
// *used = false otherwise (the caller launches pass_s).
cudaError_t launch_strided_tma(Pass pass, const PassArgs& a, cudaStream_t st, bool* used) {
  *used = false;
  if (a.E != 0 && a.E != 8) return cudaSuccess;
  switch (pass) {
    case P_HMID: return launch_s_role<P_HMID>(a, st, used);
    case P_CFWD: return launch_s_role<P_CFWD>(a, st, used);
    case P_CCORE: return launch_s_role<P_CCORE>(a, st, used);
    case P_CINV: return launch_s_role<P_CINV>(a, st, used);
    case P_AMID: return launch_s_role<P_AMID>(a, st, used);
    default: return cudaSuccess;
  }
}

// The x passes C1, C3 and AX of a complex64 solve through the bulk-copy
// pipeline when the plan and the fields allow it (solver mode, E = 8,
// M in {64, 128, 256, 512}, 16-byte aligned fields, at least two units per
// block); *used = false otherwise (the caller launches pass_x).
cudaError_t launch_xc_bulk(Pass pass, const PassArgs& a, cudaStream_t st, bool* used) {
  *used = false;
  if ((a.E != 0 && a.E != 8) || !a.solver || a.row0 != 0) return cudaSuccess;
  switch (pass) {
    case P_C1: return launch_xc_role<P_C1>(a, st, used);
    case P_C3: return launch_xc_role<P_C3>(a, st, used);
    case P_AX: return launch_xc_role<P_AX>(a, st, used);
    default: return cudaSuccess;
  }
}

}  // namespace gpe
