// gpe_fft.cuh -- in-register / shared-memory line DFTs for the per-axis
// spectral operators of eq. FFTdiscret (arXiv:1611.02045, Section 3).
//
// Convention (Section 3): forward F[f]_p = sum_k f_k e^{-2 pi i p k / M},
// unnormalised; the inverse carries 1/M, which callers fold into their
// Fourier-space multiplier.  Output is in natural DFT order p = 0..M-1
// (p >= M/2 stands for the negative frequency p - M).
//
// Layout of one line inside a thread block: the line's M points are shared by
// Tl = M/E threads; thread t of the line holds E values at positions
// t + q*Tl (q = 0..E-1) in registers.  The transform is a Stockham
// (self-sorting) decomposition M = R_1 R_2 ... with every radix R <= E; each
// stage works in registers (E/R butterflies per thread) and exchanges through
// shared memory between stages.  The final stage leaves each thread holding
// exactly the positions t + q*Tl again, so a pointwise Fourier multiplier and
// the inverse transform's first stage run with no extra exchange.
#pragma once
#include <cuda_runtime.h>

#include "gpe_ds.cuh"

namespace gpe {

template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<dsf> { using type = dsc; };
template <typename T> using cplx = typename cvec<T>::type;

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by -i (DIR = -1, forward) or +i (DIR = +1, inverse)
template <int DIR, typename C> __device__ __forceinline__ C cmul_i(C a) {
  return DIR < 0 ? cmk<C>(a.y, -a.x) : cmk<C>(-a.y, a.x);
}
// a * conj(w) when DIR = +1, a * w when DIR = -1 (w = e^{-2 pi i m / M} table)
template <int DIR, typename C> __device__ __forceinline__ C ctw(C a, C w) {
  return DIR < 0 ? cmk<C>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x)
                 : cmk<C>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

// Packed two-wide single precision (add / sub / mul .rn.f32x2, GB300): one
// instruction per complex add, subtract or real scaling of a float2, each
// lane rounded as the scalar .rn operation.  These overloads take precedence
// over the generic templates above for complex64 values.
__device__ __forceinline__ unsigned long long f2_pack(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a.x, a.y)), "l"(f2_pack(b.x, b.y)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a.x, a.y)), "l"(f2_pack(b.x, b.y)));
  return f2_unpack(d);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a.x, a.y)), "l"(f2_pack(s, s)));
  return f2_unpack(d);
}

// Twiddle loads through the read-only path where the type allows it.
__device__ __forceinline__ float2 ld_tw(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_tw(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dsc ld_tw(const dsc* p) { return *p; }

// ---------------------------------------------------------------------------
// Small DFTs on registers: y_m = sum_r x_r e^{DIR 2 pi i r m / R}
// (DIR = -1 forward, +1 inverse); computed in place.
// ---------------------------------------------------------------------------
template <int DIR, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C s = cadd(a, b), d = csub(a, b); a = s; b = d;
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = cmul_i<DIR>(csub(x1, x3));
  x0 = cadd(a, c); x2 = csub(a, c); x1 = cadd(b, d); x3 = csub(b, d);
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C (&x)[8]) {
  using R = decltype(C::x);
  const R h = R(0.70710678118654752440);  // cos(pi/4)
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  // twiddles e^{DIR 2 pi i m / 8}, m = 1, 2, 3
  C t1 = DIR < 0 ? cmk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x)) : cmk<C>(h * (o1.x - o1.y), h * (o1.y + o1.x));
  C t2 = cmul_i<DIR>(o2);
  C t3 = DIR < 0 ? cmk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y)) : cmk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y));
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, t1); x[5] = csub(e1, t1);
  x[2] = cadd(e2, t2); x[6] = csub(e2, t2);
  x[3] = cadd(e3, t3); x[7] = csub(e3, t3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft16(C (&x)[16]) {
  using R = decltype(C::x);
  C e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
  dft8<DIR>(e);
  dft8<DIR>(o);
  // w_m = e^{DIR 2 pi i m / 16} = cos(2 pi m/16) + DIR i sin(2 pi m/16)
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), h = R(0.70710678118654752440);
  const R cs[8] = {R(1), c1, h, s1, R(0), -s1, -h, -c1};
  const R sn[8] = {R(0), s1, h, c1, R(1), c1, h, s1};
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    C t;
    if (m == 0) t = o[0];
    else if (m == 4) t = cmul_i<DIR>(o[4]);
    else t = cmk<C>(o[m].x * cs[m] - R(DIR) * o[m].y * sn[m], o[m].y * cs[m] + R(DIR) * o[m].x * sn[m]);
    x[m] = cadd(e[m], t);
    x[m + 8] = csub(e[m], t);
  }
}

template <int R, int DIR, typename C> __device__ __forceinline__ void dft_small(C (&x)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<DIR>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<DIR>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8<DIR>(x);
  } else {
    static_assert(R == 16, "radix must be 1, 2, 4, 8 or 16");
    dft16<DIR>(x);
  }
}

// Lanes of the calling warp that exist in this (1D) block.
__device__ __forceinline__ unsigned block_warp_mask() {
  const unsigned n = blockDim.x - (threadIdx.x & ~31u);
  return n >= 32u ? 0xffffffffu : ((1u << n) - 1u);
}

// Barrier between exchange stages.  WARP: every line's threads lie inside one
// warp and its shared-memory slots belong to that line alone, so the warp's
// own barrier (which also orders its shared-memory accesses) is enough.
template <bool WARP> __device__ __forceinline__ void line_sync() {
  if constexpr (WARP) __syncwarp(block_warp_mask());
  else __syncthreads();
}

// ---------------------------------------------------------------------------
// Stockham stages.  SI: functor mapping a line position to a shared-memory
// element index for this thread's line slot.
// ---------------------------------------------------------------------------
// LEAD = false: the caller guarantees that no thread still reads sm (a block or
// cluster barrier since its last use), so the first exchange needs no barrier
// before its stores.
template <int M, int E, int NS, int DIR, bool WARP, bool LEAD = true, typename C, typename SI>
__device__ __forceinline__ void fft_stages(C (&v)[E], C* sm, const SI& si, int t, const C* __restrict__ tw) {
  constexpr int Tl = M / E;
  constexpr int R = (M / NS >= E) ? E : (M / NS);
  constexpr int NB = E / R;  // butterflies per thread in this stage
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = t + b * Tl;  // butterfly index, 0 .. M/R - 1
    C x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[b + r * NB];
    if constexpr (NS > 1) {
      const int k = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = ctw<DIR>(x[r], ld_tw(&tw[(k * r) * (M / (NS * R))]));
    }
    dft_small<R, DIR>(x);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b + r * NB] = x[r];
  }
  if constexpr (NS * R < M) {
    if constexpr (LEAD || NS > 1) line_sync<WARP>();  // previous readers of sm are done
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * Tl;
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[si(base + r * NS)] = v[b + r * NB];
    }
    line_sync<WARP>();
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sm[si(t + q * Tl)];
    fft_stages<M, E, NS * R, DIR, WARP>(v, sm, si, t, tw);
  }
}

// ---------------------------------------------------------------------------
// 256-point complex64 line by 16 threads of 16 values: the same radix-16 x 16
// Stockham transform as line_dft<256, 16>, with
//  * the 15 stage-2 twiddles e^{-2 pi i t r/256} (r = 1..15) of thread t read
//    from a shared table tws (dft256_twiddles), two per 16-byte load;
//  * with VEC, the stage-1 results (positions 16t .. 16t+15, contiguous and
//    16-byte aligned in the exchange layout si) stored as 16-byte pairs.
// v[q] = f[t + 16 q] on entry, F[f][t + 16 q] on return (DIR = -1 forward,
// +1 inverse unnormalised).  Every thread of the line group must call it.
// ---------------------------------------------------------------------------
constexpr int kTw256Stride = 9;  // float4 per thread row of the table (8 used + 1 pad: no bank conflicts)

// Fill tws[t * 9 + i] = {w(t, 2i), w(t, 2i + 1)} with w(t, r) = tw[(t r) mod 256]
// (tw: the e^{-2 pi i m / 256} table); caller synchronises before use.
__device__ __forceinline__ void dft256_twiddles(float4* tws, const float2* __restrict__ tw) {
  for (int i = threadIdx.x; i < 16 * 8; i += blockDim.x) {
    const int t = i >> 3, r = 2 * (i & 7);
    const float2 a = tw[(t * r) & 255], b = tw[(t * (r + 1)) & 255];
    tws[t * kTw256Stride + (i & 7)] = make_float4(a.x, a.y, b.x, b.y);
  }
}

template <int DIR, bool WARP, bool VEC, typename SI>
__device__ __forceinline__ void dft256x16(float2 (&v)[16], float2* sm, const SI& si, int t, const float4* tws) {
  dft16<DIR>(v);
  line_sync<WARP>();  // previous readers of sm are done
  if constexpr (VEC) {
    float4* d = reinterpret_cast<float4*>(sm + si(16 * t));
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) sm[si(16 * t + r)] = v[r];
  }
  line_sync<WARP>();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = sm[si(t + 16 * q)];
  const float4* w = tws + t * kTw256Stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 p = w[i];
    if (i > 0) v[2 * i] = ctw<DIR>(v[2 * i], make_float2(p.x, p.y));
    v[2 * i + 1] = ctw<DIR>(v[2 * i + 1], make_float2(p.z, p.w));
  }
  dft16<DIR>(v);
}

// Forward (DIR = -1) or inverse-unnormalised (DIR = +1) DFT of one line held
// as v[q] = f[t + q*Tl]; on return v[q] = F[f][t + q*Tl].  Every thread of the
// block (WARP: of the warp) must call it: it contains the stage barriers.
template <int M, int E, int DIR, bool WARP = false, bool LEAD = true, typename C, typename SI>
__device__ __forceinline__ void line_dft(C (&v)[E], C* sm, const SI& si, int t, const C* __restrict__ tw) {
  fft_stages<M, E, 1, DIR, WARP, LEAD>(v, sm, si, t, tw);
}

}  // namespace gpe
