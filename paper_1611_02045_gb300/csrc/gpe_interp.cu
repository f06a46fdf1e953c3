// gpe_interp.cu -- spectral (trigonometric) interpolation of a complex128
// field onto a grid twice as fine along one axis, for the multigrid
// continuation of Section 6 (ground state on M_p points, interpolated onto
// M_{p+1} = 2 M_p points as the next initial data).
//
// Along the axis, a line of Mc coarse values f is replaced by the samples at
// the Mf = 2 Mc fine points of
//   g(x) = (1/Mc) sum_p F_p e^{i xi_p (x + L)},  F = DFT_Mc(f),
// the Nyquist coefficient F_{-Mc/2} being shared equally by the modes -Mc/2
// and +Mc/2 (real data stay real).  In DFT order the fine spectrum is
//   G_k = F_k (k < Mc/2),  G_{Mf - Mc + k} = F_k (Mc/2 < k < Mc),
//   G_{Mc/2} = G_{Mf - Mc/2} = F_{Mc/2} / 2,  0 elsewhere,
// and g = IDFT_Mf(G) * Mf / Mc, i.e. the unnormalised inverse times 1/Mc.
//
// A line is held by Tl = Mc/4 threads: the coarse transform with E = 4 values
// per thread leaves F_{t + q Tl} (q < 4) in thread t, and the fine transform
// with E = 8 uses the same Tl = Mf/8, so the padded spectrum is assembled in
// registers: fine slots 0, 1 <- coarse 0, 1; slots 6, 7 <- coarse 2, 3; slot 2
// of thread 0 (index Mc/2) and slot 6 of thread 0 (index Mf - Mc/2) share the
// Nyquist value; slots 2..5 are zero otherwise.
#include "gpe_fft.cuh"
#include "gpe_internal.h"

namespace gpe {

namespace {

template <int Mc>
__global__ void __launch_bounds__(256) k_interp(InterpArgs a) {
  constexpr int Mf = 2 * Mc, Tl = Mc / 4;
  constexpr int LS = Mf + Mf / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int t = threadIdx.x % Tl, l = threadIdx.x / Tl;
  const long long line = (long long)blockIdx.x * (blockDim.x / Tl) + l;  // grid covers the lines exactly
  const long long inner = line % a.inner_count, outer = line / a.inner_count;
  const double2* __restrict__ in = a.in + outer * a.in_outer + inner * a.in_inner;
  double2* __restrict__ out = a.out + outer * a.out_outer + inner * a.out_inner;
  auto si = [l](int pos) { return l * LS + pos + (pos >> 4); };

  double2 vc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) vc[q] = in[(long long)(t + q * Tl) * a.in_stride];
  line_dft<Mc, 4, -1>(vc, sm, si, t, a.tw_c);
  const double s = 1.0 / Mc;
  const double2 z = make_double2(0.0, 0.0);
  const double2 nyq = make_double2(0.5 * s * vc[2].x, 0.5 * s * vc[2].y);
  double2 vf[8];
  vf[0] = make_double2(s * vc[0].x, s * vc[0].y);
  vf[1] = make_double2(s * vc[1].x, s * vc[1].y);
  vf[2] = (t == 0) ? nyq : z;
  vf[3] = z;
  vf[4] = z;
  vf[5] = z;
  vf[6] = (t == 0) ? nyq : make_double2(s * vc[2].x, s * vc[2].y);
  vf[7] = make_double2(s * vc[3].x, s * vc[3].y);
  line_dft<Mf, 8, +1>(vf, sm, si, t, a.tw_f);
#pragma unroll
  for (int q = 0; q < 8; ++q) out[(long long)(t + q * Tl) * a.out_stride] = vf[q];
}

template <int Mc>
cudaError_t launch_interp_one(const InterpArgs& a, cudaStream_t st) {
  constexpr int Tl = Mc / 4, LS = 2 * Mc + 2 * Mc / 16;
  long long lpb = 256 / Tl;
  if (lpb < 1) lpb = 1;
  while (lpb > 1 && a.lines % lpb != 0) lpb >>= 1;
  const size_t smem = (size_t)lpb * LS * sizeof(double2);
  static DeviceOnce attr;
  const int dev = DeviceOnce::device();
  if (!attr.done(dev)) {
    const cudaError_t e = cudaFuncSetAttribute(k_interp<Mc>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.set(dev);
  }
  k_interp<Mc><<<(unsigned)(a.lines / lpb), (unsigned)(Tl * lpb), smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp(int Mc, const InterpArgs& a, cudaStream_t st) {
  switch (Mc) {
    case 8: return launch_interp_one<8>(a, st);
    case 16: return launch_interp_one<16>(a, st);
    case 32: return launch_interp_one<32>(a, st);
    case 64: return launch_interp_one<64>(a, st);
    case 128: return launch_interp_one<128>(a, st);
    case 256: return launch_interp_one<256>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpe
