// gpe_ds.cuh -- double-single arithmetic: a real number as an unevaluated
// sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2), ~48 significant bits.
//
// Error-free transformations: TwoSum (D. E. Knuth, TAOCP vol. 2, 4.2.2),
// Fast-TwoSum and the product split by fused multiply-add (T. J. Dekker, "A
// floating-point technique for extending the available precision", Numer.
// Math. 18, 1971; the FMA form of the exact product is standard, e.g. J.-M.
// Muller et al., Handbook of Floating-Point Arithmetic, 2010, ch. 4).
// Division and square root take one Newton correction of the FP32 quotient /
// root.  Every operation runs on the FP32 pipe; on GB300 an FP64 instruction
// costs about 64 FP32 ones, so state that needs more than FP32 precision is
// carried in this form on the device.
#pragma once
#include <cuda_runtime.h>

namespace gpe {

// keep the standard overloads visible next to the double-single ones below
using ::fmax;
using ::sqrt;

struct dsf {
  float hi, lo;
  dsf() = default;
  __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dsf(float h) : hi(h), lo(0.0f) {}
  __host__ __device__ constexpr dsf(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ constexpr dsf(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit constexpr operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit constexpr operator float() const { return hi + lo; }
};

__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dsf(s, b - (s - a));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);  // s + e == a.hi + b.hi exactly
  e += a.lo + b.lo;
  return ds_fast_two_sum(s, e);
}
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // p + e == a.hi * b.hi exactly
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ds_fast_two_sum(p, e);
}
__device__ __forceinline__ dsf operator/(dsf a, dsf b) {
  const float q1 = a.hi / b.hi;
  const dsf r = a - b * dsf(q1);
  const float q2 = r.hi / b.hi;
  return ds_fast_two_sum(q1, q2);
}
__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { return a = a + b; }
__device__ __forceinline__ dsf& operator-=(dsf& a, dsf b) { return a = a - b; }
__device__ __forceinline__ dsf& operator*=(dsf& a, dsf b) { return a = a * b; }
__device__ __forceinline__ bool operator>(dsf a, dsf b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(dsf a, dsf b) { return b > a; }
__device__ __forceinline__ bool operator>=(dsf a, dsf b) { return !(b > a); }
__device__ __forceinline__ bool operator<=(dsf a, dsf b) { return !(a > b); }
__device__ __forceinline__ dsf fmax(dsf a, dsf b) { return (b > a) ? b : a; }
__device__ __forceinline__ dsf sqrt(dsf a) {
  if (!(a.hi > 0.0f)) return dsf(a.hi == 0.0f ? 0.0f : sqrtf(a.hi));  // 0, or NaN for negatives
  const float y = sqrtf(a.hi);
  const dsf r = a - dsf(y) * dsf(y);
  return ds_fast_two_sum(y, r.hi / (2.0f * y));
}

struct __align__(16) dsc {
  dsf x, y;
};

}  // namespace gpe
