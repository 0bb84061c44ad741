// Double-single arithmetic: FP64-accurate numbers as pairs of FP32 numbers on the FP32 pipe, which
// B300 runs at ~60x its FP64 rate.  Shared by the assembly kernels (paired Jacobian lanes, the
// double-single value path) and the line search's energy change.
#pragma once

#include "bp_internal.cuh"

namespace {

// An FP64-accurate number as two FP32 numbers, value = hi + lo with |lo| <= ulp(hi)/2 (error-free
// TwoSum for additions, TwoProd through fmaf for products; about 2^-47 relative error per operation,
// 8 fewer bits than FP64 but far inside the 1e-12 parity bar).
struct f64x2 {
  float hi, lo;
  __host__ __device__ constexpr f64x2() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr f64x2(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit f64x2(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit f64x2(int x) : f64x2((double)x) {}
  __host__ __device__ double value() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ f64x2 operator+(const f64x2 a, const f64x2 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return f64x2(h, e - (h - s));
}
__device__ __forceinline__ f64x2 operator-(const f64x2 a) { return f64x2(-a.hi, -a.lo); }
__device__ __forceinline__ f64x2 operator-(const f64x2 a, const f64x2 b) { return a + (-b); }
__device__ __forceinline__ f64x2 operator*(const f64x2 a, const f64x2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float h = p + e;
  return f64x2(h, e - (h - p));
}
__device__ __forceinline__ f64x2& operator+=(f64x2& a, const f64x2 b) {
  a = a + b;
  return a;
}

// a / b: quotient of the high parts, corrected by the remainder a - q b formed in pair arithmetic
__device__ __forceinline__ f64x2 operator/(const f64x2 a, const f64x2 b) {
  const float q1 = a.hi / b.hi;
  const f64x2 r = a - b * f64x2(q1, 0.f);
  const float q2 = (r.hi + r.lo) / b.hi;
  const float s = q1 + q2;
  return f64x2(s, q2 - (s - q1));
}
// FP64 -> pair: the high part rounded on the integer pipe, the remainder exact in FP64, rounded once
__device__ __forceinline__ f64x2 ds_of(const double x) {
  const float h = f32_of(x);
  return f64x2(h, f32_of(x - f64_of(h)));
}
__device__ __forceinline__ double ds_value(const f64x2 x) { return f64_of(x.hi) + f64_of(x.lo); }
// x^(-1/3): an FP32 seed y (rcbrtf) and one correction from e = 1 - x y^3 formed in pair arithmetic,
// y (1 + e/3 + 2 e^2/9) (|e| ~ 1e-7: the correction term needs FP32 accuracy only; truncation ~e^3)
__device__ __forceinline__ f64x2 ds_inv_cbrt(const f64x2 x) {
  const float y = rcbrtf(x.hi);
  const f64x2 Y(y, 0.f);
  const f64x2 e = f64x2(1.f, 0.f) - x * (Y * Y * Y);
  const float ef = e.hi + e.lo;
  const float c = y * (ef * fmaf(2.f / 9.f, ef, 1.f / 3.f));
  const float s = y + c;  // normalise (y, c): |c| << |y|
  return f64x2(s, c - (s - y));
}

}  // namespace
