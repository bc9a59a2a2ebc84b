// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 2^-46 relative precision with FP32's exponent range.  GB300 runs
// FP64 at a small fraction of its FP32 rate (a dependent FP64 multiply-add takes ~64 cycles,
// a divide ~420), so the small sequential dense solves run on the FP32 units in this format.
// The error-free transformations are the textbook ones (Knuth's two-sum, the FMA two-product;
// Dekker 1971, Bailey's double-double library; additions in the cheap form with a normwise
// bound); division and the reciprocal square root start from the FP32 approximate reciprocal /
// root and correct it once against the double-float residual (one Newton step).
#pragma once
#include <cuda_runtime.h>

namespace eig {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(float h) : hi(h), lo(0.0f) {}
  // constexpr so that constants fold at compile time (the casts round to nearest)
  __host__ __device__ constexpr dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  const float s = a + b;
  return dfl(s, b - (s - a));
}
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl(s, (a - (s - bb)) + (b - bb));
}

// Sum with a normwise error bound, |err| <= ~2^-45 (|a| + |b|) (the cheap double-float
// addition; every error bound of the small solvers is normwise, relative to the matrix norm).
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// acc + a * b with the product's error term folded into the sum
__device__ __forceinline__ dfl dfma(dfl a, dfl b, dfl acc) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const dfl s = two_sum(acc.hi, p);
  return quick_two_sum(s.hi, s.lo + (acc.lo + e));
}
__device__ __forceinline__ double dfma(double a, double b, double acc) { return fma(a, b, acc); }
// Quotient from an approximate FP32 reciprocal rb (~2^-23): q1 = a rb, then one correction
// q2 from the residual a - b q1 (~2^-23 a, computed to double-float accuracy) brings the
// relative error to ~2^-46.
__device__ __forceinline__ dfl operator/(dfl a, dfl b) {
  const float rb = rcp_approx(b.hi);
  const float q1 = a.hi * rb;
  const dfl r = a - b * dfl(q1, 0.0f);
  return quick_two_sum(q1, r.hi * rb);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
__device__ __forceinline__ dfl& operator/=(dfl& a, dfl b) { return a = a / b; }

__device__ __forceinline__ bool operator<(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dfl a, dfl b) { return b < a; }
__device__ __forceinline__ bool operator<=(dfl a, dfl b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dfl a, dfl b) { return !(a < b); }
__device__ __forceinline__ bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return !(a == b); }

__device__ __forceinline__ dfl fabs(dfl a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ dfl fmax(dfl a, dfl b) { return a < b ? b : a; }
__device__ __forceinline__ dfl fmin(dfl a, dfl b) { return b < a ? b : a; }
__device__ __forceinline__ dfl copysign(dfl mag, dfl sgn) {
  const dfl m = fabs(mag);
  return (sgn.hi < 0.0f || (sgn.hi == 0.0f && signbit(sgn.hi))) ? -m : m;
}
__device__ __forceinline__ bool isfinite(dfl a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }
// 1 / sqrt(a): the FP32 approximate root y (~2^-22) corrected once by Newton's step for
// f(y) = 1/y^2 - a, y' = y + y (1 - a y^2) / 2, with a y^2 formed to double-float accuracy
// (the correction is ~2^-22 y, so FP32 suffices for it): relative error ~2^-44.
__device__ __forceinline__ dfl rsqrt(dfl a) {
  if (!(a.hi > 0.0f)) return dfl(0.0f, 0.0f);
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
  const float y2 = y * y;
  const dfl yy(y2, fmaf(y, y, -y2));                      // y^2 exactly
  const dfl h = a * yy;
  const float r = (1.0f - h.hi) - h.lo;                  // 1 - a y^2, small
  return quick_two_sum(y, 0.5f * y * r);
}
// sqrt(a) = a / sqrt(a)
__device__ __forceinline__ dfl sqrt(dfl a) {
  if (!(a.hi > 0.0f)) return dfl(0.0f, 0.0f);
  return a * rsqrt(a);
}

// 1 when negative (the sign of the leading part), else 0
__device__ __forceinline__ int sign_bit(dfl a) { return (int)(__float_as_uint(a.hi) >> 31); }
__device__ __forceinline__ int sign_bit(double a) { return (int)((unsigned long long)__double_as_longlong(a) >> 63); }
// Leading FP32 part (a cheap magnitude for range checks)
__device__ __forceinline__ float lead_f32(dfl a) { return a.hi; }
__device__ __forceinline__ float lead_f32(double a) { return (float)a; }
// a * 2^e, exact (e within FP32's exponent range; the result neither over- nor underflows)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ dfl scale2(dfl a, int e) {
  const float f = pow2f(e);
  return dfl(a.hi * f, a.lo * f);
}
__device__ __forceinline__ double scale2(double a, int e) { return a * (double)pow2f(e); }

__device__ __forceinline__ dfl shfl_xor(dfl v, int o) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ dfl shfl(dfl v, int src) {
  return dfl(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}

// Scalar traits of the small solvers: machine epsilon and the guards against underflow.
template <typename R> struct SmallTraits;
template <> struct SmallTraits<double> {
  static constexpr double eps = 2.220446049250313e-16;
  static constexpr double tiny_abs = 1e-280, floor = 1e-300, pivmin = 1e-290, big = 1.7e308;
};
template <> struct SmallTraits<dfl> {
  static constexpr double eps = 1.4210854715202004e-14;   // 2^-46
  static constexpr double tiny_abs = 1e-30, floor = 1e-35, pivmin = 1e-32, big = 3.0e38;
};

}  // namespace eig
