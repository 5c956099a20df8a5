// Compensated single precision ("float-float"): a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi) / 2, which carries about 48
// significant bits while every operation runs on the FP32 pipes.  Used where
// FP32 rounding noise would be amplified downstream (the FFTs of the coarse
// octree levels, whose fields are extrapolated to the child block faces by
// the Lagrange interpolation of the downward pass).
//
// The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum) and the FMA form of the exact product error; the sum and
// product below follow the "double-double" arithmetic of Hida, Li & Bailey
// (sloppy add, i.e. one TwoSum on the high parts).  Every step is written out
// with plain additions so that no reassociation can remove the error terms.
#pragma once
#include <cuda_runtime.h>

namespace flgf {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(float h) : hi(h), lo(0.0f) {}  // NOLINT: implicit widening
};

__device__ __forceinline__ ff ff_fast2sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  const float e = b - (s - a);
  return ff(s, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  // TwoSum of the high parts
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return ff_fast2sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  const float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the high product
  return ff_fast2sum(p, e + (a.hi * b.lo + a.lo * b.hi));
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }

// a * b + c for every arithmetic type (fused for float and double)
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ ff mad(ff a, ff b, ff c) { return a * b + c; }

__device__ __forceinline__ float ff_to_float(ff a) { return a.hi + a.lo; }
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = (float)d;
  return ff(h, (float)(d - (double)h));
}

// A sum of products w_m x_m accumulated term by term (the rows of the
// interpolation).  float and double: one FMA per term, as mad().  ff: the
// compensated dot product of Ogita, Rump & Oishi ("Dot2", 2005) extended to
// float-float operands: the product of the high parts and the running sum of
// the high parts are error-free (FMA product error, TwoSum); those errors and
// the cross products with the low parts add into one float, and the pair is
// renormalised once at the end.  About 12 flops per term against about 20 for
// a float-float multiply-add, at the same twice-working precision.
template <typename C> struct DotAcc {
  C v;
  static __device__ __forceinline__ DotAcc zero() { return DotAcc{C(0)}; }
  static __device__ __forceinline__ DotAcc prod(C w, C x) { return DotAcc{w * x}; }
  __device__ __forceinline__ void add(C w, C x) { v = mad(w, x, v); }
  __device__ __forceinline__ C result() const { return v; }
};
template <> struct DotAcc<ff> {
  float s, c;
  static __device__ __forceinline__ DotAcc zero() { return DotAcc{0.0f, 0.0f}; }
  static __device__ __forceinline__ DotAcc prod(ff w, ff x) {
    const float p = w.hi * x.hi;
    float e = __fmaf_rn(w.hi, x.hi, -p);
    e = __fmaf_rn(w.hi, x.lo, e);
    e = __fmaf_rn(w.lo, x.hi, e);
    return DotAcc{p, e};
  }
  __device__ __forceinline__ void add(ff w, ff x) {
    const float p = w.hi * x.hi;
    float e = __fmaf_rn(w.hi, x.hi, -p);
    e = __fmaf_rn(w.hi, x.lo, e);
    e = __fmaf_rn(w.lo, x.hi, e);
    const float t = s + p;  // TwoSum(s, p)
    const float bb = t - s;
    const float q = (s - (t - bb)) + (p - bb);
    s = t;
    c = c + (q + e);
  }
  __device__ __forceinline__ ff result() const { return ff_fast2sum(s, c); }
};

// Conversions between the storage type R (float or double) and a compute
// type C (float, double or ff).
template <typename C> struct Arith;
template <> struct Arith<float> {
  static __device__ __forceinline__ float from(float v) { return v; }
  static __device__ __forceinline__ float from_d(double v) { return (float)v; }
  template <typename R> static __device__ __forceinline__ R to(float v) { return (R)v; }
};
template <> struct Arith<double> {
  static __device__ __forceinline__ double from(double v) { return v; }
  static __device__ __forceinline__ double from_d(double v) { return v; }
  template <typename R> static __device__ __forceinline__ R to(double v) { return (R)v; }
};
template <> struct Arith<ff> {
  static __device__ __forceinline__ ff from(float v) { return ff(v); }
  static __device__ __forceinline__ ff from_d(double v) { return ff_from_double(v); }
  template <typename R> static __device__ __forceinline__ R to(ff v) { return (R)ff_to_float(v); }
};

}  // namespace flgf
