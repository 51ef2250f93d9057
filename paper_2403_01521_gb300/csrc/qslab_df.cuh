// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits). Built from the error-free
// transformations two-sum (Knuth, TAOCP vol. 2, 4.2.2) and two-product with a
// fused multiply-add (the FMA computes a*b - fl(a*b) exactly).
//
// It carries the chunk-to-chunk recurrences of the FP32 path: those are long
// dependent chains, and on this GPU a dependent FP64 operation costs far more
// latency than the dozen FP32 operations that replace it.
#pragma once
#include <cuda_runtime.h>

namespace qslab {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ DF operator+(DF x, DF y) {
  DF s = df_two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF operator+(DF x, float y) {
  DF s = df_two_sum(x.hi, y);
  s.lo += x.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF operator-(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }

__device__ __forceinline__ DF operator*(DF x, DF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ DF df_from(float x) { return {x, 0.0f}; }
__device__ __forceinline__ float df_to_float(DF x) { return x.hi + x.lo; }
__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

// Arithmetic type of the carries: FP64 on the FP64 path, double-float on the
// FP32 path.
template <typename T> struct CarryNum;
template <> struct CarryNum<double> { using type = double; };
template <> struct CarryNum<float> { using type = DF; };

__device__ __forceinline__ double cn_from(double x, double*) { return x; }
__device__ __forceinline__ DF cn_from(double x, DF*) { return df_from(x); }
__device__ __forceinline__ double cn_from_t(double x, double*) { return x; }
__device__ __forceinline__ DF cn_from_t(float x, DF*) { return df_from(x); }
__device__ __forceinline__ double cn_to_t(double x) { return x; }
__device__ __forceinline__ float cn_to_t(DF x) { return df_to_float(x); }
__device__ __forceinline__ double cn_to_double(double x) { return x; }
__device__ __forceinline__ double cn_to_double(DF x) { return df_to_double(x); }
__device__ __forceinline__ double cn_zero(double*) { return 0.0; }
__device__ __forceinline__ DF cn_zero(DF*) { return {0.0f, 0.0f}; }

}  // namespace qslab
