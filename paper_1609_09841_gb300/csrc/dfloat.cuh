// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits), built from the error-free
// transformations TwoSum (Knuth) and TwoProd (with FMA), as in Dekker,
// "A floating-point technique for extending the available precision" (1971),
// and Hida, Li and Bailey's double-double library.  Used by the hybrid
// precision mode for the contractions that cancel catastrophically.
#pragma once

#include <cuda_runtime.h>

namespace hermite {

struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df32 df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float df_to_float(df32 a) { return a.hi + a.lo; }

__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
  const df32 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + df32{-b.hi, -b.lo}; }

// acc + c * x
__device__ __forceinline__ df32 df_fma(df32 c, df32 x, df32 acc) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  e = fmaf(c.lo, x.hi, e);
  const df32 s = df_two_sum(acc.hi, p);
  return df_fast_two_sum(s.hi, s.lo + (acc.lo + e));
}

}  // namespace hermite
