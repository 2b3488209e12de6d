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

// The float holding the top 24 significand bits of a double (truncation),
// composed with integer operations.  Values below 2^-126 give 0 (their low
// word is dropped too); values must be below 2^128.
__device__ __forceinline__ float df_trunc_hi(long long b) {
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return 0.f;
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
}

// The double equal to a normal float, composed with integer operations
// (zero and subnormal floats give 0).
__device__ __forceinline__ double df_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return 0.0;
  return __longlong_as_double(((unsigned long long)(u >> 31) << 63) |
                              ((unsigned long long)(e - 127 + 1023) << 52) |
                              ((unsigned long long)(u & 0x7FFFFF) << 29));
}

// Split a double into hi + lo without FP64 instructions: hi keeps the top 24
// significand bits (exact in FP32), lo the remaining 29 bits rounded to FP32
// (scaled by the exponent; values below 2^-74 keep hi only).  The pair is
// accurate to about 2^-47 relative.
__device__ __forceinline__ df32 df_from(double x) {
  const long long b = __double_as_longlong(x);
  const float hi = df_trunc_hi(b);
  const int e = (int)((b >> 52) & 0x7FF) - 1075;  // weight of the last significand bit is 2^e
  float lo = 0.f;
  if (e >= -126) {
    lo = (float)(int)(b & 0x1FFFFFFFLL) * __uint_as_float((unsigned)(e + 127) << 23);
    if (b < 0) lo = -lo;
  }
  return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df32 a) { return df_widen(a.hi) + df_widen(a.lo); }
__device__ __forceinline__ float df_to_float(df32 a) { return a.hi + a.lo; }

__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
  const df32 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + df32{-b.hi, -b.lo}; }

// Renormalise a pair whose lo may have grown (|hi| >= |lo| holds).
__device__ __forceinline__ df32 df_norm(df32 a) { return df_fast_two_sum(a.hi, a.lo); }

// acc + c * x without renormalisation (acc.lo accumulates the low parts; call
// df_norm at the end of a short chain).
__device__ __forceinline__ df32 df_mad(df32 c, df32 x, df32 acc) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  e = fmaf(c.lo, x.hi, e);
  const df32 s = df_two_sum(acc.hi, p);
  return {s.hi, s.lo + (acc.lo + e)};
}

// The same with a coefficient exact in FP32.
__device__ __forceinline__ df32 df_mad1(float c, df32 x, df32 acc) {
  const float p = c * x.hi;
  float e = fmaf(c, x.hi, -p);
  e = fmaf(c, x.lo, e);
  const df32 s = df_two_sum(acc.hi, p);
  return {s.hi, s.lo + (acc.lo + e)};
}

// acc + c * x, renormalised
__device__ __forceinline__ df32 df_fma(df32 c, df32 x, df32 acc) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  e = fmaf(c.lo, x.hi, e);
  const df32 s = df_two_sum(acc.hi, p);
  return df_fast_two_sum(s.hi, s.lo + (acc.lo + e));
}

}  // namespace hermite
