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

// Split a double into hi + lo without FP64 arithmetic: hi keeps the top 24
// significand bits (exact in FP32), lo the remaining 29 bits rounded to FP32
// (scaled by the exponent; values below 2^-74 keep hi only).  The pair is
// accurate to about 2^-47 relative.  hi is assembled from the bits (sign,
// exponent rebiased from 1023 to 127, the top 23 stored significand bits)
// when it is a normal FP32 number, which keeps the conversion off the FP64
// pipe; outside that range (zero, tiny, huge, non-finite) the masked double
// is converted, to the same value.
__device__ __forceinline__ df32 df_from(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned bh = (unsigned)((unsigned long long)b >> 32), bl = (unsigned)b;
  const int ef = (int)((bh >> 20) & 0x7FFu) - 1023 + 127;  // biased FP32 exponent of x
  float hi;
  if (ef >= 1 && ef <= 254)
    hi = __uint_as_float((bh & 0x80000000u) | ((unsigned)ef << 23) | (__funnelshift_r(bl, bh, 29) & 0x7FFFFFu));
  else
    hi = __double2float_rn(__longlong_as_double(b & ~0x1FFFFFFFLL));
  const int e = (int)((b >> 52) & 0x7FF) - 1075;  // weight of the last significand bit is 2^e
  float lo = 0.f;
  if (e >= -126) {
    lo = (float)(int)(b & 0x1FFFFFFFLL) * __int_as_float((e + 127) << 23);
    if (b < 0) lo = -lo;
  }
  return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }
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

}  // namespace hermite
