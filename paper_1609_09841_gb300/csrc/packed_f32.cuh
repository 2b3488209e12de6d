// Packed FP32 pairs for the f32x2 instructions of sm_100 and later: a 64-bit
// register pair holds two floats (lane 0 the low word), and mul/fma
// .rn.f32x2 perform the two lane-wise .rn.f32 operations in one instruction,
// with the same rounding as the scalar ones.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

namespace hermite {

__device__ __forceinline__ unsigned long long pack2f(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2f(unsigned long long v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2f(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2f(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

inline unsigned long long pack_pair_host(float lo, float hi) {
  unsigned a, b;
  std::memcpy(&a, &lo, 4);
  std::memcpy(&b, &hi, 4);
  return ((unsigned long long)b << 32) | a;
}

}  // namespace hermite
