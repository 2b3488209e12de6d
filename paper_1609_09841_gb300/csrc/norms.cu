// FP64 error norms of a state against an FP64 reference (max, relative max,
// RMS and relative L2 over the selected components).  Two launches: a grid of
// CTAs writes per-CTA partials (warp-shuffle reductions, then shared memory),
// one CTA folds the partials.
#include <cuda_runtime.h>

#include "hermite_impl.h"

namespace hermite {

namespace {
constexpr int kErrThreads = 256;
constexpr int kErrBlocks = 2 * 152;  // two CTAs per SM of a GB300

struct Acc {
  double maxd, maxb, sdd, sbb, nonfinite;
};

__device__ __forceinline__ void acc_merge(Acc &a, const Acc &b) {
  a.maxd = fmax(a.maxd, b.maxd);
  a.maxb = fmax(a.maxb, b.maxb);
  a.sdd += b.sdd;
  a.sbb += b.sbb;
  a.nonfinite += b.nonfinite;
}

__device__ Acc block_reduce(Acc v) {
  __shared__ Acc red[kErrThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    Acc w;
    w.maxd = __shfl_xor_sync(0xffffffffu, v.maxd, o);
    w.maxb = __shfl_xor_sync(0xffffffffu, v.maxb, o);
    w.sdd = __shfl_xor_sync(0xffffffffu, v.sdd, o);
    w.sbb = __shfl_xor_sync(0xffffffffu, v.sbb, o);
    w.nonfinite = __shfl_xor_sync(0xffffffffu, v.nonfinite, o);
    acc_merge(v, w);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : Acc{0, 0, 0, 0, 0};
    for (int o = 16; o > 0; o >>= 1) {
      Acc w;
      w.maxd = __shfl_xor_sync(0xffffffffu, v.maxd, o);
      w.maxb = __shfl_xor_sync(0xffffffffu, v.maxb, o);
      w.sdd = __shfl_xor_sync(0xffffffffu, v.sdd, o);
      w.sbb = __shfl_xor_sync(0xffffffffu, v.sbb, o);
      w.nonfinite = __shfl_xor_sync(0xffffffffu, v.nonfinite, o);
      acc_merge(v, w);
    }
  }
  return v;
}

template <typename TS>
__global__ void __launch_bounds__(kErrThreads)
    error_partial_kernel(const TS *__restrict__ a, const double *__restrict__ b, int nc, size_t plane,
                         unsigned mask, double *__restrict__ partial) {
  Acc v{0, 0, 0, 0, 0};
  const int ncomp = (mask & 4u) ? nc : 1;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int f = 0; f < 2; ++f) {
    if (!(mask >> f & 1u)) continue;
    for (int c = 0; c < ncomp; ++c) {
      const size_t base = (size_t)(f * nc + c) * plane;
      for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += stride) {
        const double av = (double)a[base + i], bv = b[base + i];
        const double d = av - bv;
        if (!isfinite(av) || !isfinite(bv)) {
          v.nonfinite += 1.0;
          continue;
        }
        v.maxd = fmax(v.maxd, fabs(d));
        v.maxb = fmax(v.maxb, fabs(bv));
        v.sdd = fma(d, d, v.sdd);
        v.sbb = fma(bv, bv, v.sbb);
      }
    }
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    double *p = partial + (size_t)blockIdx.x * 8;
    p[0] = v.maxd;
    p[1] = v.maxb;
    p[2] = v.sdd;
    p[3] = v.sbb;
    p[4] = v.nonfinite;
  }
}

__global__ void __launch_bounds__(kErrThreads)
    error_final_kernel(const double *__restrict__ partial, int blocks, double *__restrict__ result) {
  Acc v{0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) {
    const double *p = partial + (size_t)i * 8;
    acc_merge(v, Acc{p[0], p[1], p[2], p[3], p[4]});
  }
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    result[0] = v.maxd;
    result[1] = v.maxb;
    result[2] = v.sdd;
    result[3] = v.sbb;
    result[4] = v.nonfinite;
  }
}
template <typename TS>
__global__ void __launch_bounds__(kErrThreads)
    dot_partial_kernel(const TS *__restrict__ a, const TS *__restrict__ b, size_t n, double *__restrict__ partial) {
  Acc v{0, 0, 0, 0, 0};
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v.sdd = fma((double)a[i], (double)b[i], v.sdd);
  v = block_reduce(v);
  if (threadIdx.x == 0) {
    double *p = partial + (size_t)blockIdx.x * 8;
    p[0] = 0;
    p[1] = 0;
    p[2] = v.sdd;
    p[3] = 0;
    p[4] = 0;
  }
}
}  // namespace

int error_blocks() { return kErrBlocks; }

cudaError_t launch_dot(int state, const void *a, const void *b, size_t n, double *partial, int blocks,
                       double *result, cudaStream_t st) {
  if (state == kF64)
    dot_partial_kernel<double><<<blocks, kErrThreads, 0, st>>>((const double *)a, (const double *)b, n, partial);
  else
    dot_partial_kernel<float><<<blocks, kErrThreads, 0, st>>>((const float *)a, (const float *)b, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  error_final_kernel<<<1, kErrThreads, 0, st>>>(partial, blocks, result);
  return cudaGetLastError();
}

cudaError_t launch_error(int state, const void *a, const double *b, int m, size_t plane,
                         unsigned mask, double *partial, int blocks, double *result,
                         cudaStream_t st) {
  const int nc = (m + 1) * (m + 1) * (m + 1);
  if (state == kF64)
    error_partial_kernel<double><<<blocks, kErrThreads, 0, st>>>((const double *)a, b, nc, plane, mask,
                                                                 partial);
  else
    error_partial_kernel<float><<<blocks, kErrThreads, 0, st>>>((const float *)a, b, nc, plane, mask,
                                                                partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  error_final_kernel<<<1, kErrThreads, 0, st>>>(partial, blocks, result);
  return cudaGetLastError();
}

}  // namespace hermite
