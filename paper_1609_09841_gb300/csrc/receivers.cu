// Receivers of the differentiation workload: gather the value component of u
// at a list of nodes after a half step, and the transpose of that gather (add
// weights into the value component of u of an adjoint state).
#include <cuda_runtime.h>

#include "hermite_impl.h"

namespace hermite {

namespace {

template <typename TS>
__global__ void record_kernel(const TS *__restrict__ state, const long long *__restrict__ idx, int count,
                              double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) out[k] = (double)state[idx[k]];  // field u, orders (0,0,0): the first plane
}

template <typename TS>
__global__ void inject_kernel(TS *__restrict__ adj, const long long *__restrict__ idx, int count,
                              const double *__restrict__ w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) atomicAdd(adj + idx[k], (TS)w[k]);  // duplicate receivers add up
}

}  // namespace

cudaError_t launch_record(int state, const void *s, const long long *idx, int count, double *out,
                          cudaStream_t st) {
  const int blocks = (count + 127) / 128;
  if (state == kF64)
    record_kernel<double><<<blocks, 128, 0, st>>>((const double *)s, idx, count, out);
  else
    record_kernel<float><<<blocks, 128, 0, st>>>((const float *)s, idx, count, out);
  return cudaGetLastError();
}

cudaError_t launch_inject(int state, void *adj, const long long *idx, int count, const double *w,
                          cudaStream_t st) {
  const int blocks = (count + 127) / 128;
  if (state == kF64)
    inject_kernel<double><<<blocks, 128, 0, st>>>((double *)adj, idx, count, w);
  else
    inject_kernel<float><<<blocks, 128, 0, st>>>((float *)adj, idx, count, w);
  return cudaGetLastError();
}

}  // namespace hermite
