// FP32-arithmetic instantiations of the fused half-step kernel, with the state
// stored in FP32 or in FP64 (loaded, computed in FP32, stored back in FP64).
#include "fused.cuh"

namespace hermite {

template <typename TS>
static cudaError_t dispatch_f32(int m, const TS *in, TS *out, const Geom &g, const StepCoeffs<float> &co,
                                int zchunk, cudaStream_t st) {
  switch (m) {
    case 1: return launch_fused_cfg<TS, float, 2, 16, 8, 512>(in, out, g, co, zchunk, st);
    case 2: return launch_fused_cfg<TS, float, 3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 3: return launch_fused_cfg<TS, float, 4, 4, 4, 256>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_f32(int m, int state, const void *in, void *out, const Geom &g,
                             const StepCoeffs<float> &co, int zchunk, cudaStream_t st) {
  if (state == kF64) return dispatch_f32<double>(m, (const double *)in, (double *)out, g, co, zchunk, st);
  return dispatch_f32<float>(m, (const float *)in, (float *)out, g, co, zchunk, st);
}

}  // namespace hermite
