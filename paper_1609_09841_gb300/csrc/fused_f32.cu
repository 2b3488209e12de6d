// FP32-arithmetic instantiations of the fused half-step kernel with an FP32
// state.  Each order has a few tile shapes; the plan's schedule picks one.
#include "fused_f32.cuh"

namespace hermite {

cudaError_t launch_fused_f32_s32(int m, int tile, const float *in, float *out, const Geom &g,
                                 const StepCoeffs<float> &co, int zchunk, int *status, cudaStream_t st) {
  return dispatch_f32<float>(m, tile, in, out, g, co, zchunk, status, st);
}

cudaError_t launch_fused_f32_fullq(int m, int state, const void *in, void *out, const Geom &g,
                                   const StepCoeffs<float> &co, int zchunk, cudaStream_t st) {
  if (state == kF64) return launch_fused_f32_fullq_s64(m, (const double *)in, (double *)out, g, co, zchunk, st);
  return dispatch_f32_fullq<float>(m, (const float *)in, (float *)out, g, co, zchunk, st);
}

}  // namespace hermite
