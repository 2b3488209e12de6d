// FP32-arithmetic instantiations of the fused half-step kernel with an FP64
// state (loaded, computed in FP32, stored back in FP64).
#include "fused_f32.cuh"

namespace hermite {

cudaError_t launch_fused_f32_s64(int m, int tile, const double *in, double *out, const Geom &g,
                                 const StepCoeffs<float> &co, int zchunk, int *status, cudaStream_t st) {
  return dispatch_f32<double>(m, tile, in, out, g, co, zchunk, status, st);
}

cudaError_t launch_fused_f32_fullq_s64(int m, const double *in, double *out, const Geom &g,
                                       const StepCoeffs<float> &co, int zchunk, cudaStream_t st) {
  return dispatch_f32_fullq<double>(m, in, out, g, co, zchunk, st);
}

}  // namespace hermite
