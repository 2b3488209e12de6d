// FP64 instantiations of the fused half-step kernel (state and arithmetic in
// double; used for the plain method and its discrete adjoint).
#include "fused.cuh"

namespace hermite {

cudaError_t launch_fused_f64(int m, const double *in, double *out, const Geom &g,
                             const StepCoeffs<double> &co, int zchunk, cudaStream_t st) {
  switch (m) {
    case 1: return launch_fused_cfg<double, double, 2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 2: return launch_fused_cfg<double, double, 3, 4, 4, 160>(in, out, g, co, zchunk, st);
    case 3: return launch_fused_cfg<double, double, 4, 4, 4, 256>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hermite
