// Instantiations of the remainder-form fused half step (remainder.cuh): FP64
// state, FP32 arithmetic with exact leading sums.  One tile shape per order,
// the hybrid kernel's measured defaults (8 x 8 / 8 x 4 / 8 x 4 cells).
#include "remainder.cuh"

namespace hermite {

cudaError_t launch_remainder(int m, const double *in, double *out, const Geom &g, const RemCoeffs &co, int zchunk,
                             cudaStream_t st) {
  switch (m) {
    case 1: return launch_rem_cfg<2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 2: return launch_rem_cfg<3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 3: return launch_rem_cfg<4, 8, 4, 512>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hermite
