// FP64 instantiations of the fused half-step kernel (state and arithmetic in
// double; used for the plain method, its adjoint and dS/dc).  Each order has
// a few tile shapes (TX x TY cells per CTA, threads); the plan's schedule
// picks one (see the autotuner).
#include "fused.cuh"

namespace hermite {

int fused_tile_count(int prec, int m) {
  (void)m;
  return prec == 0 ? 5 : 8;  // FP32: 6 plain + 2 staged
}

cudaError_t launch_fused_f64(int m, int tile, const double *in, double *out, const Geom &g,
                             const StepCoeffs<double> &co, int zchunk, cudaStream_t st) {
  using T = double;
  switch (m * 8 + tile) {
    case 8 + 0: return launch_fused_cfg<T, T, 2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 8 + 1: return launch_fused_cfg<T, T, 2, 16, 4, 256>(in, out, g, co, zchunk, st);
    case 8 + 2: return launch_fused_cfg<T, T, 2, 16, 8, 512>(in, out, g, co, zchunk, st);
    case 8 + 3: return launch_fused_cfg<T, T, 2, 8, 8, 256, 2, 2>(in, out, g, co, zchunk, st);
    case 8 + 4: return launch_fused_cfg<T, T, 2, 16, 4, 256, 2, 2>(in, out, g, co, zchunk, st);
    case 16 + 0: return launch_fused_cfg<T, T, 3, 4, 4, 160>(in, out, g, co, zchunk, st);
    case 16 + 1: return launch_fused_cfg<T, T, 3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 16 + 2: return launch_fused_cfg<T, T, 3, 4, 8, 288>(in, out, g, co, zchunk, st);
    case 16 + 3: return launch_fused_cfg<T, T, 3, 4, 4, 160, 2, 3>(in, out, g, co, zchunk, st);
    case 16 + 4: return launch_fused_cfg<T, T, 3, 8, 4, 288, 2, 2>(in, out, g, co, zchunk, st);
    case 24 + 0: return launch_fused_cfg<T, T, 4, 4, 4, 256>(in, out, g, co, zchunk, st);
    case 24 + 1: return launch_fused_cfg<T, T, 4, 4, 2, 128>(in, out, g, co, zchunk, st);
    case 24 + 2: return launch_fused_cfg<T, T, 4, 8, 2, 256>(in, out, g, co, zchunk, st);
    case 24 + 3: return launch_fused_cfg<T, T, 4, 4, 4, 256, 2, 2>(in, out, g, co, zchunk, st);
    case 24 + 4: return launch_fused_cfg<T, T, 4, 4, 2, 128, 2, 3>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_f64_fullq(int m, const double *in, double *out, const Geom &g,
                                   const StepCoeffs<double> &co, int zchunk, cudaStream_t st) {
  using T = double;
  switch (m) {  // grade bound G = 2m (m = 1 needs no more than the RK4 kernel)
    case 1: return launch_fused_cfg<T, T, 2, 8, 8, 256, 2>(in, out, g, co, zchunk, st);
    case 2: return launch_fused_cfg<T, T, 3, 4, 4, 160, 4>(in, out, g, co, zchunk, st);
    case 3: return launch_fused_cfg<T, T, 4, 4, 2, 128, 6>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hermite
