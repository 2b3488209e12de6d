// Instantiations of the hybrid-precision fused half step: the grade-0 chain in
// FP64 (HiF64) or in double-float (HiDF), the rest in FP32; FP64 state.
#include "hybrid.cuh"

namespace hermite {

int hybrid_tile_count() { return 2; }

template <class Hi>
static cudaError_t dispatch_hybrid(int m, int tile, const double *in, double *out, const Geom &g,
                                   const HybridCoeffs &co, int zchunk, cudaStream_t st) {
  switch (m * 8 + tile) {
    case 8 + 0: return launch_hybrid_cfg<Hi, 2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 8 + 1: return launch_hybrid_cfg<Hi, 2, 16, 8, 512>(in, out, g, co, zchunk, st);
    case 16 + 0: return launch_hybrid_cfg<Hi, 3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 16 + 1: return launch_hybrid_cfg<Hi, 3, 4, 4, 160>(in, out, g, co, zchunk, st);
    case 24 + 0: return launch_hybrid_cfg<Hi, 4, 4, 4, 256>(in, out, g, co, zchunk, st);
    case 24 + 1: return launch_hybrid_cfg<Hi, 4, 8, 4, 512>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_hybrid(int kind, int m, int tile, const double *in, double *out, const Geom &g,
                          const HybridCoeffs &co, int zchunk, cudaStream_t st) {
  if (kind == 0) return dispatch_hybrid<HiF64>(m, tile, in, out, g, co, zchunk, st);
  return dispatch_hybrid<HiDF>(m, tile, in, out, g, co, zchunk, st);
}

}  // namespace hermite
