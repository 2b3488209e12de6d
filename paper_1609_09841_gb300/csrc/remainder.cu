// Instantiations of the remainder-form fused half step (remainder.cuh): FP64
// state, FP32 arithmetic with exact leading sums.  Three tile shapes per
// order; the plan's schedule picks one.
#include "remainder.cuh"

namespace hermite {

int remainder_tile_count() { return 3; }

// Tile 0: 8 x 8 / 8 x 4 / 8 x 4 cells (one CTA per SM at m = 3); tiles 1, 2: two CTAs of 256
// threads per SM (8 x 2 and 4 x 4 cells at m = 3, 112 / 104 KB of shared memory each), so that
// one CTA's barriers overlap the other's work.
cudaError_t launch_remainder(int m, int tile, const double *in, double *out, const Geom &g, const RemCoeffs &co,
                             int zchunk, cudaStream_t st) {
  switch (m * 8 + tile) {
    case 8 + 0: return launch_rem_cfg<2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 8 + 1: return launch_rem_cfg<2, 8, 4, 128, 4>(in, out, g, co, zchunk, st);
    case 8 + 2: return launch_rem_cfg<2, 16, 8, 512, 1>(in, out, g, co, zchunk, st);
    case 16 + 0: return launch_rem_cfg<3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 16 + 1: return launch_rem_cfg<3, 8, 2, 144, 3>(in, out, g, co, zchunk, st);
    case 16 + 2: return launch_rem_cfg<3, 4, 4, 144, 3>(in, out, g, co, zchunk, st);
    case 24 + 0: return launch_rem_cfg<4, 8, 4, 512>(in, out, g, co, zchunk, st);
    case 24 + 1: return launch_rem_cfg<4, 8, 2, 256, 2>(in, out, g, co, zchunk, st);
    case 24 + 2: return launch_rem_cfg<4, 4, 4, 256, 2>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hermite
