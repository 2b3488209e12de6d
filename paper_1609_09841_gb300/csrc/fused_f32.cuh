// Tile shapes of the FP32-arithmetic fused kernel, per order m.
#pragma once

#include "fused.cuh"

namespace hermite {

// Tiles 6 and 7 of every order are staged schedules (x-pass input copied
// into shared memory by the copy engine, launch_fused_st_cfg); `status`
// receives their copy time-outs.
template <typename TS>
cudaError_t dispatch_f32(int m, int tile, const TS *in, TS *out, const Geom &g, const StepCoeffs<float> &co,
                         int zchunk, int *status, cudaStream_t st) {
  switch (m * 8 + tile) {
    case 8 + 6: return launch_fused_st_cfg<TS, float, 2, 16, 8, 512, 2, 2>(in, out, g, co, zchunk, status, st);
    case 8 + 7: return launch_fused_st_cfg<TS, float, 2, 8, 8, 256, 2, 4>(in, out, g, co, zchunk, status, st);
    case 16 + 6: return launch_fused_st_cfg<TS, float, 3, 8, 4, 288, 2, 3>(in, out, g, co, zchunk, status, st);
    case 16 + 7: return launch_fused_st_cfg<TS, float, 3, 4, 4, 160, 2, 5>(in, out, g, co, zchunk, status, st);
    case 24 + 6: return launch_fused_st_cfg<TS, float, 4, 8, 2, 256, 2, 2>(in, out, g, co, zchunk, status, st);
    case 24 + 7: return launch_fused_st_cfg<TS, float, 4, 4, 4, 256, 2, 2>(in, out, g, co, zchunk, status, st);
    case 8 + 0: return launch_fused_cfg<TS, float, 2, 16, 8, 512>(in, out, g, co, zchunk, st);
    case 8 + 1: return launch_fused_cfg<TS, float, 2, 8, 8, 256>(in, out, g, co, zchunk, st);
    case 8 + 2: return launch_fused_cfg<TS, float, 2, 32, 4, 512>(in, out, g, co, zchunk, st);
    case 8 + 3: return launch_fused_cfg<TS, float, 2, 16, 16, 1024>(in, out, g, co, zchunk, st);
    case 8 + 4: return launch_fused_cfg<TS, float, 2, 8, 8, 256, 2, 4>(in, out, g, co, zchunk, st);
    case 8 + 5: return launch_fused_cfg<TS, float, 2, 32, 4, 512, 2, 2>(in, out, g, co, zchunk, st);
    case 16 + 0: return launch_fused_cfg<TS, float, 3, 8, 4, 288>(in, out, g, co, zchunk, st);
    case 16 + 1: return launch_fused_cfg<TS, float, 3, 4, 4, 160>(in, out, g, co, zchunk, st);
    case 16 + 2: return launch_fused_cfg<TS, float, 3, 8, 8, 576>(in, out, g, co, zchunk, st);
    case 16 + 3: return launch_fused_cfg<TS, float, 3, 16, 4, 576>(in, out, g, co, zchunk, st);
    case 16 + 4: return launch_fused_cfg<TS, float, 3, 8, 4, 288, 2, 3>(in, out, g, co, zchunk, st);
    case 16 + 5: return launch_fused_cfg<TS, float, 3, 4, 4, 160, 2, 5>(in, out, g, co, zchunk, st);
    case 24 + 0: return launch_fused_cfg<TS, float, 4, 4, 4, 256>(in, out, g, co, zchunk, st);
    case 24 + 1: return launch_fused_cfg<TS, float, 4, 8, 4, 256>(in, out, g, co, zchunk, st);
    case 24 + 2: return launch_fused_cfg<TS, float, 4, 8, 4, 512>(in, out, g, co, zchunk, st);
    case 24 + 3: return launch_fused_cfg<TS, float, 4, 4, 4, 128>(in, out, g, co, zchunk, st);
    case 24 + 4: return launch_fused_cfg<TS, float, 4, 4, 4, 256, 2, 3>(in, out, g, co, zchunk, st);
    case 24 + 5: return launch_fused_cfg<TS, float, 4, 8, 2, 256, 2, 3>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

template <typename TS>
cudaError_t dispatch_f32_fullq(int m, const TS *in, TS *out, const Geom &g, const StepCoeffs<float> &co,
                               int zchunk, cudaStream_t st) {
  switch (m) {  // grade bound G = 2m
    case 1: return launch_fused_cfg<TS, float, 2, 16, 8, 512, 2>(in, out, g, co, zchunk, st);
    case 2: return launch_fused_cfg<TS, float, 3, 8, 4, 288, 4>(in, out, g, co, zchunk, st);
    case 3: return launch_fused_cfg<TS, float, 4, 4, 4, 256, 6>(in, out, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_f32_fullq_s64(int m, const double *in, double *out, const Geom &g,
                                       const StepCoeffs<float> &co, int zchunk, cudaStream_t st);

}  // namespace hermite
