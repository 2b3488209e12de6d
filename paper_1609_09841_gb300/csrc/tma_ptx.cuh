// Inline-PTX helpers for tiled bulk tensor copies (TMA) from global into
// shared memory, paced by an mbarrier transaction count, and the host-side
// encoding of the tensor map that describes a half-step state to the copy
// engine.
//
// A state is the array [f][i3][i2][i1][z][y][x] (x fastest).  As a tensor of
// rank 4 it has the dimensions {nx, ny, nz, 2 (m+1)^3}: x, y, z and the
// coefficient row c = ((f (m+1) + i3) (m+1) + i2) (m+1) + i1.  One copy of a
// box {BW, TY + 1, 1, 2 (m+1)^3} brings every coefficient of a (TY + 1) x BW
// window of one node plane into shared memory, laid out [c][y][x].
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace hermite {
namespace tma {

// Makes the mbarrier initialisation visible to the copy engine (async proxy).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// One arrival on the mbarrier that also raises its transaction count by
// `bytes`: the phase completes once the copies have delivered that many.
__device__ __forceinline__ void arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(mbar)), "r"(bytes)
               : "memory");
}

// Tiled copy of the box at coordinates (c0 innermost .. c3) of `map` into
// shared memory at `dst` (128-byte aligned); completes `bytes` on `mbar`.
__device__ __forceinline__ void load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                        uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_addr(mbar))
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace tma

// Host: the tensor map of a state at `base` (elem_bytes 4 or 8) with nodes
// nx x ny x nz and ncoef coefficient rows, for boxes {box_x, box_y, 1, ncoef}.
// Returns false (and leaves *map unspecified) when the copy engine cannot
// address the state this way: base not 16-byte aligned, a row pitch nx *
// elem_bytes that is not a multiple of 16 bytes, a box outside the limits, or
// no driver entry point.  Callers then fill the staging buffer with plain loads.
bool encode_state_map(CUtensorMap *map, const void *base, int elem_bytes, int nx, int ny, int nz, int ncoef,
                      int box_x, int box_y);

}  // namespace hermite
