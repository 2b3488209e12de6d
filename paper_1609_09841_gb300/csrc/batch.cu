// Batched half step: many independent simulations (each its own order m,
// grid and time step) advanced by ONE persistent launch.  The host builds a
// work list of (simulation, xy-tile, z-chunk) items, heaviest order first;
// each resident CTA takes the next item with an atomic counter, copies that
// simulation's tables into shared memory and runs the fused tile body of its
// order (the same code as the single-grid kernel).  No CTA ever waits on
// another, so there is nothing to time out.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "batch.h"
#include "fused.cuh"

namespace hermite {

// Tile shapes of the batched kernel, two per order (NT = 256 threads for
// all), chosen so that the x-, y- and z-pass items split over the threads with
// little left for a last partial chunk.  Items per thread (x, y, z pass):
//   m = 1: 16 x 8 -> 4.5, 4, 2;      8 x 8 -> 2.25, 2, 1
//   m = 2: 16 x 4 -> 5.6, 4.5, 2.25; 8 x 4 -> 2.8, 2.25, 1.1
//   m = 3:  8 x 2 -> 3, 2, 1;        4 x 4 -> 2.5, 2, 1
// Every second shape needs less shared memory than the largest first one, so
// offering it costs no occupancy.  The per-node arithmetic of the tile body
// does not depend on the shape, so every shape gives the same bits.
template <int M, int K> struct BatchTile;
template <> struct BatchTile<2, 0> { static constexpr int TX = 16, TY = 8; };
template <> struct BatchTile<2, 1> { static constexpr int TX = 8, TY = 8; };
template <> struct BatchTile<3, 0> { static constexpr int TX = 16, TY = 4; };
template <> struct BatchTile<3, 1> { static constexpr int TX = 8, TY = 4; };
template <> struct BatchTile<4, 0> { static constexpr int TX = 8, TY = 2; };
template <> struct BatchTile<4, 1> { static constexpr int TX = 4, TY = 4; };
constexpr int kBatchThreads = 256;
// Resident CTAs per SM the compiler must fit the batched kernel's registers to.
#ifndef HERMITE_BATCH_MIN_BLOCKS
#define HERMITE_BATCH_MIN_BLOCKS 2
#endif

template <int M, int K>
static void shape_of(int *tx, int *ty) {
  *tx = BatchTile<M, K>::TX;
  *ty = BatchTile<M, K>::TY;
}

void batch_tile_shape(int m, int k, int *tx, int *ty) {
  switch (m * kBatchShapes + (k == 1 ? 1 : 0)) {
    case 1 * kBatchShapes + 0: shape_of<2, 0>(tx, ty); break;
    case 1 * kBatchShapes + 1: shape_of<2, 1>(tx, ty); break;
    case 2 * kBatchShapes + 0: shape_of<3, 0>(tx, ty); break;
    case 2 * kBatchShapes + 1: shape_of<3, 1>(tx, ty); break;
    case 3 * kBatchShapes + 1: shape_of<4, 1>(tx, ty); break;
    default: shape_of<4, 0>(tx, ty); break;
  }
}

// Per-simulation table record: StepCoeffs<TC>, and for FP32 arithmetic the
// same tables as packed pairs (PackedCoeffs) right after it, so that the tile
// body runs its fma.rn.f32x2 path with the pairs read from shared memory.
template <typename TC>
constexpr bool kBatchPacked = std::is_same<TC, float>::value;

template <typename TC>
constexpr size_t batch_record_bytes() {
  return sizeof(StepCoeffs<TC>) + (kBatchPacked<TC> ? sizeof(PackedCoeffs) : 0);
}

static_assert(sizeof(StepCoeffs<float>) % 8 == 0 && sizeof(StepCoeffs<double>) % 8 == 0 &&
                  sizeof(PackedCoeffs) % 8 == 0,
              "table records are copied in 8-byte words and the packed pairs read as 8-byte values");

size_t batch_coeff_record_bytes(int compute) {
  return compute == kF64 ? batch_record_bytes<double>() : batch_record_bytes<float>();
}

void batch_write_record(int compute, const StepCoeffs<double> &cd, unsigned char *dst) {
  if (compute == kF64) {
    std::memcpy(dst, &cd, sizeof(cd));
    return;
  }
  const StepCoeffs<float> cf = cast_coeffs<float>(cd);
  const PackedCoeffs pc = pack_coeffs(cf);
  std::memcpy(dst, &cf, sizeof(cf));
  std::memcpy(dst + sizeof(cf), &pc, sizeof(pc));
}

template <typename TC>
constexpr size_t batch_tables_bytes() {  // the record in shared memory, 16-byte aligned
  return (batch_record_bytes<TC>() + 15) / 16 * 16;
}

template <typename TC, int M, int K>
constexpr size_t shape_smem() {
  return FusedShape<TC, M, BatchTile<M, K>::TX, BatchTile<M, K>::TY>::SMEM;
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

template <typename TC>
constexpr size_t batch_smem_bytes() {
  return cmax(cmax(cmax(shape_smem<TC, 2, 0>(), shape_smem<TC, 2, 1>()),
                   cmax(shape_smem<TC, 3, 0>(), shape_smem<TC, 3, 1>())),
              cmax(shape_smem<TC, 4, 0>(), shape_smem<TC, 4, 1>())) +
         batch_tables_bytes<TC>();
}

static_assert(shape_smem<float, 2, 1>() <= shape_smem<float, 3, 0>() &&
                  shape_smem<float, 3, 1>() <= shape_smem<float, 3, 0>() &&
                  shape_smem<float, 4, 1>() <= shape_smem<float, 3, 0>(),
              "the second shapes must not raise the batched kernel's shared memory");

template <typename TS, typename TC, int M, int K>
__device__ __forceinline__ void batch_tile(const BatchSim &sm, const BatchItem &it, const StepCoeffs<TC> &co,
                                           const PackedCoeffs *pc, TC *sX, int s) {
  constexpr int TX = BatchTile<M, K>::TX, TY = BatchTile<M, K>::TY;
  using Sh = FusedShape<TC, M, TX, TY>;
  Geom g;
  g.nx = sm.n[0];
  g.ny = sm.n[1];
  g.nz = sm.n[2];
  g.s = s;
  g.zlo = 0;
  g.zhi = g.nz;
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (it.tile % tiles_x) * TX, y0 = (it.tile / tiles_x) * TY;
  const int z0 = it.z0, z1 = min(it.z0 + sm.zchunk, g.nz);
  fused_tile<TS, TC, M, TX, TY, kBatchThreads, 2, kBatchPacked<TC>, kBatchPacked<TC>>(
      (const TS *)sm.in, (TS *)sm.out, g, x0, y0, z0, z1, co, sX, sX + Sh::SX, pc);
}

// The generic kernel calls each (order, shape) body as its own function:
// inlined into one kernel, six bodies share one register allocation and spill
// in the tile loops (892 B); the first-shape kernel inlines its three.
template <typename TS, typename TC, int M, int K>
__device__ __noinline__ void batch_tile_fn(const BatchSim &sm, const BatchItem &it, const StepCoeffs<TC> &co,
                                           const PackedCoeffs *pc, TC *sX, int s) {
  batch_tile<TS, TC, M, K>(sm, it, co, pc, sX, s);
}

// GENERIC = false: every order on its first tile shape (three inlined bodies;
// measured 7.00 ms per half step on the 64-simulation workload against 7.83 ms
// for the generic kernel with the same shapes).  GENERIC = true: any shape per
// order.
template <typename TS, typename TC, bool GENERIC>
__global__ void __launch_bounds__(kBatchThreads, HERMITE_BATCH_MIN_BLOCKS)
    batch_step_kernel(const BatchSim *__restrict__ sims, const unsigned char *__restrict__ coeffs,
                      const BatchItem *__restrict__ items, int nitems, int *__restrict__ counter, int s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StepCoeffs<TC> *sco = reinterpret_cast<StepCoeffs<TC> *>(smem_raw);
  const PackedCoeffs *spc =
      kBatchPacked<TC> ? reinterpret_cast<const PackedCoeffs *>(smem_raw + sizeof(StepCoeffs<TC>)) : nullptr;
  TC *sX = reinterpret_cast<TC *>(smem_raw + batch_tables_bytes<TC>());
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();  // also orders the previous tile's last reads before the copy below
    const int i = s_item;
    if (i >= nitems) break;
    const BatchItem it = items[i];
    const BatchSim sm = sims[it.sim];
    {  // the simulation's table record, in 8-byte words (both parts are multiples of 8 bytes)
      const unsigned long long *src =
          reinterpret_cast<const unsigned long long *>(coeffs + (size_t)it.sim * batch_record_bytes<TC>());
      unsigned long long *dst = reinterpret_cast<unsigned long long *>(smem_raw);
      for (int k = threadIdx.x; k < (int)(batch_record_bytes<TC>() / 8); k += kBatchThreads) dst[k] = src[k];
    }
    __syncthreads();
    if constexpr (GENERIC) {
      switch (sm.m * kBatchShapes + sm.shape) {
        case 1 * kBatchShapes + 0: batch_tile_fn<TS, TC, 2, 0>(sm, it, *sco, spc, sX, s); break;
        case 1 * kBatchShapes + 1: batch_tile_fn<TS, TC, 2, 1>(sm, it, *sco, spc, sX, s); break;
        case 2 * kBatchShapes + 0: batch_tile_fn<TS, TC, 3, 0>(sm, it, *sco, spc, sX, s); break;
        case 2 * kBatchShapes + 1: batch_tile_fn<TS, TC, 3, 1>(sm, it, *sco, spc, sX, s); break;
        case 3 * kBatchShapes + 0: batch_tile_fn<TS, TC, 4, 0>(sm, it, *sco, spc, sX, s); break;
        case 3 * kBatchShapes + 1: batch_tile_fn<TS, TC, 4, 1>(sm, it, *sco, spc, sX, s); break;
        default: break;  // the host builds only the pairs above
      }
    } else {
      switch (sm.m) {
        case 1: batch_tile<TS, TC, 2, 0>(sm, it, *sco, spc, sX, s); break;
        case 2: batch_tile<TS, TC, 3, 0>(sm, it, *sco, spc, sX, s); break;
        default: batch_tile<TS, TC, 4, 0>(sm, it, *sco, spc, sX, s); break;
      }
    }
    __syncthreads();  // every thread is done with sco, sX, sY and s_item
  }
}

template <typename TS, typename TC, bool GENERIC>
static SmemAttrOnce &batch_smem_once() {  // dynamic shared-memory limit raised, per device
  static SmemAttrOnce once;
  return once;
}

template <typename TS, typename TC, bool GENERIC>
static cudaError_t launch_batch_t(const BatchSim *sims, const void *coeffs, const BatchItem *items, int nitems,
                                  int *counter, int s, int grid, cudaStream_t st) {
  auto kern = batch_step_kernel<TS, TC, GENERIC>;
  constexpr size_t smem = batch_smem_bytes<TC>() + 16;
  cudaError_t e = raise_smem_limit(batch_smem_once<TS, TC, GENERIC>(), kern, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  kern<<<grid, kBatchThreads, smem, st>>>(sims, (const unsigned char *)coeffs, items, nitems, counter, s);
  return cudaGetLastError();
}

template <typename TS, typename TC, bool GENERIC>
static int occupancy_t() {
  int blocks = 0;
  constexpr size_t smem = batch_smem_bytes<TC>() + 16;
  auto kern = batch_step_kernel<TS, TC, GENERIC>;
  if (raise_smem_limit(batch_smem_once<TS, TC, GENERIC>(), kern, smem) != cudaSuccess) cudaGetLastError();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kBatchThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return blocks > 0 ? blocks : 1;
}

template <typename TS, typename TC>
static int occupancy_both() {  // both kernels take the same persistent grid
  const int a = occupancy_t<TS, TC, false>(), b = occupancy_t<TS, TC, true>();
  return a < b ? a : b;
}

int batch_blocks_per_sm(int compute, int state) {
  if (compute == kF64) return occupancy_both<double, double>();
  return state == kF64 ? occupancy_both<double, float>() : occupancy_both<float, float>();
}

template <bool GENERIC>
static cudaError_t launch_batch_g(int compute, int state, const BatchSim *sims, const void *coeffs,
                                  const BatchItem *items, int nitems, int *counter, int s, int grid,
                                  cudaStream_t st) {
  if (compute == kF64)
    return launch_batch_t<double, double, GENERIC>(sims, coeffs, items, nitems, counter, s, grid, st);
  if (state == kF64) return launch_batch_t<double, float, GENERIC>(sims, coeffs, items, nitems, counter, s, grid, st);
  return launch_batch_t<float, float, GENERIC>(sims, coeffs, items, nitems, counter, s, grid, st);
}

cudaError_t launch_batch(int compute, int state, bool generic, const BatchSim *sims, const void *coeffs,
                         const BatchItem *items, int nitems, int *counter, int s, int grid, cudaStream_t st) {
  return generic ? launch_batch_g<true>(compute, state, sims, coeffs, items, nitems, counter, s, grid, st)
                 : launch_batch_g<false>(compute, state, sims, coeffs, items, nitems, counter, s, grid, st);
}

}  // namespace hermite
