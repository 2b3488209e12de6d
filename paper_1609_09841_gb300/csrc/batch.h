// Device-side descriptors of the batched half step.
#pragma once

#include <cuda_runtime.h>

#include "hermite_impl.h"

namespace hermite {

struct BatchSim {      // one simulation of a batch, as the kernel sees it
  const void *in;      // input state (plan's state type)
  void *out;           // output state
  int n[3];            // nodes along x1, x2, x3
  int m;               // order
  int zchunk;          // cells per work item along x3
  int shape;           // tile shape index of this order, 0 .. kBatchShapes-1
};

struct BatchItem {     // one unit of work: a TX x TY x zchunk block of one simulation
  int sim;
  int tile;            // xy-tile index (x fastest)
  int z0;              // first output z layer
  int pad;
};

constexpr int kBatchShapes = 2;  // tile shapes compiled per order
void batch_tile_shape(int m, int shape, int *tx, int *ty);
// One simulation's table record as the kernel reads it (compute kF32:
// StepCoeffs<float> then its PackedCoeffs; kF64: StepCoeffs<double>).
size_t batch_coeff_record_bytes(int compute);
void batch_write_record(int compute, const StepCoeffs<double> &cd, unsigned char *dst);
int batch_blocks_per_sm(int compute, int state);
// generic = false: every order on tile shape 0 (the kernel with those bodies
// inlined); true: the kernel that takes any shape per order.
cudaError_t launch_batch(int compute, int state, bool generic, const BatchSim *sims, const void *coeffs,
                         const BatchItem *items, int nitems, int *counter, int s, int grid, cudaStream_t st);

}  // namespace hermite
