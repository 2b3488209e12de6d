// C ABI of the batched half step (include/hermite.h): batched plans, their
// work lists, per-buffer-set descriptor arrays and CUDA-graph runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hermite.h"
#include "batch.h"
#include "hermite_impl.h"
#include "plan.h"

namespace hermite {

struct DescSet {                // device BatchSim array for one (in[], out[]) pointer set
  std::vector<const void *> in;
  std::vector<void *> out;
  BatchSim *dev = nullptr;
};

struct GraphRun {               // an instantiated graph of nhalf batched half steps
  int nhalf;
  BatchSim *a, *b;
  cudaGraphExec_t exec = nullptr;
};

struct BatchPlan {
  int nsims, prec, state, compute;
  std::vector<int> m, zc;       // per simulation: order, z-chunk
  std::vector<int> n;           // 3 per simulation
  std::vector<size_t> elems;
  int zchunk[4] = {0, 16, 16, 16};  // per order
  int shape[4] = {0, 0, 0, 0};      // tile shape index per order (batch_tile_shape)
  void *coeffs = nullptr;       // device table records, one per simulation (batch_write_record)
  BatchItem *items = nullptr;   // device work list
  int nitems = 0;
  int *counter = nullptr;
  int grid = 0;                 // resident CTAs of the persistent launch
  std::vector<DescSet> sets;
  std::vector<GraphRun> graphs;
  cudaStream_t capture = nullptr;
};

void destroy_batch(BatchPlan *b) {
  if (!b) return;
  for (auto &g : b->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto &s : b->sets)
    if (s.dev) cudaFree(s.dev);
  if (b->coeffs) cudaFree(b->coeffs);
  if (b->items) cudaFree(b->items);
  if (b->counter) cudaFree(b->counter);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

namespace {

void clear_graphs(BatchPlan *b) {
  for (auto &g : b->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

// Work list: every (sim, xy-tile, z-chunk) block, heaviest order first so that
// the atomic scheduler hands out the long items early.
int build_items(BatchPlan *b) {
  std::vector<BatchItem> items;
  for (int order = 3; order >= 1; --order)
    for (int i = 0; i < b->nsims; ++i) {
      if (b->m[i] != order) continue;
      int tx, ty;
      batch_tile_shape(order, b->shape[order], &tx, &ty);
      const int *n = &b->n[3 * i];
      const int tiles = ((n[0] + tx - 1) / tx) * ((n[1] + ty - 1) / ty);
      b->zc[i] = b->zchunk[order];
      for (int z0 = 0; z0 < n[2]; z0 += b->zc[i])
        for (int t = 0; t < tiles; ++t) items.push_back(BatchItem{i, t, z0, 0});
    }
  if (b->items) cudaFree(b->items);
  b->items = nullptr;
  cudaError_t e = dev_malloc((void **)&b->items, sizeof(BatchItem) * items.size());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HERMITE_ENOMEM, "batched work list");
  }
  e = cudaMemcpy(b->items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "work list upload");
  b->nitems = (int)items.size();
  for (auto &s : b->sets) {  // z-chunks live in the descriptors too
    if (s.dev) cudaFree(s.dev);
    s.dev = nullptr;
  }
  b->sets.clear();
  clear_graphs(b);
  return HERMITE_OK;
}

int get_set(BatchPlan *b, const void *const *in, void *const *out, BatchSim **dev) {
  for (auto &s : b->sets)
    if (std::equal(s.in.begin(), s.in.end(), in) && std::equal(s.out.begin(), s.out.end(), out)) {
      *dev = s.dev;
      return HERMITE_OK;
    }
  std::vector<BatchSim> host(b->nsims);
  for (int i = 0; i < b->nsims; ++i) {
    if (!in[i] || !out[i]) return fail(HERMITE_EINVAL, "null state pointer of simulation %d", i);
    const size_t bytes = b->elems[i] * (b->state == HERMITE_STATE_FP64 ? 8 : 4);
    const uintptr_t x = (uintptr_t)in[i], y = (uintptr_t)out[i];
    if (x < y + bytes && y < x + bytes) return fail(HERMITE_EINVAL, "in and out of simulation %d overlap", i);
    if ((x | y) & 15u) return fail(HERMITE_EINVAL, "state pointers of simulation %d not 16-byte aligned", i);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, in[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
        cudaPointerGetAttributes(&a, out[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return fail(HERMITE_EINVAL, "states of simulation %d must be device memory", i);
    }
    host[i] = BatchSim{in[i], out[i], {b->n[3 * i], b->n[3 * i + 1], b->n[3 * i + 2]}, b->m[i], b->zc[i],
                       b->shape[b->m[i]]};
  }
  DescSet s;
  s.in.assign(in, in + b->nsims);
  s.out.assign(out, out + b->nsims);
  cudaError_t e = dev_malloc((void **)&s.dev, sizeof(BatchSim) * b->nsims);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HERMITE_ENOMEM, "batch descriptors");
  }
  e = cudaMemcpy(s.dev, host.data(), sizeof(BatchSim) * b->nsims, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
  b->sets.push_back(s);
  *dev = s.dev;
  return HERMITE_OK;
}

int launch(BatchPlan *b, BatchSim *d, int parity, cudaStream_t st) {
  const bool generic = b->shape[1] != 0 || b->shape[2] != 0 || b->shape[3] != 0;
  const cudaError_t e = launch_batch(b->compute, b->state == HERMITE_STATE_FP64 ? kF64 : kF32, generic, d, b->coeffs,
                                     b->items, b->nitems, b->counter, parity == 0 ? 0 : -1, b->grid, st);
  return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "batched half-step launch");
}

}  // namespace
}  // namespace hermite

using namespace hermite;

extern "C" {

int hermite_batch_plan(hermite_plan_t *out, int nsims, const int *m, const int *grid, const double *h,
                       const double *c, const double *dt, int prec, int state_dtype) {
  if (!out) return fail(HERMITE_EINVAL, "out is NULL");
  *out = nullptr;
  if (nsims < 1 || nsims > (1 << 16)) return fail(HERMITE_EINVAL, "nsims = %d out of range", nsims);
  if (!m || !grid || !h || !c || !dt) return fail(HERMITE_EINVAL, "null array argument");
  if (prec != HERMITE_FP64 && prec != HERMITE_FP32)
    return fail(HERMITE_EUNSUPPORTED, "batched plans take FP64 or FP32 arithmetic, not %d", prec);
  if (state_dtype != HERMITE_STATE_FP64 && state_dtype != HERMITE_STATE_FP32)
    return fail(HERMITE_EINVAL, "state type %d unknown", state_dtype);
  if (prec == HERMITE_FP64 && state_dtype != HERMITE_STATE_FP64)
    return fail(HERMITE_EUNSUPPORTED, "FP64 arithmetic needs an FP64 state");
  // every simulation must also be a valid single plan (same checks)
  for (int i = 0; i < nsims; ++i) {
    hermite_plan_t probe = nullptr;
    int rc = hermite_plan(&probe, m[i], grid + 3 * i, h + 3 * i, c[i], dt[i], prec, state_dtype, HERMITE_FUSED);
    if (rc) return rc;
    hermite_destroy(probe);
  }
  hermite_plan_s *p = host_new<hermite_plan_s>();
  BatchPlan *b = host_new<BatchPlan>();
  if (!p || !b) {
    delete p;
    delete b;
    return fail(HERMITE_ENOMEM, "batched plan allocation");
  }
  p->batch = b;
  p->m = 0;
  p->prec = prec;
  p->state = state_dtype;
  b->nsims = nsims;
  b->prec = prec;
  b->state = state_dtype;
  b->compute = prec == HERMITE_FP64 ? kF64 : kF32;
  b->m.assign(m, m + nsims);
  b->n.assign(grid, grid + 3 * nsims);
  b->zc.assign(nsims, 16);
  const size_t csize = batch_coeff_record_bytes(b->compute);
  std::vector<unsigned char> host(csize * nsims);
  for (int i = 0; i < nsims; ++i) {
    b->elems.push_back((size_t)2 * (m[i] + 1) * (m[i] + 1) * (m[i] + 1) * grid[3 * i] * grid[3 * i + 1] *
                       grid[3 * i + 2]);
    StepCoeffs<double> cd;
    build_step_coeffs(m[i], h + 3 * i, c[i], 0.5 * dt[i], kForward, 4, &cd);
    batch_write_record(b->compute, cd, host.data() + csize * i);
  }
  cudaError_t e = dev_malloc((void **)&b->coeffs, host.size());
  if (e == cudaSuccess) e = cudaMemcpy(b->coeffs, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dev_malloc((void **)&b->counter, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    hermite_destroy(p);
    return cuda_fail(e, "batched plan set-up");
  }
  b->grid = sms * batch_blocks_per_sm(b->compute, state_dtype == HERMITE_STATE_FP64 ? kF64 : kF32);
  int rc = build_items(b);
  if (rc) {
    hermite_destroy(p);
    return rc;
  }
  *out = p;
  return HERMITE_OK;
}

size_t hermite_batch_elems(hermite_plan_t p, int sim) {
  if (!p || !p->batch || sim < 0 || sim >= p->batch->nsims) return 0;
  return p->batch->elems[sim];
}

int hermite_batch_set_schedule(hermite_plan_t p, const int zchunk[3]) {
  if (!p || !p->batch || !zchunk) return fail(HERMITE_EINVAL, "not a batched plan");
  for (int k = 0; k < 3; ++k)
    if (zchunk[k] < 1 || zchunk[k] > 4096) return fail(HERMITE_EINVAL, "zchunk[%d] = %d out of range", k, zchunk[k]);
  for (int k = 0; k < 3; ++k) p->batch->zchunk[k + 1] = zchunk[k];
  return build_items(p->batch);
}

int hermite_batch_set_tiles(hermite_plan_t p, const int tile[3]) {
  if (!p || !p->batch || !tile) return fail(HERMITE_EINVAL, "not a batched plan");
  for (int k = 0; k < 3; ++k)
    if (tile[k] < 0 || tile[k] >= kBatchShapes)
      return fail(HERMITE_EINVAL, "tile[%d] = %d out of range [0, %d)", k, tile[k], kBatchShapes);
  for (int k = 0; k < 3; ++k) p->batch->shape[k + 1] = tile[k];
  return build_items(p->batch);
}

int hermite_batch_tile_shape(int m, int tile, int *tx, int *ty) {
  if (m < 1 || m > 3 || tile < 0 || tile >= kBatchShapes || !tx || !ty)
    return fail(HERMITE_EINVAL, "no batched tile shape %d for order %d", tile, m);
  batch_tile_shape(m, tile, tx, ty);
  return HERMITE_OK;
}

int hermite_batch_step(hermite_plan_t p, const void *const *in, void *const *out, int parity, void *stream) {
  if (!p || !p->batch) return fail(HERMITE_EINVAL, "not a batched plan");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (!in || !out) return fail(HERMITE_EINVAL, "null pointer array");
  BatchSim *d = nullptr;
  int rc = get_set(p->batch, in, out, &d);
  if (rc) return rc;
  return launch(p->batch, d, parity, (cudaStream_t)stream);
}

int hermite_batch_run(hermite_plan_t p, void *const *a, void *const *bb, int nhalf, void *stream) {
  if (!p || !p->batch) return fail(HERMITE_EINVAL, "not a batched plan");
  if (nhalf < 1) return fail(HERMITE_EINVAL, "nhalf must be positive");
  if (!a || !bb) return fail(HERMITE_EINVAL, "null pointer array");
  BatchPlan *b = p->batch;
  BatchSim *dab = nullptr, *dba = nullptr;
  int rc = get_set(b, (const void *const *)a, bb, &dab);
  if (rc) return rc;
  rc = get_set(b, (const void *const *)bb, a, &dba);
  if (rc) return rc;
  GraphRun *run = nullptr;
  for (auto &g : b->graphs)
    if (g.nhalf == nhalf && g.a == dab && g.b == dba) run = &g;
  if (!run) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int lrc = HERMITE_OK;
    for (int k = 0; k < nhalf && lrc == HERMITE_OK; ++k) lrc = launch(b, k % 2 ? dba : dab, k % 2, b->capture);
    e = cudaStreamEndCapture(b->capture, &graph);
    if (lrc) {
      if (graph) cudaGraphDestroy(graph);
      return lrc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graphs.push_back(GraphRun{nhalf, dab, dba, exec});
    run = &b->graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(run->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "graph launch");
}

}  // extern "C"
