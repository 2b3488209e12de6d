// Allocation-free variant of the split half step.
//
// Some callers cannot call cudaMalloc: code that runs while another library
// owns the device memory (a framework's caching allocator or a fixed memory
// budget), code that must not pay allocation latency or risk fragmentation in
// a time-critical loop, or code that only enqueues work into a stream it did
// not create.  hermite_step_split_static serves them: it runs the same two
// kernels as the split variant of hermite_step, but its workspace is the
// file-scope device array below instead of plan-owned memory, and it calls
// no allocating routine.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/hermite.h"
#include "hermite_impl.h"
#include "plan.h"

namespace hermite {
namespace {

constexpr size_t kStaticBytes = HERMITE_STATIC_WORKSPACE_BYTES;

// Workspace of the interpolation kernel (Ru of one z-slab of cells).  Every
// GPU that loads the library holds it until the process exits.  Host code
// must not use the symbol as a device address: it is translated per device
// with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_split_ws[kStaticBytes];

std::atomic<void *> g_ws_addr[kMaxDevices];
std::mutex g_ws_mutex;

// Device address of g_split_ws on the current device, looked up once per
// device (the first call on a device does it; that call must not be inside
// a stream capture).
int workspace_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(HERMITE_EUNSUPPORTED, "device ordinal %d above %d", dev, kMaxDevices);
  void *p = g_ws_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    p = g_ws_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
      e = cudaGetSymbolAddress(&p, g_split_ws);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static workspace");
      g_ws_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return HERMITE_OK;
}

}  // namespace
}  // namespace hermite

using namespace hermite;

extern "C" {

size_t hermite_static_workspace_bytes(void) { return kStaticBytes; }

int hermite_step_split_static(hermite_plan_t p, const void *in, void *out, int parity, void *stream) {
  if (!p || p->batch) return fail(HERMITE_EINVAL, "plan is NULL or batched");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "the allocation-free step is for wave-equation plans");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (p->prec != HERMITE_FP64 && p->prec != HERMITE_FP32)
    return fail(HERMITE_EUNSUPPORTED, "the split kernels have no hybrid precision");
  if (int rc = check_device_only(p, in, out, "hermite_step_split_static")) return rc;
  const int P = 2 * p->m + 2;
  const size_t elt = p->prec == HERMITE_FP64 ? sizeof(double) : sizeof(float);
  const size_t per_layer = (size_t)2 * P * P * P * p->n[0] * p->n[1] * elt;
  if (per_layer > kStaticBytes)
    return fail(HERMITE_EINVAL,
                "one z-layer of cell polynomials needs %zu bytes, above the %zu-byte static workspace "
                "(use hermite_step, which allocates)",
                per_layer, kStaticBytes);
  void *ws = nullptr;
  int rc = workspace_address(&ws);
  if (rc) return rc;
  const int nzl = (int)(kStaticBytes / per_layer < (size_t)p->n[2] ? kStaticBytes / per_layer : (size_t)p->n[2]);
  Geom g;
  g.nx = p->n[0];
  g.ny = p->n[1];
  g.nz = p->n[2];
  g.s = parity == 0 ? 0 : -1;
  g.zlo = 0;
  g.zhi = g.nz;
  const int compute = p->prec == HERMITE_FP64 ? kF64 : kF32;
  const int state = p->state == HERMITE_STATE_FP64 ? kF64 : kF32;
  cudaStream_t st = (cudaStream_t)stream;
  for (int z0 = 0; z0 < p->n[2]; z0 += nzl) {
    const int nl = nzl < p->n[2] - z0 ? nzl : p->n[2] - z0;
    cudaError_t e = launch_interp(p->m, state, compute, in, ws, g, z0, nl, p->interp, st);
    if (e != cudaSuccess) return cuda_fail(e, "interpolation kernel launch");
    e = launch_evolve(p->m, state, compute, ws, out, g, z0, nl, p->evolve, st);
    if (e != cudaSuccess) return cuda_fail(e, "evolution kernel launch");
  }
  return HERMITE_OK;
}

}  // extern "C"
