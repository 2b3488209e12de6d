// Internal definition of the opaque plan (shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/hermite.h"

#include "advect.h"
#include "hermite_impl.h"

namespace hermite {
struct BatchPlan;
void destroy_batch(BatchPlan *b);
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
}  // namespace hermite

struct hermite_plan_s {
  int m;
  int n[3];
  double h[3];
  double c, dt, tau;
  int prec, state, variant;
  size_t elems;
  double H[64];
  hermite::StepCoeffs<double> fwd, adj, dc;
  hermite::StepCoeffs<float> fwd32, adj32, dc32;
  hermite::HybridCoeffs hyb_fwd, hyb_adj, hyb_dc;
  hermite::TcBTable tc_fwd, tc_adj, tc_dc;  // tensor-core precisions: z-pass B operands
  hermite::RemCoeffs rem;                   // remainder-form precision: forward tables
  int *status = nullptr;                    // device status word of the tensor-core kernel
  hermite::DebugRecord *dbg = nullptr;      // debug build: record of the kernels' bounds checks
  size_t dbg_bound = 0;                     // debug self-test: bound handed to the kernels (0: elems)
  int drill = 0;                            // debug build: the next step is a bounded-wait drill
  hermite::InterpCoeffs<double> interp;
  hermite::EvolveParams evolve;
  int q = 4;                // Taylor stages of the local evolution (4 = RK4)
  int eq = 0;               // equation: 0 the scalar wave equation, 1 advection (Eq. 1)
  double a[3] = {0, 0, 0};  // advection velocity
  hermite::KronCoeffs<double> adv_fused, adv_interp;     // advection: 1-D factors (FP64)
  hermite::KronCoeffs<float> adv_fused32, adv_interp32;  // and their FP32 roundings
  hermite::AdvEvolveParams adv_ev;                       // advection: split evolution constants
  int tile;                 // fused kernel: index of the compiled tile shape
  int zchunk;               // fused kernel: cells per CTA along x3
  size_t ws_limit;          // split variant: workspace budget in bytes
  void *ws = nullptr;       // split workspace (device), grown on demand
  size_t ws_bytes = 0;
  void *stage[2] = {nullptr, nullptr};  // host-buffer steps: device copies of in / out
  double *red = nullptr;    // error reduction scratch (device)
  double *red_host = nullptr;  // pinned result
  hermite::BatchPlan *batch = nullptr;  // set for batched plans (hermite_batch_plan)
  cudaStream_t copy_in = nullptr, copy_out = nullptr;  // host-buffer steps: copy streams
  cudaEvent_t ev[2 * 16 + 2] = {};                     // host-buffer steps: chunk events
};

namespace hermite {

// Argument checks on state buffers, shared by every entry point that takes
// them, so that a host pointer never reaches a kernel.

inline size_t state_bytes(const hermite_plan_s *p) {
  return p->elems * (p->state == HERMITE_STATE_FP64 ? sizeof(double) : sizeof(float));
}

enum PtrKind { kHostPtr, kDevicePtr, kBadPtr };

// Where a pointer lives: device (or managed) memory, host memory (pageable
// or pinned), or unknown to the runtime (no device, or the query failed).
inline PtrKind classify(const void *ptr) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return kBadPtr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return kDevicePtr;
  return kHostPtr;
}

inline bool overlaps(const void *a, const void *b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

// Non-null, non-overlapping, 16-byte aligned (EINVAL otherwise).
inline int check_device_pair(const hermite_plan_s *p, const void *in, void *out) {
  if (!in || !out) return fail(HERMITE_EINVAL, "null state pointer");
  if (overlaps(in, out, state_bytes(p)))
    return fail(HERMITE_EINVAL, "input and output states overlap (a half step is not in place)");
  if (((uintptr_t)in | (uintptr_t)out) & 15u)
    return fail(HERMITE_EINVAL, "device state pointers must be 16-byte aligned");
  return HERMITE_OK;
}

// check_device_pair, and both buffers in device memory (EINVAL for host
// buffers, ECUDA when the runtime cannot tell).  `what` names the call.
// Tensor-core precisions (the z-pass on tcgen05).
inline bool is_tc_prec(int prec) { return prec == HERMITE_3XTF32 || prec == HERMITE_SPLITBF16; }

inline int check_device_only(const hermite_plan_s *p, const void *in, void *out, const char *what) {
  if (int rc = check_device_pair(p, in, out)) return rc;
  const PtrKind ki = classify(in), ko = classify(out);
  if (ki == kBadPtr || ko == kBadPtr) return fail(HERMITE_ECUDA, "cannot query pointer attributes (no CUDA device?)");
  if (ki != kDevicePtr || ko != kDevicePtr) return fail(HERMITE_EINVAL, "%s takes device buffers", what);
  return HERMITE_OK;
}

}  // namespace hermite
