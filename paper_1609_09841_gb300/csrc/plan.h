// Internal definition of the opaque plan (shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <string>

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
