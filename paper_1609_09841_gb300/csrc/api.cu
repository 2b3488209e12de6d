// C ABI of libhermite (include/hermite.h): plans, argument checks, dispatch to
// the fused or split kernels, host-buffer staging and the error norms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/hermite.h"
#include "hermite_impl.h"
#include "plan.h"

using namespace hermite;


namespace hermite {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  const int code = e == cudaErrorMemoryAllocation ? HERMITE_ENOMEM : HERMITE_ECUDA;
  return fail(code, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Injection window of the allocation gate: after g_alloc_skip more
// allocations succeed, the next g_alloc_fail ones fail.
std::atomic<long long> g_alloc_skip{0}, g_alloc_fail{0};

bool alloc_injected_failure() {
  if (g_alloc_fail.load(std::memory_order_relaxed) <= 0) return false;
  if (g_alloc_skip.fetch_sub(1, std::memory_order_relaxed) > 0) return false;
  return g_alloc_fail.fetch_sub(1, std::memory_order_relaxed) > 0;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
  if (alloc_injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t host_malloc_pinned(void **p, size_t bytes) {
  if (alloc_injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

}  // namespace hermite

namespace {

// Largest x1-x2 plane of a plan: the kernels index nodes within a plane with
// 32-bit offsets (plane offsets and field strides are 64-bit).
constexpr long long kMaxPlaneNodes = (1LL << 31) - 1;

// Stability limit of c*tau/h per order m and Taylor order q: the first step
// at which the largest spectral radius of the Fourier symbol of the isotropic
// half step, over a 7^3 grid of theta in [0, pi]^3, exceeds 1 + 1e-10
// (hermite_max_radius scanned in steps of 0.0025, then bisected to 1e-4),
// rounded down to two decimals.  q = 4 is RK4.  The limit is not monotone in
// q (m = 3 with q = 5 is stable only up to 0.09), and at m = 3 the stable
// steps do not form an interval: for q >= 9 the symbol is weakly unstable
// from 0.373 to about 0.39 and stable again at 0.40, so the entry is 0.37.
constexpr int kMaxQ = 21;
const double kStabilityLimit[4][kMaxQ + 1] = {
    {0},
    {0, 0, 0, 0, 0.45, 0.47, 0.47, 0.47, 0.47, 0.47},
    {0, 0, 0, 0, 0.30, 0.34, 0.38, 0.36, 0.41, 0.42, 0.42, 0.42, 0.42, 0.42, 0.42, 0.42},
    {0, 0, 0, 0, 0.26, 0.09, 0.20, 0.24, 0.33, 0.37, 0.37, 0.37, 0.37, 0.37, 0.37, 0.37, 0.37, 0.37, 0.37,
     0.37, 0.37, 0.37},
};

double limit_of(int m, int q) {
  return (m >= 1 && m <= 3 && q >= 4 && q <= 3 * (2 * m + 1)) ? kStabilityLimit[m][q] : 0.0;
}

int check_stable(int m, int q, double c, double tau, const double h[3]) {
  for (int k = 0; k < 3; ++k) {
    const double lam = c * tau / h[k];
    if (lam > limit_of(m, q) * (1.0 + 1e-12))
      return fail(HERMITE_EUNSTABLE, "c*(dt/2)/h[%d] = %.6g above the stability limit %.3g of order %d, q = %d", k,
                  lam, limit_of(m, q), m, q);
  }
  return HERMITE_OK;
}

Geom geom_of(const hermite_plan_s *p, int s) {
  Geom g;
  g.nx = p->n[0];
  g.ny = p->n[1];
  g.nz = p->n[2];
  g.s = s;
  g.zlo = 0;
  g.zhi = g.nz;
  g.elems = p->dbg_bound ? p->dbg_bound : p->elems;
  g.dbg = p->dbg;
  g.drill = p->drill;
  return g;
}

// Debug build: the record of the kernels' bounds checks, allocated by the
// first step of a plan (zero flags, no offending offset).
int ensure_dbg(hermite_plan_s *p) {
  if (!kDebugBuild || p->dbg) return HERMITE_OK;
  cudaError_t e = dev_malloc((void **)&p->dbg, sizeof(DebugRecord));
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->dbg = nullptr;
    return fail(HERMITE_ENOMEM, "debug record");
  }
  const DebugRecord init{0, 0, ~0ull};
  e = cudaMemcpy(p->dbg, &init, sizeof init, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "debug record");
}

int ensure_ws(hermite_plan_s *p, size_t bytes) {
  if (p->ws_bytes >= bytes) return HERMITE_OK;
  if (p->ws) cudaFree(p->ws);
  p->ws = nullptr;
  p->ws_bytes = 0;
  cudaError_t e = dev_malloc(&p->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HERMITE_ENOMEM, "split workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  p->ws_bytes = bytes;
  return HERMITE_OK;
}

// Reduction scratch: (error_blocks() + 1) * 8 doubles on the device (result
// first, then the per-CTA partials) and an 8-double pinned result buffer.
int ensure_red(hermite_plan_s *p) {
  if (p->red && p->red_host) return HERMITE_OK;
  if (!p->red) {
    cudaError_t e = dev_malloc((void **)&p->red, sizeof(double) * (size_t)(error_blocks() + 1) * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p->red = nullptr;
      return fail(HERMITE_ENOMEM, "reduction scratch");
    }
  }
  cudaError_t e = host_malloc_pinned((void **)&p->red_host, sizeof(double) * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->red_host = nullptr;
    return fail(HERMITE_ENOMEM, "pinned result buffer");
  }
  return HERMITE_OK;
}

// Advection (Eq. 1 with a constant velocity a): largest max_k |a_k| tau / h_k
// per order m and Taylor order q, the smaller of the limits of the Fourier
// symbol for a mode along x1 (a along x1) and for the diagonal (a = (1, 1, 1)
// direction, 7^3 theta grid), rounded down to two decimals; every entry is at
// or below the first instability found by hermite_adv_max_radius on a 0.0025
// scan (no unstable window lies below an entry).  With the whole
// series (q = 3(2m+1)) the half step is a Kronecker product of 1-D maps and the
// limit is the half cell of Sec. 2; q = 1 (forward Euler) has no stable step.
const double kAdvLimit[4][kMaxQ + 1] = {
    {0},
    {0, 0.01, 0.16, 0.25, 0.31, 0.37, 0.42, 0.45, 0.48, 0.50},
    {0, 0.00, 0.03, 0.15, 0.20, 0.18, 0.23, 0.26, 0.29, 0.34, 0.38, 0.41, 0.46, 0.48, 0.49, 0.50},
    {0, 0.00, 0.00, 0.10, 0.14, 0.05, 0.13, 0.16, 0.19, 0.23, 0.26, 0.28, 0.29, 0.32, 0.35, 0.39,
     0.41, 0.44, 0.47, 0.49, 0.49, 0.50},
};

double adv_limit_of(int m, int q) {
  return (m >= 1 && m <= 3 && q >= 1 && q <= 3 * (2 * m + 1)) ? kAdvLimit[m][q] : 0.0;
}

// Advection half step: the fused Kronecker kernel (whole series), or the
// split pair (interpolation to the workspace, Alg. 4) z-slab by z-slab.
int run_adv_step(hermite_plan_s *p, const void *in, void *out, int parity, cudaStream_t st, int zlo, int zhi) {
  Geom g = geom_of(p, parity == 0 ? 0 : -1);
  if (zhi >= 0) {
    g.zlo = zlo;
    g.zhi = zhi;
  }
  const int compute = p->prec == HERMITE_FP64 ? kF64 : kF32;
  const int state = p->state == HERMITE_STATE_FP64 ? kF64 : kF32;
  cudaError_t e;
  if (p->variant != HERMITE_SPLIT) {
    e = launch_adv_fused(p->m, p->tile, state, compute, in, out, g, p->adv_fused, p->adv_fused32, p->zchunk, st);
    return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "advection half-step launch");
  }
  const int P = 2 * p->m + 2;
  const size_t elt = compute == kF64 ? sizeof(double) : sizeof(float);
  const size_t per_layer = (size_t)P * P * P * p->n[0] * p->n[1] * elt;
  const int nzl = (int)std::max<size_t>(1, std::min<size_t>((size_t)(g.zhi - g.zlo), p->ws_limit / per_layer));
  int rc = ensure_ws(p, per_layer * nzl);
  if (rc) return rc;
  for (int z0 = g.zlo; z0 < g.zhi; z0 += nzl) {
    const int nl = std::min(nzl, g.zhi - z0);
    e = launch_adv_interp(p->m, state, compute, in, p->ws, g, z0, nl, p->adv_interp, p->adv_interp32, st);
    if (e != cudaSuccess) return cuda_fail(e, "advection interpolation launch");
    e = launch_adv_evolve(p->m, state, compute, p->ws, out, g, z0, nl, p->adv_ev, st);
    if (e != cudaSuccess) return cuda_fail(e, "advection evolution launch");
  }
  return HERMITE_OK;
}

// Device-pointer half step of either direction (adjoint: transposed tables,
// mirrored corner offset).
// The plan's device status word (time-outs of bounded device waits), made on
// first use and read back by hermite_device_status.
int ensure_status(hermite_plan_s *p) {
  if (p->status) return HERMITE_OK;
  cudaError_t e = dev_malloc((void **)&p->status, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->status = nullptr;
    return fail(HERMITE_ENOMEM, "device status word");
  }
  e = cudaMemset(p->status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "device status word");
  return HERMITE_OK;
}

int run_step(hermite_plan_s *p, const void *in, void *out, int parity, int mode, cudaStream_t st, int zlo = 0,
             int zhi = -1) {
  if (int rc = ensure_dbg(p)) return rc;
  if (p->eq == 1) return run_adv_step(p, in, out, parity, st, zlo, zhi);
  const int s_fwd = parity == 0 ? 0 : -1;
  const bool adjoint = mode == kAdjoint;
  const int s = adjoint ? -s_fwd - 1 : s_fwd;
  Geom g = geom_of(p, s);
  if (zhi >= 0) {
    g.zlo = zlo;
    g.zhi = zhi;
  }
  const bool split = p->variant == HERMITE_SPLIT && mode == kForward;
  cudaError_t e = cudaSuccess;
  if (!split) {
    if (p->prec == HERMITE_HYBRID64 || p->prec == HERMITE_HYBRIDDF) {
      const HybridCoeffs &ch = mode == kAdjoint ? p->hyb_adj : (mode == kDc ? p->hyb_dc : p->hyb_fwd);
      e = launch_hybrid(p->prec == HERMITE_HYBRID64 ? 0 : 1, p->m, p->tile, (const double *)in, (double *)out, g, ch,
                        p->zchunk, st);
      if (e != cudaSuccess) return cuda_fail(e, "hybrid half-step launch");
      return HERMITE_OK;
    }
    const StepCoeffs<double> &cd = mode == kAdjoint ? p->adj : (mode == kDc ? p->dc : p->fwd);
    const StepCoeffs<float> &cf = mode == kAdjoint ? p->adj32 : (mode == kDc ? p->dc32 : p->fwd32);
    if (p->prec == HERMITE_REMAINDER) {
      if (mode != kForward) return fail(HERMITE_EUNSUPPORTED, "the remainder-form precision has forward steps only");
      e = launch_remainder(p->m, p->tile, (const double *)in, (double *)out, g, p->rem, p->zchunk, st);
      if (e != cudaSuccess) return cuda_fail(e, "remainder-form half-step launch");
      return HERMITE_OK;
    }
    if (is_tc_prec(p->prec)) {
      if (int rc = ensure_status(p)) return rc;
      const TcBTable &bt = mode == kAdjoint ? p->tc_adj : (mode == kDc ? p->tc_dc : p->tc_fwd);
      e = launch_fused_tc(p->prec == HERMITE_3XTF32 ? 0 : 1, p->m, p->state == HERMITE_STATE_FP64 ? kF64 : kF32, in,
                          out, g, cf, bt, p->zchunk, p->status, st);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core half-step launch");
      return HERMITE_OK;
    }
    const bool rk4 = p->q == 4;  // longer series run the kernels with more grades
    if (p->prec == HERMITE_FP64)
      e = rk4 ? launch_fused_f64(p->m, p->tile, (const double *)in, (double *)out, g, cd, p->zchunk, st)
              : launch_fused_f64_fullq(p->m, (const double *)in, (double *)out, g, cd, p->zchunk, st);
    else {
      if (rk4 && p->tile >= kFirstStagedTile)
        if (int rc = ensure_status(p)) return rc;
      if (p->state == HERMITE_STATE_FP64)
        e = rk4 ? launch_fused_f32_s64(p->m, p->tile, (const double *)in, (double *)out, g, cf, p->zchunk, p->status,
                                       st)
                : launch_fused_f32_fullq(p->m, kF64, in, out, g, cf, p->zchunk, st);
      else
        e = rk4 ? launch_fused_f32_s32(p->m, p->tile, (const float *)in, (float *)out, g, cf, p->zchunk, p->status,
                                       st)
                : launch_fused_f32_fullq(p->m, kF32, in, out, g, cf, p->zchunk, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fused half-step launch");
    return HERMITE_OK;
  }
  // Split pair, z-slab by z-slab so that the workspace stays within budget.
  const int P = 2 * p->m + 2;
  const size_t elt = p->prec == HERMITE_FP64 ? sizeof(double) : sizeof(float);
  const size_t per_layer = (size_t)2 * P * P * P * p->n[0] * p->n[1] * elt;
  int nzl = (int)std::max<size_t>(1, std::min<size_t>((size_t)p->n[2], p->ws_limit / per_layer));
  int rc = ensure_ws(p, per_layer * nzl);
  if (rc) return rc;
  const int compute = p->prec == HERMITE_FP64 ? kF64 : kF32;
  const int state = p->state == HERMITE_STATE_FP64 ? kF64 : kF32;
  for (int z0 = 0; z0 < p->n[2]; z0 += nzl) {
    const int nl = std::min(nzl, p->n[2] - z0);
    e = launch_interp(p->m, state, compute, in, p->ws, g, z0, nl, p->interp, st);
    if (e != cudaSuccess) return cuda_fail(e, "interpolation kernel launch");
    e = launch_evolve(p->m, state, compute, p->ws, out, g, z0, nl, p->evolve, st);
    if (e != cudaSuccess) return cuda_fail(e, "evolution kernel launch");
  }
  return HERMITE_OK;
}

// z planes [a, b) (wrapping modulo nz) of every component, between a host and
// a device state: one strided copy per contiguous run.
int copy_planes(hermite_plan_s *p, void *dst, const void *src, int a, int b, cudaMemcpyKind kind,
                cudaStream_t st) {
  const int nz = p->n[2];
  const size_t elt = p->state == HERMITE_STATE_FP64 ? sizeof(double) : sizeof(float);
  const size_t pxy = (size_t)p->n[0] * p->n[1] * elt, plane = pxy * nz;
  const size_t ncomp = p->elems / ((size_t)p->n[0] * p->n[1] * nz);
  while (a < b) {
    const int za = ((a % nz) + nz) % nz;
    const int len = std::min(b - a, nz - za);
    cudaError_t e = cudaMemcpy2DAsync((char *)dst + za * pxy, plane, (const char *)src + za * pxy, plane, len * pxy,
                                      ncomp, kind, st);
    if (e != cudaSuccess) return cuda_fail(e, "state slab copy");
    a += len;
  }
  return HERMITE_OK;
}

// Host-buffer half step, pipelined over z-slabs: the copy of slab k+1 in, the
// half step of slab k and the copy of slab k-1 out overlap on three streams.
// Output layers [zb_k, zb_k+1) read input planes zb_k + s .. zb_k+1 + s, i.e.
// slab k's planes and the first plane of slab k+1.
int host_step(hermite_plan_s *p, const void *in, void *out, int parity, cudaStream_t st) {
  const size_t bytes = state_bytes(p);
  if (overlaps(in, out, bytes)) return fail(HERMITE_EINVAL, "input and output states overlap");
  for (int k = 0; k < 2; ++k)
    if (!p->stage[k]) {
      cudaError_t e = dev_malloc(&p->stage[k], bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        p->stage[k] = nullptr;
        return fail(HERMITE_ENOMEM, "staging buffer of %zu bytes", bytes);
      }
    }
  if (!p->copy_in) {
    cudaError_t e = cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->copy_out, cudaStreamNonBlocking);
    for (auto &ev : p->ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "copy streams");
  }
  const int nz = p->n[2];
  const int K = p->variant == HERMITE_SPLIT ? 1 : std::min(nz, 16);
  const int s = parity == 0 ? 0 : -1;
  cudaEvent_t *ein = p->ev, *eout = p->ev + 16, start = p->ev[32], done = p->ev[33];
  cudaError_t e = cudaEventRecord(start, st);  // order after earlier work on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_in, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_out, start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  auto zb = [&](int k) { return (int)((long long)k * nz / K); };
  for (int k = 0; k < K; ++k) {
    int rc = copy_planes(p, p->stage[0], in, zb(k) + s, zb(k + 1) + s, cudaMemcpyHostToDevice, p->copy_in);
    if (rc) return rc;
    e = cudaEventRecord(ein[k], p->copy_in);
    if (e != cudaSuccess) return cuda_fail(e, "event");
  }
  for (int k = 0; k < K; ++k) {
    e = cudaStreamWaitEvent(st, ein[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ein[(k + 1) % K], 0);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    int rc = K == 1 ? run_step(p, p->stage[0], p->stage[1], parity, kForward, st)
                    : run_step(p, p->stage[0], p->stage[1], parity, kForward, st, zb(k), zb(k + 1));
    if (rc) return rc;
    e = cudaEventRecord(eout[k], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_out, eout[k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    rc = copy_planes(p, out, p->stage[1], zb(k), zb(k + 1), cudaMemcpyDeviceToHost, p->copy_out);
    if (rc) return rc;
  }
  e = cudaEventRecord(done, p->copy_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, done, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer step");
  return HERMITE_OK;
}

// (Re)build the forward, adjoint and dS/dc tables of the plan's q-stage
// series, their FP32 copies and the double-float pairs of the hybrid modes.
void build_tables(hermite_plan_s *p) {
  const double tau = p->tau;
  build_step_coeffs(p->m, p->h, p->c, tau, kForward, p->q, &p->fwd);
  build_step_coeffs(p->m, p->h, p->c, tau, kAdjoint, p->q, &p->adj);
  build_step_coeffs(p->m, p->h, p->c, tau, kDc, p->q, &p->dc);
  p->fwd32 = cast_coeffs<float>(p->fwd);
  p->adj32 = cast_coeffs<float>(p->adj);
  p->dc32 = cast_coeffs<float>(p->dc);
  const StepCoeffs<double> *srcs[3] = {&p->fwd, &p->adj, &p->dc};
  HybridCoeffs *dsts[3] = {&p->hyb_fwd, &p->hyb_adj, &p->hyb_dc};
  for (int k = 0; k < 3; ++k) {
    dsts[k]->d = *srcs[k];
    dsts[k]->hi = cast_coeffs<float>(*srcs[k]);
    StepCoeffs<double> rest = *srcs[k];
    double *r = &rest.gx[0][0];
    const float *hi = &dsts[k]->hi.gx[0][0];
    for (size_t q = 0; q < sizeof(StepCoeffs<double>) / sizeof(double); ++q) r[q] -= (double)hi[q];
    dsts[k]->lo = cast_coeffs<float>(rest);
  }
  if (p->prec == HERMITE_REMAINDER) build_rem_coeffs(p->m, p->h, p->c, p->tau, p->fwd32, &p->rem);
  if (is_tc_prec(p->prec)) {
    const int kind = p->prec == HERMITE_3XTF32 ? 0 : 1;
    p->tc_fwd = build_tc_btable(p->m, kind, p->fwd);
    p->tc_adj = build_tc_btable(p->m, kind, p->adj);
    p->tc_dc = build_tc_btable(p->m, kind, p->dc);
  }
}

}  // namespace

extern "C" {

const char *hermite_last_error(void) { return g_last_error.c_str(); }

double hermite_stability_limit(int m) { return limit_of(m, 4); }

double hermite_stability_limit_taylor(int m, int q) { return limit_of(m, q); }

int hermite_plan(hermite_plan_t *out, int m, const int grid[3], const double h[3], double c, double dt,
                 int prec, int state_dtype, int variant) {
  return hermite_plan_taylor(out, m, grid, h, c, dt, prec, state_dtype, variant, 4);
}

int hermite_plan_taylor(hermite_plan_t *out, int m, const int grid[3], const double h[3], double c, double dt,
                        int prec, int state_dtype, int variant, int q) {
  g_last_error.clear();
  if (!out) return fail(HERMITE_EINVAL, "out is NULL");
  *out = nullptr;
  if (m < 1 || m > 3) return fail(HERMITE_EINVAL, "order m = %d not in 1..3", m);
  if (!grid || !h) return fail(HERMITE_EINVAL, "grid or h is NULL");
  for (int k = 0; k < 3; ++k) {
    if (grid[k] < 1 || grid[k] > (1 << 20)) return fail(HERMITE_EINVAL, "grid[%d] = %d out of range", k, grid[k]);
    if (!(h[k] > 0.0) || !std::isfinite(h[k])) return fail(HERMITE_EINVAL, "h[%d] must be positive", k);
  }
  if ((long long)grid[0] * grid[1] > kMaxPlaneNodes)
    return fail(HERMITE_EINVAL, "grid[0]*grid[1] = %lld nodes per x3-plane, above %lld", (long long)grid[0] * grid[1],
                kMaxPlaneNodes);
  if (!(c > 0.0) || !std::isfinite(c)) return fail(HERMITE_EINVAL, "wave speed c must be positive");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(HERMITE_EINVAL, "time step dt must be positive");
  if (prec != HERMITE_FP64 && prec != HERMITE_FP32 && prec != HERMITE_HYBRID64 && prec != HERMITE_HYBRIDDF &&
      !is_tc_prec(prec) && prec != HERMITE_REMAINDER)
    return fail(HERMITE_EUNSUPPORTED, "precision %d not provided", prec);
  if (state_dtype != HERMITE_STATE_FP64 && state_dtype != HERMITE_STATE_FP32)
    return fail(HERMITE_EINVAL, "state type %d unknown", state_dtype);
  if (prec != HERMITE_FP32 && !is_tc_prec(prec) && state_dtype != HERMITE_STATE_FP64)
    return fail(HERMITE_EUNSUPPORTED, "FP64 and hybrid arithmetic need an FP64 state");
  if ((is_tc_prec(prec) || prec == HERMITE_REMAINDER) && variant == HERMITE_SPLIT)
    return fail(HERMITE_EUNSUPPORTED, "the tensor-core and remainder-form precisions run the fused kernel only");
  if (variant != HERMITE_AUTO && variant != HERMITE_FUSED && variant != HERMITE_SPLIT)
    return fail(HERMITE_EINVAL, "variant %d unknown", variant);
  if (variant == HERMITE_SPLIT && (prec == HERMITE_HYBRID64 || prec == HERMITE_HYBRIDDF))
    return fail(HERMITE_EUNSUPPORTED, "the split variant has no hybrid precision");
  if (q < 4 || q > 3 * (2 * m + 1))
    return fail(HERMITE_EINVAL, "q = %d outside 4..%d (3(2m+1)) for order %d", q, 3 * (2 * m + 1), m);
  if (q != 4 && (prec == HERMITE_HYBRID64 || prec == HERMITE_HYBRIDDF || is_tc_prec(prec) || prec == HERMITE_REMAINDER))
    return fail(HERMITE_EUNSUPPORTED, "the hybrid, tensor-core and remainder-form precisions run the 4-stage series only");
  const double tau = 0.5 * dt;
  if (int rc = check_stable(m, q, c, tau, h)) return rc;
  const size_t nodes = (size_t)grid[0] * grid[1] * grid[2];
  hermite_plan_s *p = host_new<hermite_plan_s>();
  if (!p) return fail(HERMITE_ENOMEM, "plan allocation");
  p->m = m;
  for (int k = 0; k < 3; ++k) {
    p->n[k] = grid[k];
    p->h[k] = h[k];
  }
  p->c = c;
  p->dt = dt;
  p->tau = tau;
  p->prec = prec;
  p->q = q;
  p->state = state_dtype;
  p->variant = variant == HERMITE_AUTO ? HERMITE_FUSED : variant;
  p->elems = (size_t)2 * (m + 1) * (m + 1) * (m + 1) * nodes;
  build_H(m, p->H);
  build_tables(p);
  p->evolve.tau = tau;
  for (int k = 0; k < 3; ++k) p->evolve.c2h[k] = c * c / (h[k] * h[k]);
  p->evolve.q = q;
  build_interp_coeffs(m, &p->interp);
  p->tile = prec == HERMITE_REMAINDER ? 1 : 0;  // remainder form: two CTAs per SM (measured at m = 3, 256^3)
  p->zchunk = 16;
  p->ws_limit = (size_t)1 << 30;
  *out = p;
  return HERMITE_OK;
}

double hermite_adv_stability_limit(int m, int q) { return adv_limit_of(m, q == 0 ? 3 * (2 * m + 1) : q); }

int hermite_adv_plan(hermite_plan_t *out, int m, const int grid[3], const double h[3], const double a[3], double dt,
                     int q, int prec, int state_dtype, int variant) {
  g_last_error.clear();
  if (!out) return fail(HERMITE_EINVAL, "out is NULL");
  *out = nullptr;
  if (m < 1 || m > 3) return fail(HERMITE_EINVAL, "order m = %d not in 1..3", m);
  if (!grid || !h || !a) return fail(HERMITE_EINVAL, "grid, h or a is NULL");
  for (int k = 0; k < 3; ++k) {
    if (grid[k] < 1 || grid[k] > (1 << 20)) return fail(HERMITE_EINVAL, "grid[%d] = %d out of range", k, grid[k]);
    if (!(h[k] > 0.0) || !std::isfinite(h[k])) return fail(HERMITE_EINVAL, "h[%d] must be positive", k);
    if (!std::isfinite(a[k])) return fail(HERMITE_EINVAL, "velocity a[%d] is not finite", k);
  }
  if ((long long)grid[0] * grid[1] > kMaxPlaneNodes)
    return fail(HERMITE_EINVAL, "grid[0]*grid[1] = %lld nodes per x3-plane, above %lld", (long long)grid[0] * grid[1],
                kMaxPlaneNodes);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(HERMITE_EINVAL, "time step dt must be positive");
  const int qfull = 3 * (2 * m + 1);
  if (q == 0) q = qfull;
  if (q < 1 || q > qfull) return fail(HERMITE_EINVAL, "q = %d outside 1..%d (3(2m+1)) for order %d", q, qfull, m);
  if (prec != HERMITE_FP64 && prec != HERMITE_FP32)
    return fail(HERMITE_EUNSUPPORTED, "advection runs in FP64 or FP32 arithmetic");
  if (state_dtype != HERMITE_STATE_FP64 && state_dtype != HERMITE_STATE_FP32)
    return fail(HERMITE_EINVAL, "state type %d unknown", state_dtype);
  if (prec == HERMITE_FP64 && state_dtype != HERMITE_STATE_FP64)
    return fail(HERMITE_EUNSUPPORTED, "FP64 arithmetic needs an FP64 state");
  if (variant != HERMITE_AUTO && variant != HERMITE_FUSED && variant != HERMITE_SPLIT)
    return fail(HERMITE_EINVAL, "variant %d unknown", variant);
  if (variant == HERMITE_AUTO) variant = q == qfull ? HERMITE_FUSED : HERMITE_SPLIT;
  if (variant == HERMITE_FUSED && q != qfull)
    return fail(HERMITE_EUNSUPPORTED, "the fused advection kernel runs the whole series (q = %d) only", qfull);
  const double tau = 0.5 * dt;
  for (int k = 0; k < 3; ++k) {
    const double lam = std::fabs(a[k]) * tau / h[k];
    if (lam > adv_limit_of(m, q) * (1.0 + 1e-12))
      return fail(HERMITE_EUNSTABLE, "|a[%d]|*(dt/2)/h[%d] = %.6g above the stability limit %.3g of order %d, q = %d",
                  k, k, lam, adv_limit_of(m, q), m, q);
  }
  hermite_plan_s *p = host_new<hermite_plan_s>();
  if (!p) return fail(HERMITE_ENOMEM, "plan allocation");
  p->eq = 1;
  p->m = m;
  for (int k = 0; k < 3; ++k) {
    p->n[k] = grid[k];
    p->h[k] = h[k];
    p->a[k] = a[k];
  }
  p->c = 0.0;
  p->dt = dt;
  p->tau = tau;
  p->prec = prec;
  p->q = q;
  p->state = state_dtype;
  p->variant = variant;
  p->elems = (size_t)(m + 1) * (m + 1) * (m + 1) * grid[0] * grid[1] * grid[2];
  build_H(m, p->H);
  build_adv_coeffs(m, h, a, tau, &p->adv_fused, &p->adv_interp);
  p->adv_fused32 = cast_kron<float>(p->adv_fused);
  p->adv_interp32 = cast_kron<float>(p->adv_interp);
  p->adv_ev.tau = tau;
  for (int k = 0; k < 3; ++k) p->adv_ev.ah[k] = a[k] / h[k];
  p->adv_ev.q = q;
  // fastest fused schedules measured at 150^3 on GB300, [FP64?][m - 1]
  // (hermite_set_schedule overrides)
  static const int kAdvDefaultTile[2][3] = {{5, 5, 3}, {1, 5, 4}};
  p->tile = kAdvDefaultTile[prec == HERMITE_FP64 ? 1 : 0][m - 1];
  p->zchunk = 16;
  p->ws_limit = (size_t)1 << 30;
  *out = p;
  return HERMITE_OK;
}

int hermite_set_taylor_order(hermite_plan_t p, int q) {
  if (!p || p->batch) return fail(HERMITE_EINVAL, "plan is NULL or batched");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "advection plans fix q at hermite_adv_plan");
  if (q < 4 || q > 3 * (2 * p->m + 1))
    return fail(HERMITE_EINVAL, "q = %d outside 4..%d (3(2m+1)) for order %d", q, 3 * (2 * p->m + 1), p->m);
  if (q != 4 && (p->prec == HERMITE_HYBRID64 || p->prec == HERMITE_HYBRIDDF || is_tc_prec(p->prec) ||
                 p->prec == HERMITE_REMAINDER))
    return fail(HERMITE_EUNSUPPORTED, "the hybrid, tensor-core and remainder-form precisions run the 4-stage series only");
  if (int rc = check_stable(p->m, q, p->c, p->tau, p->h)) return rc;
  p->q = q;
  p->evolve.q = q;
  build_tables(p);
  return HERMITE_OK;
}

int hermite_taylor_order(hermite_plan_t p) { return p && !p->batch ? p->q : 0; }

size_t hermite_state_elems(hermite_plan_t p) { return p ? p->elems : 0; }

int hermite_schedule_count(hermite_plan_t p) {
  if (!p || p->batch) return 0;
  if (p->eq) return p->variant == HERMITE_SPLIT ? 1 : kAdvFusedTiles;
  if (p->prec == HERMITE_HYBRID64 || p->prec == HERMITE_HYBRIDDF) return hybrid_tile_count();
  if (p->prec == HERMITE_REMAINDER) return remainder_tile_count();
  if (is_tc_prec(p->prec)) return 1;
  return fused_tile_count(p->prec == HERMITE_FP64 ? 0 : 1, p->m);
}

int hermite_set_schedule(hermite_plan_t p, int tile, int zchunk) {
  if (!p || p->batch) return fail(HERMITE_EINVAL, "plan is NULL or batched");
  if (tile < 0 || tile >= hermite_schedule_count(p)) return fail(HERMITE_EINVAL, "tile %d out of range", tile);
  if (zchunk < 1 || zchunk > 4096) return fail(HERMITE_EINVAL, "zchunk %d out of range", zchunk);
  p->tile = tile;
  p->zchunk = zchunk;
  return HERMITE_OK;
}

int hermite_plan_operator(hermite_plan_t p, double *out) {
  if (!p || !out) return fail(HERMITE_EINVAL, "null argument");
  const int P = 2 * p->m + 2;
  std::memcpy(out, p->H, sizeof(double) * P * P);
  return HERMITE_OK;
}

int hermite_step(hermite_plan_t p, const void *in, void *out, int parity, void *stream) {
  if (!p) return fail(HERMITE_EINVAL, "plan is NULL");
  if (p->batch) return fail(HERMITE_EINVAL, "batched plan: use hermite_batch_step");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (!in || !out) return fail(HERMITE_EINVAL, "null state pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const PtrKind ki = classify(in), ko = classify(out);
  if (ki == kBadPtr || ko == kBadPtr) return fail(HERMITE_ECUDA, "cannot query pointer attributes (no CUDA device?)");
  if (ki != ko) return fail(HERMITE_EINVAL, "in and out must both be device or both be host buffers");
  if (ki == kDevicePtr) {
    int rc = check_device_pair(p, in, out);
    if (rc) return rc;
    return run_step(p, in, out, parity, kForward, st);
  }
  return host_step(p, in, out, parity, st);
}

int hermite_adjoint_step(hermite_plan_t p, const void *out_adj, void *in_adj, int parity, void *stream) {
  if (!p) return fail(HERMITE_EINVAL, "plan is NULL");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "no adjoint for advection plans");
  if (p->batch) return fail(HERMITE_EINVAL, "batched plan: use hermite_batch_step");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (int rc = check_device_only(p, out_adj, in_adj, "hermite_adjoint_step")) return rc;
  return run_step(p, out_adj, in_adj, parity, kAdjoint, (cudaStream_t)stream);
}

int hermite_step_dc(hermite_plan_t p, const void *in, void *out, int parity, void *stream) {
  if (!p) return fail(HERMITE_EINVAL, "plan is NULL");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "dS/dc is defined for the wave equation only");
  if (p->batch) return fail(HERMITE_EINVAL, "batched plan: use hermite_batch_step");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (int rc = check_device_only(p, in, out, "hermite_step_dc")) return rc;
  return run_step(p, in, out, parity, kDc, (cudaStream_t)stream);
}

int hermite_record(hermite_plan_t p, const void *state, const long long *idx, int count, double *out,
                   void *stream) {
  if (!p || !state || !idx || !out) return fail(HERMITE_EINVAL, "null argument");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "receivers are defined for the wave equation only");
  if (count < 0) return fail(HERMITE_EINVAL, "negative receiver count");
  if (count == 0) return HERMITE_OK;
  cudaError_t e = launch_record(p->state == HERMITE_STATE_FP64 ? kF64 : kF32, state, idx, count, out,
                                (cudaStream_t)stream);
  return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "record launch");
}

int hermite_inject(hermite_plan_t p, void *adj, const long long *idx, int count, const double *w, void *stream) {
  if (!p || !adj || !idx || !w) return fail(HERMITE_EINVAL, "null argument");
  if (p->eq) return fail(HERMITE_EUNSUPPORTED, "receivers are defined for the wave equation only");
  if (count < 0) return fail(HERMITE_EINVAL, "negative receiver count");
  if (count == 0) return HERMITE_OK;
  cudaError_t e = launch_inject(p->state == HERMITE_STATE_FP64 ? kF64 : kF32, adj, idx, count, w,
                                (cudaStream_t)stream);
  return e == cudaSuccess ? HERMITE_OK : cuda_fail(e, "inject launch");
}

int hermite_error(hermite_plan_t p, const void *state, const void *ref, unsigned mask, double out[4],
                  void *stream) {
  if (!p || !state || !ref || !out) return fail(HERMITE_EINVAL, "null argument");
  if (p->batch) return fail(HERMITE_EINVAL, "batched plan");
  if ((mask & 3u) == 0) return fail(HERMITE_EINVAL, "component mask selects no field");
  if (p->eq && (mask & 2u)) return fail(HERMITE_EINVAL, "an advection state has one field (mask bit 1 only)");
  if (classify(state) != kDevicePtr || classify(ref) != kDevicePtr)
    return fail(HERMITE_EINVAL, "hermite_error takes device buffers");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = error_blocks();
  int rc = ensure_red(p);
  if (rc) return rc;
  const size_t plane = (size_t)p->n[0] * p->n[1] * p->n[2];
  cudaError_t e = launch_error(p->state == HERMITE_STATE_FP64 ? kF64 : kF32, state, (const double *)ref, p->m,
                               plane, mask, p->red + 8, blocks, p->red, st);
  if (e != cudaSuccess) return cuda_fail(e, "error-norm launch");
  e = cudaMemcpyAsync(p->red_host, p->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "norm copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
  const double *r = p->red_host;
  out[0] = r[0];
  out[1] = r[1] > 0 ? r[0] / r[1] : INFINITY;
  out[2] = std::sqrt(r[2]);
  out[3] = r[3] > 0 ? std::sqrt(r[2] / r[3]) : INFINITY;
  if (r[4] > 0) return fail(HERMITE_ENONFINITE, "%.0f non-finite entries", r[4]);
  return HERMITE_OK;
}

int hermite_inject_alloc_failure(long long skip, long long count) {
  if (skip < 0 || count < 0) return fail(HERMITE_EINVAL, "negative skip or count");
  g_alloc_fail.store(0, std::memory_order_relaxed);
  g_alloc_skip.store(skip, std::memory_order_relaxed);
  g_alloc_fail.store(count, std::memory_order_relaxed);
  return HERMITE_OK;
}

int hermite_debug_build(void) { return kDebugBuild ? 1 : 0; }

int hermite_debug_status(hermite_plan_t p, int *flags, unsigned long long *first, void *stream) {
  if (!p || !flags || !first) return fail(HERMITE_EINVAL, "null argument");
  *flags = 0;
  *first = ~0ull;
  if (!p->dbg) return HERMITE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DebugRecord r{};
  const DebugRecord init{0, 0, ~0ull};
  cudaError_t e = cudaMemcpyAsync(&r, p->dbg, sizeof r, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(p->dbg, &init, sizeof init, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "debug record read");
  *flags = r.flags;
  *first = r.first;
  return HERMITE_OK;
}

int hermite_debug_selftest(hermite_plan_t p, const void *in, void *out, int parity, double fraction, void *stream) {
  if (!kDebugBuild) return fail(HERMITE_EUNSUPPORTED, "not a debug build");
  if (!p || p->batch || p->eq) return fail(HERMITE_EINVAL, "plan is NULL, batched or advection");
  if (!(fraction > 0.0 && fraction <= 1.0)) return fail(HERMITE_EINVAL, "fraction %g outside (0, 1]", fraction);
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (int rc = check_device_only(p, in, out, "hermite_debug_selftest")) return rc;
  p->dbg_bound = (size_t)((double)p->elems * fraction);
  if (p->dbg_bound == 0) p->dbg_bound = 1;
  const int rc = run_step(p, in, out, parity, kForward, (cudaStream_t)stream);
  p->dbg_bound = 0;
  return rc;
}

int hermite_debug_wait_drill(hermite_plan_t p, const void *in, void *out, int parity, void *stream) {
  if (!kDebugBuild) return fail(HERMITE_EUNSUPPORTED, "not a debug build");
  if (!p || p->batch || p->eq) return fail(HERMITE_EINVAL, "plan is NULL, batched or advection");
  const bool staged = p->prec == HERMITE_FP32 && p->q == 4 && p->variant != HERMITE_SPLIT && p->tile >= kFirstStagedTile;
  if (!staged && !is_tc_prec(p->prec))
    return fail(HERMITE_EINVAL, "the drill needs a tensor-core precision or a staged FP32 schedule");
  if (parity != 0 && parity != 1) return fail(HERMITE_EINVAL, "parity %d not 0 or 1", parity);
  if (int rc = check_device_only(p, in, out, "hermite_debug_wait_drill")) return rc;
  p->drill = 1;
  const int rc = run_step(p, in, out, parity, kForward, (cudaStream_t)stream);
  p->drill = 0;
  return rc;
}

int hermite_device_status(hermite_plan_t p, int *status, void *stream) {
  if (!p || !status) return fail(HERMITE_EINVAL, "null argument");
  *status = 0;
  if (!p->status) return HERMITE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device status read");
  *status = v;
  return HERMITE_OK;
}

int hermite_dot(hermite_plan_t p, const void *a, const void *b, double *out, void *stream) {
  if (!p || !a || !b || !out) return fail(HERMITE_EINVAL, "null argument");
  if (p->batch) return fail(HERMITE_EINVAL, "batched plan");
  if (classify(a) != kDevicePtr || classify(b) != kDevicePtr) return fail(HERMITE_EINVAL, "hermite_dot takes device buffers");
  int rc = ensure_red(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_dot(p->state == HERMITE_STATE_FP64 ? kF64 : kF32, a, b, p->elems, p->red + 8,
                             error_blocks(), p->red, st);
  if (e != cudaSuccess) return cuda_fail(e, "dot launch");
  e = cudaMemcpyAsync(p->red_host, p->red, sizeof(double) * 8, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "dot copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
  *out = p->red_host[2];
  return HERMITE_OK;
}

void hermite_destroy(hermite_plan_t p) {
  if (!p) return;
  for (auto &ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  if (p->copy_in) cudaStreamDestroy(p->copy_in);
  if (p->copy_out) cudaStreamDestroy(p->copy_out);
  if (p->batch) destroy_batch(p->batch);
  if (p->ws) cudaFree(p->ws);
  for (int k = 0; k < 2; ++k)
    if (p->stage[k]) cudaFree(p->stage[k]);
  if (p->red) cudaFree(p->red);
  if (p->red_host) cudaFreeHost(p->red_host);
  if (p->status) cudaFree(p->status);
  if (p->dbg) cudaFree(p->dbg);
  delete p;
}

}  // extern "C"
