/*
 * hermite.h -- C ABI of libhermite: the Hermite half step of the 3-D scalar
 * linear wave equation u_t = v, v_t = c^2 (u_xx + u_yy + u_zz) on a staggered
 * primal/dual periodic tensor grid, on one NVIDIA GB300 (sm_103a).
 *
 * The method is that of Vargas, Chan, Hagstrom and Warburton, "GPU
 * Acceleration of Hermite Methods for the Simulation of Wave Propagation"
 * (arXiv:1609.09841):
 *   - Eq. 2: each node stores the scaled derivatives
 *       h1^i1 h2^i2 h3^i3 / (i1! i2! i3!) d^i f,  0 <= i1, i2, i3 <= m,
 *     of each field f in {u, v};
 *   - Eq. 3, Sec. 3.1, Alg. 1/2: on every cell the 8 corner nodes' data are
 *     interpolated, dimension by dimension, into a polynomial of degree 2m+1
 *     per variable whose coefficients are the scaled derivatives at the cell
 *     centre;
 *   - Eq. 4, Alg. 3/4: that polynomial is evolved locally over half a time
 *     step (here classical RK4, equal to a 4-term Taylor series for this
 *     linear operator);
 *   - Sec. 2: its coefficients of order <= m become the data of the dual
 *     node at the cell centre; the next half step maps dual -> primal.
 *
 * Conventions (all entry points)
 *   m           order: 1, 2 or 3 (the paper's N).  M = m+1 derivative orders
 *               per dimension, P = 2m+2 coefficients per dimension.
 *   grid[3]     (n1, n2, n3) = nodes along (x1, x2, x3); the grid is periodic.
 *   h[3]        (h1, h2, h3) node spacings (> 0).
 *   dt          the FULL time step of Eq. 4; every hermite_step advances the
 *               state by dt/2.
 *   state       2 * M^3 * n1*n2*n3 values, layout [f][i3][i2][i1][z][y][x]
 *               (field, derivative order along x3, x2, x1, then node with x1
 *               fastest: the tensor u[m3][m2][m1][n3][n2][n1] of Sec. 3.1 for
 *               each field).  Element type: double for HERMITE_STATE_FP64,
 *               float for HERMITE_STATE_FP32.  Buffers are contiguous and owned
 *               by the caller; device buffers must be 16-byte aligned.  The
 *               library cannot see a buffer's size or type: one smaller than
 *               the state, or of the other element type, is read or written
 *               past its end.  The Python binding checks both before the call.
 *   parity      0: the input lives on the primal grid (node i at i*h) and the
 *               output on the dual grid (node i at (i+1/2)*h, the centre of the
 *               cell with primal corners i, i+1); 1: dual -> primal (primal node
 *               i is the centre of the cell with dual corners i-1, i).
 *   stream      a cudaStream_t cast to void* (NULL = the legacy default stream).
 *               All work is enqueued on it and the calls return without waiting,
 *               except hermite_error, hermite_dot and host-buffer steps.
 *
 * Errors: every int-returning call returns HERMITE_OK (0) or a negative
 * hermite_status; hermite_last_error() then describes the failure (a
 * thread-local string owned by the library).  Invalid arguments never reach
 * the GPU.
 */
#ifndef HERMITE_H
#define HERMITE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hermite_plan_s *hermite_plan_t; /* opaque; owned by the library */

enum hermite_status {
  HERMITE_OK = 0,
  HERMITE_EINVAL = -1,       /* bad argument: order, sizes, pointers, parity, in == out */
  HERMITE_ENOMEM = -2,       /* a device or host allocation failed */
  HERMITE_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
  HERMITE_EUNSUPPORTED = -4, /* combination of precision / state type / variant not provided */
  HERMITE_EUNSTABLE = -5,    /* c*(dt/2)/h_k above the stability limit of order m */
  HERMITE_ETIMEOUT = -6,     /* a bounded device-side wait gave up (batched scheduler) */
  HERMITE_ENONFINITE = -7,   /* hermite_error saw a NaN or Inf */
  HERMITE_ENOCONV = -8       /* the eigenvalue iteration of a symbol did not converge */
};

/* Arithmetic of the contractions (interpolation and evolution). */
enum hermite_prec {
  HERMITE_FP64 = 0,     /* FP64 throughout (state must be FP64) */
  HERMITE_FP32 = 1,     /* FP32 contractions, state FP32 or FP64 (loaded, computed in FP32, stored) */
  /* FP32 x- and y-passes; the z-pass (the mode product along x3 of the 1-D
     evolution-and-truncation factors, Sec. 3.1 Alg. 1/2 with Sec. 3.2's
     evolution folded in) on the tensor cores (tcgen05) with FP32 accumulation,
     its operands split into pieces of the tensor-core input type.  State FP32
     or FP64 (loaded, computed, stored back).  Fused variant, RK4 (q = 4),
     single-grid plans only. */
  HERMITE_3XTF32 = 2,   /* y = a1 + a2 (TF32 pieces); a1 b1 + a1 b2 + a2 b1 */
  HERMITE_SPLITBF16 = 3, /* y = a1 + a2 + a3 (BF16 pieces); the six products of total order <= 2 */
  HERMITE_HYBRID64 = 4, /* FP64 state; every contraction applied to grade-0 data (the node data,
                           the x- and y-interpolants) in FP64, the rest (small grade >= 1 terms of
                           the Taylor series) in FP32.  Fused variant only. */
  HERMITE_HYBRIDDF = 5, /* as HYBRID64 with the FP64 part in double-float (pairs of FP32) */
  /* FP64 state; every 1-D factor applied in the one-sided Taylor-remainder
     form G_a [L; R] = TS_a L + RR_a (R - T L), which Hermite interpolation's
     exactness on polynomials of degree <= 2m+1 (Sec. 3.1) allows: T L is the
     right node's data of the left node's degree-m Taylor polynomial.  The
     large entries of RR_a then act on the small remainder, in FP32; the
     remainder and the grade-0 chain (short dyadic coefficients) are exact
     FP32 sums on a per-item grid.  Fused variant, RK4 (q = 4), forward steps
     (hermite_step) of single-grid plans. */
  HERMITE_REMAINDER = 6
};

enum hermite_state_type { HERMITE_STATE_FP64 = 0, HERMITE_STATE_FP32 = 1 };

/* Kernel design.  FUSED: one kernel per half step does interpolation,
 * evolution and truncation per cell (Sec. 3.3's monolithic design, re-done
 * with a Kronecker-sum factorisation of the whole half step).  SPLIT: an
 * interpolation kernel writes the cell polynomials to a workspace and an
 * evolution kernel runs the Taylor/RK4 loop on them (Sec. 3.1 + Sec. 3.2),
 * processed in z-slabs to bound the workspace.  AUTO = FUSED. */
enum hermite_variant { HERMITE_AUTO = 0, HERMITE_FUSED = 1, HERMITE_SPLIT = 2 };

/* Create a plan.  Checks every argument, the stability limit
 * (max_k c*(dt/2)/h_k <= hermite_stability_limit(m)) and builds the 1-D
 * operator tables in exact rational arithmetic on the host.  No GPU work and
 * no device allocation happen here, so a plan can be made without a GPU.
 * grid[k] (nodes along x1, x2, x3, periodic) runs from 1 to 2^20, with
 * grid[0] * grid[1] < 2^31 (EINVAL otherwise; the same bounds hold for
 * hermite_adv_plan and every simulation of a batched plan).
 * Returns EINVAL, EUNSTABLE, EUNSUPPORTED or ENOMEM; *out is NULL on failure. */
int hermite_plan(hermite_plan_t *out, int m, const int grid[3], const double h[3], double c,
                 double dt, int prec, int state_dtype, int variant);

/* The same with q Taylor stages for the local evolution (Alg. 4, Sec. 3.2;
 * q = 4 is RK4 and hermite_plan is this call with q = 4).  q runs from 4 to
 * 3(2m+1), where the series is exact for the cell polynomial.  The stability
 * check is max_k c*(dt/2)/h_k <= hermite_stability_limit_taylor(m, q), so a
 * plan with the full series may take a larger step than RK4 allows.  EINVAL
 * for q outside 4..3(2m+1); EUNSUPPORTED for q != 4 with a hybrid precision. */
int hermite_plan_taylor(hermite_plan_t *out, int m, const int grid[3], const double h[3], double c,
                        double dt, int prec, int state_dtype, int variant, int q);

/* One half step (Sec. 2): out = S_parity(in).  in and out are either both
 * device pointers (the step is only enqueued on `stream`) or both host
 * pointers (the library copies in -> device, steps and copies back through
 * plan-owned staging buffers, synchronising `stream` before it returns).
 * in == out (or overlapping buffers) is EINVAL: a half step is not in place. */
int hermite_step(hermite_plan_t plan, const void *in_state, void *out_state, int parity,
                 void *stream);

/* Discrete adjoint of hermite_step: in_adj = S_parity^T out_adj, where
 * out_adj lives on the output grid of the forward step with that parity and
 * in_adj on its input grid.  Same buffer rules as hermite_step (device
 * pointers only). */
int hermite_adjoint_step(hermite_plan_t plan, const void *out_adj, void *in_adj, int parity,
                         void *stream);

/* Error norms of `state` (the plan's state type) against `ref` (always FP64,
 * same layout), both device pointers, over the components selected by
 * component_mask: bit0 field u, bit1 field v, bit2 all derivative orders
 * (else the values i = (0,0,0) only).  out[0] = max|a-b|, out[1] =
 * max|a-b| / max|b|, out[2] = ||a-b||_2, out[3] = ||a-b||_2/||b||_2.
 * FP64 reduction on the device; synchronises `stream`.  Returns ENONFINITE
 * (with out filled) if any selected entry of either array is NaN or Inf. */
int hermite_error(hermite_plan_t plan, const void *state, const void *ref, unsigned component_mask,
                  double out[4], void *stream);

/* Derivative of the half step with respect to the wave speed:
 * out = (dS_parity / dc) in.  Every term of the half step's Taylor series of
 * order s in the Laplacian (Alg. 4) scales as c^(2s), so dS/dc is the same
 * operator with that term weighted by 2s/c.  Used to assemble gradients with
 * respect to c from forward states (recomputed from checkpoints) and adjoint
 * states.  Device buffers only; same rules as hermite_step. */
int hermite_step_dc(hermite_plan_t plan, const void *in_state, void *out_state, int parity,
                    void *stream);

/* FP64 dot product sum_i a_i b_i of two device states of the plan's state
 * type (all 2 M^3 n1 n2 n3 entries).  Synchronises `stream`. */
int hermite_dot(hermite_plan_t plan, const void *a, const void *b, double *out, void *stream);

/* Receivers.  idx (device, count entries) holds flat node indices
 * z*n1*n2 + y*n1 + x.  hermite_record writes out[k] (device, FP64) = the value
 * of u (orders (0,0,0)) at node idx[k] of `state`; hermite_inject adds w[k]
 * (device, FP64) to the same entries of an adjoint state (its transpose;
 * repeated indices accumulate).  Both only enqueue work on `stream`. */
int hermite_record(hermite_plan_t plan, const void *state, const long long *idx, int count,
                   double *out, void *stream);
int hermite_inject(hermite_plan_t plan, void *adj_state, const long long *idx, int count,
                   const double *w, void *stream);

/* Testing hook for allocation failures: after this call, the next `skip`
 * allocations of the library (host or device, in any plan or call) succeed
 * and the `count` after them fail as if memory were exhausted, so that the
 * calls that make them return HERMITE_ENOMEM and leave their plan usable.
 * count = 0 disarms it.  Not thread-safe against concurrent allocations in
 * other threads (the window is global).  EINVAL for negative arguments. */
int hermite_inject_alloc_failure(long long skip, long long count);

/* Debug build (the library compiled with -DHERMITE_DEBUG, libhermite_debug.so
 * from the package's build script): every global load and store of a state
 * in the fused kernels (FP64, FP32, hybrid, tensor-core and remainder-form
 * precisions, single-grid plans) is checked against the state size; an
 * out-of-range element offset is skipped (a load reads zero) and recorded.
 * hermite_debug_build returns 1 for such a library, 0 otherwise.
 * hermite_debug_status returns the flags raised since the last call (bit 1:
 * a load, bit 2: a store out of range; 0 in release builds) and the smallest
 * offending offset (~0 if none), then clears them; synchronises `stream`. */
int hermite_debug_build(void);
int hermite_debug_status(hermite_plan_t plan, int *flags, unsigned long long *first_index, void *stream);
/* Self-test of the debug build's checks: one forward half step of device
 * buffers in -> out (full-size states) in which the kernels are told that a
 * state holds only fraction x hermite_state_elems(plan) elements; every access
 * past that must be flagged and skipped (no access can leave the real
 * buffers).  EUNSUPPORTED in release builds; EINVAL for fraction outside
 * (0, 1], batched or advection plans and the buffer rules of hermite_step. */
int hermite_debug_selftest(hermite_plan_t plan, const void *in, void *out, int parity, double fraction,
                           void *stream);

/* Debug builds only (EUNSUPPORTED in release builds): one forward half step
 * as a drill of the kernels' bounded waits.  The awaited work is never issued
 * (no plane copy of a staged FP32 schedule, tiles 6 and 7; no MMA of a
 * tensor-core precision) and every wait gives up after a few polls, so each
 * CTA that would wait takes its failure path: it sets bit 0 of the status
 * word (hermite_device_status), waits once more (bounded), releases what it
 * holds and leaves its tile.  `out` is then incomplete.  EINVAL for other
 * plans or schedules and for the buffer rules of hermite_step. */
int hermite_debug_wait_drill(hermite_plan_t plan, const void *in, void *out, int parity, void *stream);

/* Device status of the plan's kernels: *status receives the OR of the flags
 * that kernels raised since the last call (0: none) and the flags are
 * cleared.  Bit 0: a CTA gave up after a bounded wait, its outputs then
 * incomplete: a CTA of the tensor-core kernel (HERMITE_3XTF32,
 * HERMITE_SPLITBF16) waiting for its MMAs, or a CTA of a staged FP32 schedule
 * waiting for a node plane's bulk copy.  Synchronises `stream`.  The word is
 * allocated by the plan's first step that can raise it; make that step outside
 * any stream capture. */
int hermite_device_status(hermite_plan_t plan, int *status, void *stream);

/* Kernel schedule of the fused half step: `tile` picks one of
 * hermite_schedule_count(plan) compiled tile shapes (cells per CTA in x1, x2
 * and threads per CTA, fixed per order and precision), `zchunk` the cells
 * each CTA marches along x3 (1..4096).  Defaults: tile 0, zchunk 16.  The
 * autotuner of the Python package times the choices on the device.  With
 * FP32 arithmetic (HERMITE_FP32) tiles 6 and 7 are staged: each node plane
 * is copied into shared memory by the bulk tensor-copy engine (TMA) while the
 * previous plane is computed; results equal the other tiles' bit for bit. */
int hermite_schedule_count(hermite_plan_t plan);
int hermite_set_schedule(hermite_plan_t plan, int tile, int zchunk);

/* Batched half step: nsims independent simulations, simulation i with order
 * m[i], grid grid[3i..3i+2], spacings h[3i..3i+2], wave speed c[i] and full
 * time step dt[i] (each checked as hermite_plan would), all with the same
 * precision and state type, advanced together by one persistent kernel launch
 * per half step.  The work list of (simulation, xy-tile, z-chunk) items is
 * handed out by an atomic counter, heaviest order first.  The returned plan
 * works only with the hermite_batch_* calls and hermite_destroy.  Creating it
 * allocates the per-simulation tables and the work list on the current
 * device. */
int hermite_batch_plan(hermite_plan_t *out, int nsims, const int *m, const int *grid, const double *h,
                       const double *c, const double *dt, int prec, int state_dtype);

/* State elements of simulation `sim` of a batched plan (0 if out of range). */
size_t hermite_batch_elems(hermite_plan_t plan, int sim);

/* z-chunk (cells per work item along x3) for orders 1, 2, 3; rebuilds the
 * work list and drops cached descriptor sets and graphs.  Default 16. */
int hermite_batch_set_schedule(hermite_plan_t plan, const int zchunk[3]);

/* Tile shape index (0 or 1, see hermite_batch_tile_shape) for orders 1, 2,
 * 3; rebuilds the work list and drops cached descriptor sets and graphs.
 * Default 0 for every order.  Results do not depend on the shape. */
int hermite_batch_set_tiles(hermite_plan_t plan, const int tile[3]);

/* The xy-tile (tx cells along x1, ty along x2) of tile shape `tile` of
 * order m in the batched kernel: m = 1: 16x8, 8x8; m = 2: 16x4, 8x4;
 * m = 3: 8x2, 4x4.  EINVAL outside m in 1..3, tile in 0..1. */
int hermite_batch_tile_shape(int m, int tile, int *tx, int *ty);

/* One half step of every simulation: out[i] = S_parity(in[i]).  in and out
 * are arrays of nsims device pointers.  The first call with a given pointer
 * set uploads a descriptor array (synchronously) and keeps it for later calls. */
int hermite_batch_step(hermite_plan_t plan, const void *const *in, void *const *out, int parity,
                       void *stream);

/* nhalf half steps of every simulation from the primal grid, ping-ponging
 * between the device buffer sets a[] and b[] (step k reads a if k is even, b if
 * odd, and writes the other; parity k % 2); the result is in a if nhalf is
 * even, else in b.  The steps are captured once into a CUDA graph (on a
 * plan-owned stream; call it the first time outside any stream capture) and
 * the graph is launched on `stream`. */
int hermite_batch_run(hermite_plan_t plan, void *const *a, void *const *b, int nhalf, void *stream);

/* Allocation-free half step (the paper has no counterpart: this serves
 * callers that cannot allocate device memory).  Callers that run while
 * another library owns the device memory (a framework's caching allocator or
 * a fixed memory budget), or time-critical loops that must not pay for
 * cudaMalloc or risk fragmentation, can call this instead of hermite_step.
 * It computes exactly what hermite_step computes with the SPLIT variant
 * (same kernels, same results) for device buffers in and out, which the
 * caller still provides, but its workspace is a static device array of
 * HERMITE_STATIC_WORKSPACE_BYTES (16 MiB) that every GPU loading the library
 * holds until the process exits, and it calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   - Size limit: one z-layer of cell polynomials, 2 (2m+2)^3 n1 n2 values of
 *     the arithmetic type, must fit in the array; otherwise EINVAL with a
 *     message naming both sizes.  Larger grids are processed in z-slabs.
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call outside any stream capture.
 *   - Sharing: every call on a device uses the same array and leaves its last
 *     contents there (nothing in it needs to start at zero: each call writes
 *     every entry it reads).  Calls whose work overlaps on the GPU (different
 *     streams, or graphs replayed concurrently) race on the array; order them
 *     on one stream.
 * Same argument rules and error codes as hermite_step (device pointers). */
#define HERMITE_STATIC_WORKSPACE_BYTES ((size_t)16 << 20)
int hermite_step_split_static(hermite_plan_t plan, const void *in_state, void *out_state, int parity,
                              void *stream);

/* HERMITE_STATIC_WORKSPACE_BYTES, as compiled into the library. */
size_t hermite_static_workspace_bytes(void);

/* Change the number of Taylor stages q of the local evolution (Alg. 4,
 * Sec. 3.2).  q = 4 is classical RK4 (the same polynomial in tau L).  Up to
 * q = 3(2m+1) = d(2N+1) stages the series is exact for the cell polynomial
 * (the paper's choice for the largest stable step).  Rebuilds the plan's
 * tables; the fused kernel then carries more grades of the series.  EINVAL
 * outside 4..3(2m+1); EUNSUPPORTED for the hybrid precisions (4 only);
 * EUNSTABLE when the plan's c*(dt/2)/h exceeds
 * hermite_stability_limit_taylor(m, q) (the plan keeps its old q).
 * Batched plans always use q = 4. */
int hermite_set_taylor_order(hermite_plan_t plan, int q);
int hermite_taylor_order(hermite_plan_t plan);

/* ---- Advection (Eq. 1) -------------------------------------------------
 * The 3-D advection equation of Sec. 2 with a constant velocity a:
 *   u_t = a1 u_x1 + a2 u_x2 + a3 u_x3   (Eq. 1 is a = (1, 1, 1)),
 * whose exact solution is u(x, t) = u(x + a t, 0).  One field: the state is
 * u[i3][i2][i1][n3][n2][n1] with the scaling and staggering of the wave
 * equation's states, (m+1)^3 * n1*n2*n3 elements.  The half step interpolates
 * (Sec. 3.1), evolves with the q-stage Hermite-Taylor loop (Alg. 4, the
 * recursion of Eq. 5) over dt/2 and truncates to orders <= m (Sec. 2).
 *
 * q = 0 selects q = 3(2m+1) = d(2N+1), the whole series, for which the
 * evolution is the exact translation of the cell polynomial and the half step
 * is one Kronecker product of 1-D maps (FUSED kernel).  1 <= q < 3(2m+1) runs
 * the SPLIT pair (interpolation kernel, then the Alg. 4 loop); AUTO picks
 * FUSED for the whole series and SPLIT otherwise; FUSED with a shorter series
 * is EUNSUPPORTED.  prec: FP64 (FP64 state) or FP32 (FP32 or FP64 state);
 * the hybrid precisions are EUNSUPPORTED.  The plan checks
 * max_k |a_k| (dt/2)/h_k <= hermite_adv_stability_limit(m, q) (EUNSTABLE).
 *
 * hermite_step, hermite_error (mask bit 1 only; bit 2 selects a field that
 * does not exist: EINVAL), hermite_dot, hermite_state_elems,
 * hermite_set_schedule (tile 0, zchunk), hermite_plan_operator and
 * hermite_destroy take advection plans; the adjoint, dS/dc, receiver,
 * Taylor-order, batched and allocation-free calls return EUNSUPPORTED. */
int hermite_adv_plan(hermite_plan_t *out, int m, const int grid[3], const double h[3], const double a[3],
                     double dt, int q, int prec, int state_dtype, int variant);

/* Largest max_k |a_k| (dt/2)/h_k of a stable advection half step of order m
 * with q stages (0: the whole series, whose limit is the half cell of Sec. 2,
 * 0.5).  The smaller of the Fourier-symbol limits for a mode along x1 and for
 * the diagonal direction, rounded down to two decimals; 0 where no step is
 * stable (q = 1) or for arguments out of range. */
double hermite_adv_stability_limit(int m, int q);

/* Number of state elements: 2 * (m+1)^3 * n1*n2*n3 (advection: (m+1)^3 * n1*n2*n3). */
size_t hermite_state_elems(hermite_plan_t plan);

/* Largest c*(dt/2)/h for which the half step of order m (1..3) is stable,
 * from the Fourier symbol of the isotropic half step; 0 for other m. */
double hermite_stability_limit(int m);

/* The same for q Taylor stages (4..3(2m+1)); 0 outside that range.  Not
 * monotone in q: m = 3 with q = 5 is stable only up to 0.09, while the full
 * series reaches 0.47 / 0.42 / 0.37 for m = 1 / 2 / 3 (at m = 3 the first
 * instability, 0.373, lies below a stable band around 0.40). */
double hermite_stability_limit_taylor(int m, int q);

/* ---- Stability tool (Sec. 2's stability condition, computed) ------------
 * The spectral radius of the Fourier symbol of one half step, and the
 * largest stable time step for a given order, series length and grid.  For
 * a mode exp(i theta . x / h) the symbol is the 2(m+1)^3 (wave) or (m+1)^3
 * (advection) square complex matrix of the half step; the scheme is stable
 * when its spectral radius is at most one for every theta.  Host-only
 * computations (no GPU, no plan needed): the wave symbol is assembled from
 * the same 1-D tables the kernels use, the advection symbol from the cell
 * matrix of interpolation + Alg. 4 + truncation; eigenvalues by a Hessenberg
 * reduction and the shifted QR iteration.
 *
 * hermite_symbol_radius: rho(G(theta)) of the wave half step with q Taylor
 *   stages (4..3(2m+1)), speed c, spacings h, full step dt.
 * hermite_max_radius: max rho over an npts^3 grid of theta in [0, pi]^3
 *   (the symbol at -theta is the conjugate), 1 <= npts <= 64.
 * hermite_max_dt: the largest dt such that max rho <= 1 + 1e-10 at every
 *   step up to it, for the given (possibly anisotropic) h and 2 <= npts <= 64.
 *   The stable steps need not form an interval (m = 3 with the whole series
 *   is weakly unstable for c tau / h in about (0.373, 0.39) and stable again
 *   at 0.40), so the steps 1.2 h_min k / (60 c), k = 1, 2, ..., are scanned
 *   to the first unstable one, whose bracket is then bisected to 1e-4
 *   relative; a window of instability narrower than the scan step can be
 *   missed.  hermite_plan's tables are this bound for h1 = h2 = h3 on a finer
 *   scan, rounded down.  Runs on up to 16 host threads; about a minute for
 *   m = 3 at npts = 7.
 * hermite_adv_symbol_radius / hermite_adv_max_dt: the same for advection
 *   with velocity a (q = 0: the whole series); a = 0 is EINVAL for the bound.
 * Errors: EINVAL for arguments out of range, ENOCONV if an eigenvalue
 * iteration did not converge. */
int hermite_symbol_radius(int m, int q, double c, const double h[3], double dt, const double theta[3],
                          double *rho);
int hermite_max_dt(int m, int q, double c, const double h[3], int npts, double *dt);
int hermite_max_radius(int m, int q, double c, const double h[3], double dt, int npts, double *rho);
int hermite_adv_symbol_radius(int m, int q, const double a[3], const double h[3], double dt,
                              const double theta[3], double *rho);
int hermite_adv_max_dt(int m, int q, const double a[3], const double h[3], int npts, double *dt);
int hermite_adv_max_radius(int m, int q, const double a[3], const double h[3], double dt, int npts,
                           double *rho);

/* Copy the plan's 1-D interpolation operator H (P x P, row-major, H[j][(side,i)]:
 * monomial coefficient j from [left i = 0..m, right i = 0..m], Sec. 3.1) to
 * out[0 .. P*P-1].  Host only; for inspection and tests. */
int hermite_plan_operator(hermite_plan_t plan, double *out);

/* Release the plan and every device buffer it owns (workspace, staging,
 * reduction scratch).  NULL is ignored. */
void hermite_destroy(hermite_plan_t plan);

/* Description of the last failure on the calling thread ("" if none). */
const char *hermite_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HERMITE_H */
