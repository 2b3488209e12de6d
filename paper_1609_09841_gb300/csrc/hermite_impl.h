// Internal declarations of libhermite: operator tables and kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <new>

namespace hermite {

constexpr int kMaxM = 4;  // largest M = m + 1
constexpr int kMaxDevices = 64;  // device ordinals the per-device records below cover

// Allocation gate: every host and device allocation of the library goes
// through these, so that hermite_inject_alloc_failure (a testing hook) can
// make chosen allocations fail as if memory were exhausted.
bool alloc_injected_failure();  // consumes one allocation of the injection window
cudaError_t dev_malloc(void **p, size_t bytes);          // cudaMalloc
cudaError_t host_malloc_pinned(void **p, size_t bytes);  // cudaMallocHost
template <typename T>
T *host_new() {  // new (std::nothrow) T()
  return alloc_injected_failure() ? nullptr : new (std::nothrow) T();
}

// Per-device record that a kernel's dynamic shared-memory limit has been
// raised.  The attribute belongs to each device's context, so a launcher keeps
// one record per kernel instantiation (a function-local static, zero at load)
// and raises the limit on every device it first runs on.
struct SmemAttrOnce {
  std::atomic<bool> done[kMaxDevices];
};

template <typename Kern>
cudaError_t raise_smem_limit(SmemAttrOnce &once, Kern kern, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kMaxDevices;
  if (tracked && once.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && tracked) once.done[dev].store(true, std::memory_order_release);
  return e;
}

// Tables of the fused half step.  For one cell and one input field the half
// step is the Kronecker sum  sum_s beta_s sum_{a+b+c=s} Gz_c (x) Gy_b (x) Gx_a
// (a, b, c <= 2), where G_a = T1 (lam^2 d^2/dxi^2)^a / a! H is the 1-D factor
// "interpolate (Sec. 3.1), differentiate twice a times (Alg. 3), keep orders
// <= m (Sec. 2)" and beta_s couples the fields through the 4-term Taylor
// series of RK4 (Alg. 4).  Every G_a satisfies G[r][(left, i)] =
// (-1)^(r+i) G[r][(right, i)], so only the right block is stored and the
// kernels apply it to R_i + (-1)^(r+i) L_i (an even/odd butterfly).
// Largest grade of the Kronecker factors in one dimension (a <= m <= 3) and
// of the y-pass results (a + b <= 2m <= 6).
constexpr int kMaxA = 4, kMaxG = 7;

template <typename T>
struct StepCoeffs {
  T gx[kMaxA][16];           // right block of G_a along x1, [a][r * 4 + i]
  T gy[kMaxA][16];           // same along x2
  T kz[2][2][kMaxG][16];     // [f_out][f_in][grade g][r * 4 + i] = sum_c beta_{g+c} Gz_c (right block)
};

// Tables of the split pair: the right block of H (interpolation) and the
// constants of the local evolution.
template <typename T>
struct InterpCoeffs {
  T hr[8][4];  // H[r][M + i], r < P
};
struct EvolveParams {
  double tau;     // half-step duration dt / 2
  double c2h[3];  // c^2 / h_k^2 along x1, x2, x3
  int q;          // Taylor stages (Alg. 4)
};

// Host-side construction (exact rational arithmetic, then rounded once).
void build_H(int m, double *H);  // P x P row-major
// mode: the half step S (kForward), its transpose S^T (kAdjoint), or its
// derivative dS/dc with respect to the wave speed (kDc).
enum CoeffMode { kForward = 0, kAdjoint = 1, kDc = 2 };
// q: stages of the Taylor series of the local evolution (4 = RK4).
void build_step_coeffs(int m, const double h[3], double c, double tau, int mode, int q,
                       StepCoeffs<double> *out);
void build_interp_coeffs(int m, InterpCoeffs<double> *out);

template <typename T>
StepCoeffs<T> cast_coeffs(const StepCoeffs<double> &in) {
  StepCoeffs<T> o;
  for (int a = 0; a < kMaxA; ++a)
    for (int k = 0; k < 16; ++k) {
      o.gx[a][k] = (T)in.gx[a][k];
      o.gy[a][k] = (T)in.gy[a][k];
    }
  for (int f = 0; f < 2; ++f)
    for (int g = 0; g < 2; ++g)
      for (int s = 0; s < kMaxG; ++s)
        for (int k = 0; k < 16; ++k) o.kz[f][g][s][k] = (T)in.kz[f][g][s][k];
  return o;
}

// Tables of the hybrid-precision kernel: the same tables in double, and as
// double-float pairs (hi = float(d), lo = float(d - hi)).
struct HybridCoeffs {
  StepCoeffs<double> d;
  StepCoeffs<float> hi;
  StepCoeffs<float> lo;
};

// Grid geometry of one launch.
// Record of the debug build's bounds checks (device memory): the flags
// raised (bit 1: a load, bit 2: a store outside the state) and the smallest
// offending element offset.
struct DebugRecord {
  int flags;
  int pad;
  unsigned long long first;
};

struct Geom {
  int nx, ny, nz;
  int s;         // corner offset: corners of output node o are o + s + {0, 1} per dimension
  int zlo, zhi;  // output z layers [zlo, zhi) computed by a launch (the fused and hybrid kernels)
  size_t elems = 0;             // elements of one state (debug build: the bound of every index; 0: unchecked)
  DebugRecord *dbg = nullptr;   // debug build: where out-of-range accesses are recorded
  int drill = 0;                // debug build: bounded-wait drill (hermite_debug_wait_drill)
};

// Polls of a bounded wait in a drill step: the awaited copy or MMA is never
// issued, so every wait runs out after these polls and takes its failure path.
constexpr unsigned kDrillPolls = 64;

// Bounds checks of the debug build (compiled with -DHERMITE_DEBUG): the
// fused kernels route every global load and store of a state through these;
// an element offset at or beyond g.elems raises `bit` and is recorded in
// *g.dbg, and the access is skipped (a load returns zero).  Release builds
// compile to the plain access.
template <typename T>
__device__ __forceinline__ T state_load(const Geom &g, const T *base, const T *ptr) {
#ifdef HERMITE_DEBUG
  const size_t off = (size_t)(ptr - base);
  if (g.elems && off >= g.elems) {
    if (g.dbg) {
      atomicOr(&g.dbg->flags, 2);
      atomicMin(&g.dbg->first, (unsigned long long)off);
    }
    return T(0);
  }
#else
  (void)g;
  (void)base;
#endif
  return __ldg(ptr);
}
template <typename T>
__device__ __forceinline__ void state_store(const Geom &g, T *base, T *ptr, T v) {
#ifdef HERMITE_DEBUG
  const size_t off = (size_t)(ptr - base);
  if (g.elems && off >= g.elems) {
    if (g.dbg) {
      atomicOr(&g.dbg->flags, 4);
      atomicMin(&g.dbg->first, (unsigned long long)off);
    }
    return;
  }
#else
  (void)g;
  (void)base;
#endif
  *ptr = v;
}
constexpr bool kDebugBuild =
#ifdef HERMITE_DEBUG
    true;
#else
    false;
#endif

// Cells per CTA along x3 such that ceil(nzl / zchunk) CTAs fit gridDim.y
// (and gridDim.z), at most 65535: the requested chunk, or a larger one.
inline int clamp_zchunk(int nzl, int zchunk) {
  if (zchunk < 1) zchunk = 1;
  if (nzl > 0 && (nzl + zchunk - 1) / zchunk > 65535) zchunk = (nzl + 65534) / 65535;
  return zchunk;
}

enum StateKind { kF64 = 0, kF32 = 1 };

// Fused half step (forward or adjoint: the adjoint is the same kernel with
// transposed tables and the mirrored offset).
// Kernels for more than 4 Taylor stages (one tile shape each): enough grades
// for any q <= 3(2m+1).
cudaError_t launch_fused_f64_fullq(int m, const double *in, double *out, const Geom &g,
                                   const StepCoeffs<double> &co, int zchunk, cudaStream_t st);
cudaError_t launch_fused_f32_fullq(int m, int state, const void *in, void *out, const Geom &g,
                                   const StepCoeffs<float> &co, int zchunk, cudaStream_t st);
// `tile` selects one of fused_tile_count(prec, m) compiled tile shapes.
int fused_tile_count(int prec, int m);
constexpr int kFirstStagedTile = 6;  // FP32 arithmetic: tiles 6 and 7 are staged
cudaError_t launch_fused_f64(int m, int tile, const double *in, double *out, const Geom &g,
                             const StepCoeffs<double> &co, int zchunk, cudaStream_t st);
// FP32 arithmetic: tiles 6 and 7 are staged (their copy time-outs set bit 0
// of *status, a device word the caller owns; the other tiles ignore it).
cudaError_t launch_fused_f32_s32(int m, int tile, const float *in, float *out, const Geom &g,
                                 const StepCoeffs<float> &co, int zchunk, int *status, cudaStream_t st);
cudaError_t launch_fused_f32_s64(int m, int tile, const double *in, double *out, const Geom &g,
                                 const StepCoeffs<float> &co, int zchunk, int *status, cudaStream_t st);

// Hybrid-precision fused half step (FP64 state): kind 0 = grade-0 chain in
// FP64, kind 1 = in double-float; `tile` < hybrid_tile_count().
int hybrid_tile_count();
cudaError_t launch_hybrid(int kind, int m, int tile, const double *in, double *out, const Geom &g,
                          const HybridCoeffs &co, int zchunk, cudaStream_t st);

// Fused half step with the z-pass on the tensor cores (tcgen05): kind 0 =
// 3xTF32, kind 1 = BF16 x 3, FP32 accumulation; FP32 (kF32) or FP64 (kF64)
// state.  The z-pass B operand is built once per plan on the host.  A CTA
// whose wait for its MMAs gives up sets bit 0 of *status (device int).
// The z-pass B operand (all pieces, in shared-memory byte order), built on the
// host from the Kz tables; at most 3 pieces x 16 x 32 BF16 or 2 x 16 x 24 TF32.
struct TcBTable {
  uint4 words[192];
};
TcBTable build_tc_btable(int m, int kind, const StepCoeffs<double> &co);
cudaError_t launch_fused_tc(int kind, int m, int state, const void *in, void *out, const Geom &g,
                            const StepCoeffs<float> &co, const TcBTable &bt, int zchunk, int *status,
                            cudaStream_t st);

// Tables of the remainder-form kernel (remainder.cuh), per dimension d = x1,
// x2, x3 and grade a of the 1-D factor G_a = lam^(2a)/a! T1 (d^2/dxi^2)^a H:
// G_a [L; R] = ts_a L + rr_a rho with rho the remainder of the left node's
// degree-m Taylor polynomial at the right node.
struct RemCoeffs {
  float ts[3][3][4][4];  // [d][a][r][j]: coefficient of xi^r of (d/dxi)^(2a) p_L (exact dyadic)
  float rr[3][3][4][4];  // [d][a][r][i]: right-node block of T1 (d^2/dxi^2)^a H (exact dyadic)
  float scale[3][3];     // [d][a]: lam_d^(2a)/a!
  float beta[2][2][3];   // beta_c[fo][fi] of the 4-term series for the z-grades c of the grade-0 chain
  float gy[3][16];       // right blocks of Gy_b (FP32), for Gy_b X_a with a >= 1
  float kz[2][2][3][16]; // Kz[fo][fi][g] (FP32), for the y-results of grade g >= 1
  // the same as pairs of rows (r, r+1) = (2 rp, 2 rp + 1) for fma.rn.f32x2 (low word row 2 rp)
  unsigned long long gy2[3][2][4];        // [b][rp][i]
  unsigned long long kz2[2][2][2][2][4];  // [fo][fi][g - 1][rp][i]
  unsigned long long rr2[3][3][2][4];     // [d][a][rp][i]: rows (2 rp, 2 rp + 1) of rr[d][a]
  // the remainder's -C(j, i) and the Taylor shift's C(j, r) 2^-(j-r), each in both words
  unsigned long long edge2[4][4];         // [i][j], j >= i
  unsigned long long ts02[4][4];          // [r][j], j > r
};
void build_rem_coeffs(int m, const double h[3], double c, double tau, const StepCoeffs<float> &f32,
                      RemCoeffs *out);
int remainder_tile_count();
cudaError_t launch_remainder(int m, int tile, const double *in, double *out, const Geom &g, const RemCoeffs &co,
                             int zchunk, cudaStream_t st);

// Split pair.  Interpolation writes Ru[f][jz][jy][jx][cell] for the cells of
// output z-layers [z0, z0 + nzl); evolution reads it and writes the new node
// data of those layers.
cudaError_t launch_interp(int m, int state, int compute, const void *in, void *ru, const Geom &g,
                          int z0, int nzl, const InterpCoeffs<double> &co, cudaStream_t st);
cudaError_t launch_evolve(int m, int state, int compute, const void *ru, void *out, const Geom &g,
                          int z0, int nzl, const EvolveParams &ep, cudaStream_t st);

// FP64 error reduction.  `partial` holds blocks * 8 doubles of scratch,
// `result` 8 doubles.
cudaError_t launch_error(int state, const void *a, const double *b, int m, size_t plane,
                         unsigned mask, double *partial, int blocks, double *result,
                         cudaStream_t st);
int error_blocks();

// FP64 dot product sum_i a_i b_i of two states (a of the state type, b the
// same type), same partial/result scratch convention as launch_error.
cudaError_t launch_dot(int state, const void *a, const void *b, size_t n, double *partial, int blocks,
                       double *result, cudaStream_t st);

// Receivers: out[k] = value of u at flat node index idx[k]; adjoint: add w[k]
// to the same entries of an adjoint state.
cudaError_t launch_record(int state, const void *s, const long long *idx, int count, double *out,
                          cudaStream_t st);
cudaError_t launch_inject(int state, void *adj, const long long *idx, int count, const double *w,
                          cudaStream_t st);

}  // namespace hermite
