// Internal declarations of the advection half step (Eq. 1 with a constant
// velocity a: u_t = a1 u_x1 + a2 u_x2 + a3 u_x3, one field).
//
// With the whole Taylor series (q = 3(2m+1) = d(2N+1) stages, Sec. 3.2) the
// local evolution of the cell polynomial is exact: the polynomial is
// translated by a tau, p(xi) -> p(xi + sigma) with sigma_k = a_k tau / h_k in
// the scaled variables of Eq. 3.  Interpolation (Sec. 3.1), translation and
// truncation to orders <= m (Sec. 2) are then one Kronecker product
// Gz (x) Gy (x) Gx of 1-D factors G_k = T1 Shift(sigma_k) H (M x P), and the
// fused kernel applies it in three passes.  Shorter series are not products
// (the Taylor terms couple the dimensions through their total degree) and run
// as the split pair: interpolation to the full cell polynomial (the same
// Kronecker kernel with the P x P factor H in every dimension), then the
// q-stage loop of Alg. 4 on it.
#pragma once

#include <cuda_runtime.h>

#include "hermite_impl.h"

namespace hermite {

constexpr int kAdvMaxP = 8;

// Row-major 1-D factors for x1, x2, x3: g[k][r][side * M + i], r < rows.
template <typename T>
struct KronCoeffs {
  T g[3][kAdvMaxP][kAdvMaxP];
};

template <typename T>
KronCoeffs<T> cast_kron(const KronCoeffs<double> &in) {
  KronCoeffs<T> o;
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < kAdvMaxP; ++r)
      for (int c = 0; c < kAdvMaxP; ++c) o.g[k][r][c] = (T)in.g[k][r][c];
  return o;
}

struct AdvEvolveParams {
  double tau;    // dt / 2
  double ah[3];  // a_k / h_k: d/dx_k = h_k^{-1} d/dxi_k
  int q;         // Taylor stages (Alg. 4)
};

// Host tables: the fused factors T1 Shift(a_k tau / h_k) H (rows r <= m) and
// the interpolation factors H (all P rows), from the exact H rounded once.
void build_adv_coeffs(int m, const double h[3], const double a[3], double tau, KronCoeffs<double> *fused,
                      KronCoeffs<double> *interp);

// Fused half step for output cells z in [g.zlo, g.zhi).  state / compute:
// kF32 or kF64 (compute kF64 needs state kF64); tile < kAdvFusedTiles picks
// one of the compiled CTA shapes.
constexpr int kAdvFusedTiles = 6;
cudaError_t launch_adv_fused(int m, int tile, int state, int compute, const void *in, void *out, const Geom &g,
                             const KronCoeffs<double> &cd, const KronCoeffs<float> &cf, int zchunk, cudaStream_t st);
// Split pair on the z-slab of cells [z0, z0 + nzl): interpolation into the
// workspace ws[jz][jy][jx][cell of the slab] (compute type), then Alg. 4 and
// truncation into the output state.
cudaError_t launch_adv_interp(int m, int state, int compute, const void *in, void *ws, const Geom &g, int z0, int nzl,
                              const KronCoeffs<double> &cd, const KronCoeffs<float> &cf, cudaStream_t st);
cudaError_t launch_adv_evolve(int m, int state, int compute, const void *ws, void *out, const Geom &g, int z0,
                              int nzl, const AdvEvolveParams &ep, cudaStream_t st);

}  // namespace hermite
