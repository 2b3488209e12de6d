// Hybrid-precision fused half step.
//
// In FP32 the half step loses accuracy through catastrophic cancellation.
// The high-order coefficients of the interpolant (Sec. 3.1) are small
// combinations of node data of the size of the field, and the evolution
// (Alg. 3/4) weights exactly those coefficients.  The rounding of the
// O(|u|)-sized grade-0 data (node values, the x-pass and y-pass interpolants
// X_0, Y_0) therefore enters the result amplified by (k h)^-2 and more, and
// the error of the FP32 kernel grows with resolution and with the number of
// half steps.  Every contraction whose input is grade-0 data -- the whole
// x-pass, the y-pass applied to X_0 and the z-pass applied to Y_0 -- runs here
// in the high-precision type Hi::T (FP64, or double-float pairs of FP32).  The
// contractions of grade >= 1 data, small quantities whose own relative
// rounding does not cancel, run in FP32.  The state is FP64.
//
// Same tiling, marching and butterflies as fused.cuh.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "fused.cuh"
#include "hermite_impl.h"

namespace hermite {

struct HiF64 {  // high-precision part in FP64
  using T = double;
  static __device__ __forceinline__ T from(double x) { return x; }
  static __device__ __forceinline__ double to_double(T x) { return x; }
  static __device__ __forceinline__ float to_float(T x) { return (float)x; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T mad(T c, T x, T acc) { return ::fma(c, x, acc); }
  static __device__ __forceinline__ T mad_exact(double c, float, T x, T acc) { return ::fma(c, x, acc); }
  static __device__ __forceinline__ T norm(T x) { return x; }
  static __device__ __forceinline__ double to_double_plus(T x, float f) { return x + (double)f; }
  static __device__ __forceinline__ T gx(const HybridCoeffs &c, int a, int q) { return c.d.gx[a][q]; }
  static __device__ __forceinline__ T gy(const HybridCoeffs &c, int b, int q) { return c.d.gy[b][q]; }
  static __device__ __forceinline__ T kz(const HybridCoeffs &c, int fo, int fi, int q) { return c.d.kz[fo][fi][0][q]; }
};

struct HiDF {  // high-precision part in double-float
  using T = df32;
  static __device__ __forceinline__ T from(double x) { return df_from(x); }
  static __device__ __forceinline__ double to_double(T x) { return df_to_double(x); }
  static __device__ __forceinline__ float to_float(T x) { return df_to_float(x); }
  static __device__ __forceinline__ T zero() { return df32{0.f, 0.f}; }
  static __device__ __forceinline__ T mad(T c, T x, T acc) { return df_mad(c, x, acc); }
  // G_0 = T1 H has dyadic entries with numerators <= 35: exact in FP32, no low word
  static __device__ __forceinline__ T mad_exact(double, float c, T x, T acc) { return df_mad1(c, x, acc); }
  static __device__ __forceinline__ T norm(T x) { return df_norm(x); }
  static __device__ __forceinline__ double to_double_plus(T x, float f) { return df_to_double(x + df32{f, 0.f}); }
  static __device__ __forceinline__ T gx(const HybridCoeffs &c, int a, int q) { return {c.hi.gx[a][q], c.lo.gx[a][q]}; }
  static __device__ __forceinline__ T gy(const HybridCoeffs &c, int b, int q) { return {c.hi.gy[b][q], c.lo.gy[b][q]}; }
  static __device__ __forceinline__ T kz(const HybridCoeffs &c, int fo, int fi, int q) {
    return {c.hi.kz[fo][fi][0][q], c.lo.kz[fo][fi][0][q]};
  }
};

template <int M, int TX, int TY>
struct HybridShape {
  static constexpr int NYN = TY + 1;
  static constexpr int NA = (M == 2) ? 2 : 3;
  static constexpr int SX0 = 2 * M * M * M * NYN * TX;             // Hi: X_0 [f][iz][iy][ix'][ey][ex]
  static constexpr int SX1 = 2 * M * M * (NA - 1) * M * NYN * TX;  // float: X_a, a >= 1 [f][iz][iy][a-1][ix'][ey][ex]
  static constexpr int SY0 = 2 * M * M * M * TX * TY;              // Hi: Y_0 [f][iz][iy'][ix'][fy][fx], per plane
  static constexpr int SY1 = 2 * 2 * M * M * M * TX * TY;          // float: Y_1, Y_2 [f][g-1][iz][iy'][ix'][fy][fx]
  static constexpr size_t SMEM = (size_t)(SX0 + 2 * SY0) * 8 + (size_t)(SX1 + 2 * SY1) * 4;
  static constexpr int XITEMS = 2 * M * M * NYN * TX;
  static constexpr int YITEMS = 2 * M * M * TY * TX;
  static constexpr int ZITEMS = M * M * TX * TY;
};

template <class Hi, int M, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
    hybrid_step_kernel(const double *__restrict__ in, double *__restrict__ out, const Geom g, int zchunk,
                       const HybridCoeffs co) {
  using H = typename Hi::T;
  using Sh = HybridShape<M, TX, TY>;
  constexpr int NYN = Sh::NYN, NA = Sh::NA;
  constexpr int XPT = (Sh::XITEMS + NT - 1) / NT;
  constexpr int YPT = (Sh::YITEMS + NT - 1) / NT;
  constexpr int ZPT = (Sh::ZITEMS + NT - 1) / NT;
  constexpr int XS = NYN * TX, YS = TY * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  H *sX0 = reinterpret_cast<H *>(smem_raw);
  H *sY0 = sX0 + Sh::SX0;                                   // two planes
  float *sX1 = reinterpret_cast<float *>(sY0 + 2 * Sh::SY0);
  float *sY1 = sX1 + Sh::SX1;                               // two planes

  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const int tiles_x = (nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = g.zlo + blockIdx.y * zchunk;
  if (z0 >= g.zhi) return;
  const int z1 = min(z0 + zchunk, g.zhi);
  const size_t pxy = (size_t)nx * ny;
  const size_t plane = pxy * nz;

  const double *xsrc[XPT];
  int xl[XPT], xr[XPT], xd0[XPT], xd1[XPT];
#pragma unroll
  for (int k = 0; k < XPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::XITEMS ? e : 0;
    const int ex = t % TX; t /= TX;
    const int ey = t % NYN; t /= NYN;
    const int iy = t % M; t /= M;
    const int iz = t % M;
    const int f = t / M;
    const int gy = wrap_index(y0 + s + ey, ny);
    const int q = (f * M + iz) * M + iy;
    xsrc[k] = in + (size_t)(q * M) * plane;
    xl[k] = gy * nx + wrap_index(x0 + s + ex, nx);
    xr[k] = gy * nx + wrap_index(x0 + s + ex + 1, nx);
    xd0[k] = e < Sh::XITEMS ? q * M * XS + ey * TX + ex : -1;
    xd1[k] = q * (NA - 1) * M * XS + ey * TX + ex;
  }
  int ys0[YPT], ys1[YPT], yd0[YPT], yd1[YPT];
#pragma unroll
  for (int k = 0; k < YPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::YITEMS ? e : 0;
    const int fx = t % TX; t /= TX;
    const int fy = t % TY; t /= TY;
    const int ixp = t % M; t /= M;
    const int iz = t % M;
    const int f = t / M;
    ys0[k] = ((f * M + iz) * M * M + ixp) * XS + fy * TX + fx;               // + iy * M * XS
    ys1[k] = ((f * M + iz) * M * (NA - 1) * M + ixp) * XS + fy * TX + fx;    // + (iy * (NA-1) + a-1) * M * XS
    yd0[k] = e < Sh::YITEMS ? ((f * M + iz) * M * M + ixp) * YS + fy * TX + fx : -1;   // + r * M * YS
    yd1[k] = ((f * 2 * M + iz) * M * M + ixp) * YS + fy * TX + fx;           // + ((g-1) M^3 + r M) * YS
  }
  int zs[ZPT], zxy[ZPT], zcomp[ZPT];
#pragma unroll
  for (int k = 0; k < ZPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::ZITEMS ? e : 0;
    const int cx = t % TX; t /= TX;
    const int cy = t % TY; t /= TY;
    const int ixp = t % M;
    const int iyp = t / M;
    zs[k] = (iyp * M + ixp) * YS + cy * TX + cx;
    zcomp[k] = iyp * M + ixp;
    const int ox = x0 + cx, oy = y0 + cy;
    zxy[k] = (e < Sh::ZITEMS && ox < nx && oy < ny) ? oy * nx + ox : -1;
  }

  for (int p = 0; p <= z1 - z0; ++p) {
    const size_t zoff = (size_t)wrap_index(z0 + s + p, nz) * pxy;
    // x-pass: every output comes from grade-0 node data -> high precision
    double Lv[XPT][M], Rv[XPT][M];
#pragma unroll
    for (int k = 0; k < XPT; ++k) {
      if (xd0[k] < 0) continue;
      const double *src = xsrc[k] + zoff;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Lv[k][i] = state_load(g, in, src + i * plane + xl[k]);
        Rv[k][i] = state_load(g, in, src + i * plane + xr[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < XPT; ++k) {
      if (xd0[k] < 0) continue;
      H sv[M], dv[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const H L = Hi::from(Lv[k][i]), R = Hi::from(Rv[k][i]);
        sv[i] = (i & 1) ? R - L : R + L;
        dv[i] = (i & 1) ? R + L : R - L;
      }
#pragma unroll
      for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int r = 0; r < M; ++r) {
          H acc = Hi::zero();
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const int q = r * 4 + i;
            if (a == 0)
              acc = Hi::mad_exact(co.d.gx[0][q], co.hi.gx[0][q], (r & 1) ? dv[i] : sv[i], acc);
            else
              acc = Hi::mad(Hi::gx(co, a, q), (r & 1) ? dv[i] : sv[i], acc);
          }
          acc = Hi::norm(acc);
          if (a == 0)
            sX0[xd0[k] + r * XS] = acc;
          else
            sX1[xd1[k] + ((a - 1) * M + r) * XS] = Hi::to_float(acc);
        }
    }
    __syncthreads();
    // y-pass: Gy_b applied to X_0 in high precision, to X_1, X_2 in FP32
#pragma unroll
    for (int k = 0; k < YPT; ++k) {
      if (yd0[k] < 0) continue;
      H s0[M], d0[M];
      float sa[NA - 1][M], da[NA - 1][M];
#pragma unroll
      for (int iy = 0; iy < M; ++iy) {
        const H *x = sX0 + ys0[k] + iy * M * XS;
        const H L = x[0], R = x[TX];
        s0[iy] = (iy & 1) ? R - L : R + L;
        d0[iy] = (iy & 1) ? R + L : R - L;
#pragma unroll
        for (int a = 1; a < NA; ++a) {
          const float *xf = sX1 + ys1[k] + (iy * (NA - 1) + a - 1) * M * XS;
          const float Lf = xf[0], Rf = xf[TX];
          sa[a - 1][iy] = (iy & 1) ? Rf - Lf : Rf + Lf;
          da[a - 1][iy] = (iy & 1) ? Rf + Lf : Rf - Lf;
        }
      }
      H *y0o = sY0 + (p & 1) * Sh::SY0 + yd0[k];
      float *y1o = sY1 + (p & 1) * Sh::SY1 + yd1[k];
#pragma unroll
      for (int gg = 0; gg < 3; ++gg)
#pragma unroll
        for (int r = 0; r < M; ++r) {
          H acc = Hi::zero();
          if (gg < NA) {
#pragma unroll
            for (int i = 0; i < M; ++i) {
              const int q = r * 4 + i;
              if (gg == 0)
                acc = Hi::mad_exact(co.d.gy[0][q], co.hi.gy[0][q], (r & 1) ? d0[i] : s0[i], acc);
              else
                acc = Hi::mad(Hi::gy(co, gg, q), (r & 1) ? d0[i] : s0[i], acc);
            }
            acc = Hi::norm(acc);
          }
          if (gg == 0) {
            y0o[r * M * YS] = acc;
          } else {
            float accf = 0.f;
#pragma unroll
            for (int a = 1; a < NA; ++a) {
              const int b = gg - a;
              if (b < 0 || b >= NA) continue;
#pragma unroll
              for (int i = 0; i < M; ++i)
                accf = fmaf(co.hi.gy[b][r * 4 + i], (r & 1) ? da[a - 1][i] : sa[a - 1][i], accf);
            }
            y1o[((gg - 1) * M * M * M + r * M) * YS] = Hi::to_float(acc) + accf;
          }
        }
    }
    __syncthreads();
    // z-pass: Kz[.][.][g=0] on the Y_0 butterflies in high precision, g = 1, 2 in FP32
    if (p > 0) {
      const H *c0 = sY0 + (p & 1) * Sh::SY0, *p0 = sY0 + ((p - 1) & 1) * Sh::SY0;
      const float *c1 = sY1 + (p & 1) * Sh::SY1, *p1 = sY1 + ((p - 1) & 1) * Sh::SY1;
#pragma unroll
      for (int k = 0; k < ZPT; ++k) {
        if (zxy[k] < 0) continue;
        H s0[2][M], d0[2][M];
        float s1[2][2][M], d1[2][2][M];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int iz = 0; iz < M; ++iz) {
            const int q = zs[k] + (f * M + iz) * M * M * YS;
            const H L = p0[q], R = c0[q];
            s0[f][iz] = (iz & 1) ? R - L : R + L;
            d0[f][iz] = (iz & 1) ? R + L : R - L;
#pragma unroll
            for (int gm = 0; gm < 2; ++gm) {
              const int q1 = zs[k] + ((f * 2 + gm) * M + iz) * M * M * YS;
              const float Lf = p1[q1], Rf = c1[q1];
              s1[f][gm][iz] = (iz & 1) ? Rf - Lf : Rf + Lf;
              d1[f][gm][iz] = (iz & 1) ? Rf + Lf : Rf - Lf;
            }
          }
        double *o = out + (size_t)(z0 + p - 1) * pxy + zxy[k] + (size_t)zcomp[k] * plane;
#pragma unroll
        for (int fo = 0; fo < 2; ++fo)
#pragma unroll
          for (int r = 0; r < M; ++r) {
            H acc = Hi::zero();
            float accf = 0.f;
#pragma unroll
            for (int fi = 0; fi < 2; ++fi) {
#pragma unroll
              for (int i = 0; i < M; ++i) acc = Hi::mad(Hi::kz(co, fo, fi, r * 4 + i), (r & 1) ? d0[fi][i] : s0[fi][i], acc);
#pragma unroll
              for (int gm = 0; gm < 2; ++gm)
#pragma unroll
                for (int i = 0; i < M; ++i)
                  accf = fmaf(co.hi.kz[fo][fi][gm + 1][r * 4 + i], (r & 1) ? d1[fi][gm][i] : s1[fi][gm][i], accf);
            }
            state_store(g, out, &o[(size_t)((fo * M + r) * M * M) * plane], Hi::to_double_plus(Hi::norm(acc), accf));
          }
      }
    }
  }
}

template <class Hi, int M, int TX, int TY, int NT>
cudaError_t launch_hybrid_cfg(const double *in, double *out, const Geom &g, const HybridCoeffs &co, int zchunk,
                              cudaStream_t st) {
  using Sh = HybridShape<M, TX, TY>;
  auto kern = hybrid_step_kernel<Hi, M, TX, TY, NT>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, Sh::SMEM); e != cudaSuccess) return e;
  if (zchunk <= 0) zchunk = 16;
  zchunk = clamp_zchunk(g.zhi - g.zlo, zchunk);
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (g.zhi - g.zlo + zchunk - 1) / zchunk);
  kern<<<grid, NT, Sh::SMEM, st>>>(in, out, g, zchunk, co);
  return cudaGetLastError();
}

}  // namespace hermite
