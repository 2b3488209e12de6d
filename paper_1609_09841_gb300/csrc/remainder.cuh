// Fused half step in the one-sided Taylor-remainder form, FP64 state, FP32
// arithmetic with exact leading sums.
//
// Hermite interpolation (Sec. 3.1) reproduces every polynomial of degree
// <= 2m+1, so along one dimension the interpolant of the edge data [L; R] is
//   p_L + (interpolant of [0; rho]),   rho_i = R_i - sum_{j>=i} C(j, i) L_j,
// where p_L(xi) = sum_j L_j (xi + 1/2)^j is the degree-m Taylor polynomial of
// the left node (its data at the right node is sum_j C(j, i) L_j) and rho is
// the remainder of that expansion, O((kh)^(m+1)) times the field for resolved
// data.  Every 1-D factor of the half step (interpolate, differentiate 2a
// times (Alg. 3), keep orders <= m) therefore splits into
//   G_a [L; R] = TS_a L + RR_a rho,
// TS_a the derivatives of p_L at the cell centre (binomial/dyadic entries)
// and RR_a the right-node block of G_a.  The large entries of RR_a (sums up
// to 3e4 at m = 3, a = 2) now multiply the small remainder instead of
// O(|u|) node data, so the cancellation that ruins FP32 arithmetic in the
// plain form (fused.cuh, hybrid.cuh) does not occur: the grade >= 1 parts run
// in plain FP32.
//
// The remainders and the grade-0 chain (the x-interpolant X_0 of the node
// data, the y-interpolant Y_0 of X_0, the z-interpolant of Y_0 that is the
// main part of the output) need more than FP32.  The remainder and the Taylor
// shift to the centre have short dyadic coefficients (C(j,i) <= 3, 2^-k), so
// they are evaluated as exact sums (RR_0 rho, small, is added in FP32): each input x of an item is split on a
// power-of-two grid q fixed per item (x = h + l, h an integer multiple of q,
// |h| <= 2^B q, |l| <= q/2); every product c h is then a multiple of q times
// the coefficient's denominator, and every partial sum stays below 2^24 such
// multiples, so the h-sum is exact in FP32.  The l-sum is rounded (relative
// error about 2^-24 of a quantity 2^-B smaller).  One fma.rn.f32x2 carries
// both sums: lane 0 the exact h-sum, lane 1 the l-sum.
//
// Same tiling, marching and shared-memory layout as hybrid.cuh (X_0 and Y_0
// as pairs, X_a and Y_g of grade >= 1 as floats, two planes of y-results).
// Forward steps only: the transposed factors of the adjoint have no
// interpolation structure.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "fused.cuh"
#include "hermite_impl.h"
#include "hybrid.cuh"
#include "packed_f32.cuh"

namespace hermite {

// Grid bits of the exact sums over node data, X_0 or Y_0 (Taylor shift TS_0
// with entries C(j,r) 2^-(j-r), row sums <= 27/8 over the denominator 8;
// remainder with row sums <= 7: 27 * 2^18 < 2^24).
constexpr int kRemBitsIn = 18;

// The split constant of a grid: for |x| <= m, C = 1.5 * 2^(E - B + 23) with
// 2^E > m, so that (x + C) - C rounds x to a multiple of 2^(E - B).
template <int B>
__device__ __forceinline__ float grid_constant(float maxabs) {
  const int eb = (int)((__float_as_uint(maxabs) >> 23) & 0xFFu);  // maxabs < 2^(eb - 126)
  int ec = eb + 24 - B;
  ec = ec < 1 ? 1 : (ec > 254 ? 254 : ec);
  return __uint_as_float(((unsigned)ec << 23) | 0x400000u);
}
// x = hi + lo (|lo| small against hi) split on the grid of C: (h, l), h exact.
__device__ __forceinline__ unsigned long long grid_split(float hi, float lo, float C) {
  const float h = __fsub_rn(__fadd_rn(hi, C), C);
  const float l = __fadd_rn(__fsub_rn(hi, h), lo);
  return pack2f(h, l);
}

// Remainder and Taylor shift of one edge whose left and right data are the
// grid-split pairs Lp[j], Rp[i]:  rho_i (pairs) and TS_0 L (pairs).  The
// coefficients come as pairs from the tables (e2[i][j] = -C(j, i), t2[r][j] =
// C(j, r) 2^-(j-r) in both words), so that each fma.rn.f32x2 reads its pair
// as one operand.
template <int M>
__device__ __forceinline__ void rem_edge(const unsigned long long (&Lp)[M], const unsigned long long (&Rp)[M],
                                         const unsigned long long (&e2)[4][4], const unsigned long long (&t2)[4][4],
                                         unsigned long long (&rho)[M], unsigned long long (&x0)[M]) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    unsigned long long acc = Rp[i];
#pragma unroll
    for (int j = i; j < M; ++j) acc = fma2f(e2[i][j], Lp[j], acc);
    rho[i] = acc;
  }
#pragma unroll
  for (int r = 0; r < M; ++r) {
    unsigned long long acc = Lp[r];
#pragma unroll
    for (int j = r + 1; j < M; ++j) acc = fma2f(t2[r][j], Lp[j], acc);
    x0[r] = acc;
  }
}

// x0 += RR_0 rho, and rho collapsed to floats for the FP32 parts.  rho is
// about (kh)^(m+1)/(m+1)! of the field, so RR_0 rho in FP32 (row sums <= 14.6)
// is off by about 2^-24 x 14.6 |rho|, 2^-39 of the field at kh = 0.08; it is
// merged with the exact Taylor shift by an error-free TwoSum of the leading
// parts, and x0 becomes a normalised pair.  (An exact sum of RR_0 rho on rho's
// own grid measured 3.9e-7 at t = 1 on the 128^3 precision workload against
// 4.7e-7 this way, at 8 % more time.)
template <int M>
__device__ __forceinline__ void rem_add_rr0(const float (&rr0)[4][4], const unsigned long long (&rho)[M],
                                            unsigned long long (&x0)[M], float (&rf)[M]) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float h, l;
    unpack2f(rho[i], h, l);
    rf[i] = h + l;
  }
#pragma unroll
  for (int r = 0; r < M; ++r) {
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) t = fmaf(rr0[r][i], rf[i], t);
    float h0, l0;
    unpack2f(x0[r], h0, l0);
    const df32 q = df_two_sum(h0, t);
    x0[r] = pack2f(q.hi, q.lo + l0);
  }
}

// Grades a = 1 .. NA-1 of a factor in the remainder form, in FP32:
// out[a-1][r] = lam^(2a)/a! (TS_a L + RR_a rho) on the collapsed remainder
// rf (TS_a L is nonzero only for 2a <= m, where it is the main part).  Rows
// (r, r+1) share their input and go through one fma.rn.f32x2.
template <int M, int NA>
__device__ __forceinline__ void rem_grades(const float (&ts)[3][4][4], const float (&rr)[3][4][4],
                                           const unsigned long long (&rr2)[3][2][4], const float (&scale)[3],
                                           const float (&Lf)[M], const float (&rf)[M],
                                           float (&outg)[NA > 1 ? NA - 1 : 1][M]) {
#pragma unroll
  for (int a = 1; a < NA; ++a) {
#pragma unroll
    for (int rp = 0; rp < M / 2; ++rp) {
      unsigned long long acc = 0ull;
#pragma unroll
      for (int i = 0; i < M; ++i) acc = fma2f(rr2[a][rp][i], pack2f(rf[i], rf[i]), acc);
      float t0, t1;
      unpack2f(acc, t0, t1);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j >= 2 * rp + 2 * a) t0 = fmaf(ts[a][2 * rp][j], Lf[j], t0);
        if (j >= 2 * rp + 1 + 2 * a) t1 = fmaf(ts[a][2 * rp + 1][j], Lf[j], t1);
      }
      outg[a - 1][2 * rp] = scale[a] * t0;
      outg[a - 1][2 * rp + 1] = scale[a] * t1;
    }
    if constexpr (M & 1) {
      constexpr int r = M - 1;
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < M; ++i) t = fmaf(rr[a][r][i], rf[i], t);
#pragma unroll
      for (int j = 0; j < M; ++j)
        if (j >= r + 2 * a) t = fmaf(ts[a][r][j], Lf[j], t);
      outg[a - 1][r] = scale[a] * t;
    }
  }
}

template <int M, int TX, int TY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    rem_step_kernel(const double *__restrict__ in, double *__restrict__ out, const Geom g, int zchunk,
                    const RemCoeffs co) {
  using H = df32;  // (h, l) pairs in shared memory
  using Sh = HybridShape<M, TX, TY>;
  constexpr int NYN = Sh::NYN, NA = Sh::NA;
  constexpr int XPT = (Sh::XITEMS + NT - 1) / NT;
  constexpr int YPT = (Sh::YITEMS + NT - 1) / NT;
  constexpr int ZPT = (Sh::ZITEMS + NT - 1) / NT;
  constexpr int XS = NYN * TX, YS = TY * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  H *sX0 = reinterpret_cast<H *>(smem_raw);
  H *sY0 = sX0 + Sh::SX0;  // two planes
  float *sX1 = reinterpret_cast<float *>(sY0 + 2 * Sh::SY0);
  float *sY1 = sX1 + Sh::SX1;  // two planes

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
    ys0[k] = ((f * M + iz) * M * M + ixp) * XS + fy * TX + fx;
    ys1[k] = ((f * M + iz) * M * (NA - 1) * M + ixp) * XS + fy * TX + fx;
    yd0[k] = e < Sh::YITEMS ? ((f * M + iz) * M * M + ixp) * YS + fy * TX + fx : -1;
    yd1[k] = ((f * 2 * M + iz) * M * M + ixp) * YS + fy * TX + fx;
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
    // ---- x-pass: remainder form on the node data ----
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
      df32 Ld[M], Rd[M];
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Ld[i] = df_from(Lv[k][i]);
        Rd[i] = df_from(Rv[k][i]);
        mx = fmaxf(mx, fmaxf(fabsf(Ld[i].hi), fabsf(Rd[i].hi)));
      }
      const float C = grid_constant<kRemBitsIn>(mx);
      unsigned long long Lp[M], Rp[M], rho[M], xa[M];
      float Lf[M], rf[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Lp[i] = grid_split(Ld[i].hi, Ld[i].lo, C);
        Rp[i] = grid_split(Rd[i].hi, Rd[i].lo, C);
        Lf[i] = Ld[i].hi + Ld[i].lo;  // rounded to nearest (hi alone is truncated)
      }
      rem_edge<M>(Lp, Rp, co.edge2, co.ts02, rho, xa);
      rem_add_rr0<M>(co.rr[0][0], rho, xa, rf);
#pragma unroll
      for (int r = 0; r < M; ++r) {
        float h, l;
        unpack2f(xa[r], h, l);
        sX0[xd0[k] + r * XS] = df32{h, l};
      }
      float xg[NA > 1 ? NA - 1 : 1][M];
      rem_grades<M, NA>(co.ts[0], co.rr[0], co.rr2[0], co.scale[0], Lf, rf, xg);
#pragma unroll
      for (int a = 1; a < NA; ++a)
#pragma unroll
        for (int r = 0; r < M; ++r) sX1[xd1[k] + ((a - 1) * M + r) * XS] = xg[a - 1][r];
    }
    __syncthreads();
    // ---- y-pass: remainder form on X_0, FP32 butterflies on X_1, X_2 ----
#pragma unroll
    for (int k = 0; k < YPT; ++k) {
      if (yd0[k] < 0) continue;
      H L0[M], R0[M];
      float sa[NA - 1][M], da[NA - 1][M];
      unsigned long long sda[NA - 1][M];  // (sum, difference) butterfly pairs of X_a, a >= 1
      float mx = 0.f;
#pragma unroll
      for (int iy = 0; iy < M; ++iy) {
        const H *x = sX0 + ys0[k] + iy * M * XS;
        L0[iy] = x[0];
        R0[iy] = x[TX];
        mx = fmaxf(mx, fmaxf(fabsf(L0[iy].hi), fabsf(R0[iy].hi)));
#pragma unroll
        for (int a = 1; a < NA; ++a) {
          const float *xf = sX1 + ys1[k] + (iy * (NA - 1) + a - 1) * M * XS;
          const float Lf = xf[0], Rf = xf[TX];
          sa[a - 1][iy] = (iy & 1) ? Rf - Lf : Rf + Lf;
          da[a - 1][iy] = (iy & 1) ? Rf + Lf : Rf - Lf;
          sda[a - 1][iy] = pack2f(sa[a - 1][iy], da[a - 1][iy]);
        }
      }
      const float C = grid_constant<kRemBitsIn>(mx);
      unsigned long long Lp[M], Rp[M], rho[M], ya[M];
      float Lf[M], rf[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Lp[i] = grid_split(L0[i].hi, L0[i].lo, C);
        Rp[i] = grid_split(R0[i].hi, R0[i].lo, C);
        Lf[i] = L0[i].hi + L0[i].lo;
      }
      rem_edge<M>(Lp, Rp, co.edge2, co.ts02, rho, ya);
      rem_add_rr0<M>(co.rr[1][0], rho, ya, rf);
      float yg[NA > 1 ? NA - 1 : 1][M];
      rem_grades<M, NA>(co.ts[1], co.rr[1], co.rr2[1], co.scale[1], Lf, rf, yg);
      H *y0o = sY0 + (p & 1) * Sh::SY0 + yd0[k];
      float *y1o = sY1 + (p & 1) * Sh::SY1 + yd1[k];
#pragma unroll
      for (int r = 0; r < M; ++r) {
        float h, l;
        unpack2f(ya[r], h, l);
        y0o[r * M * YS] = df32{h, l};
      }
#pragma unroll
      for (int gg = 1; gg < 3; ++gg) {
        // rows (2 rp, 2 rp + 1) share their inputs: (sum, difference) pairs
#pragma unroll
        for (int rp = 0; rp < M / 2; ++rp) {
          unsigned long long acc2 = gg < NA ? pack2f(yg[gg - 1][2 * rp], yg[gg - 1][2 * rp + 1]) : 0ull;
#pragma unroll
          for (int a = 1; a < NA; ++a) {
            const int b = gg - a;
            if (b < 0 || b >= NA) continue;
#pragma unroll
            for (int i = 0; i < M; ++i) acc2 = fma2f(co.gy2[b][rp][i], sda[a - 1][i], acc2);
          }
          float lo, hi;
          unpack2f(acc2, lo, hi);
          y1o[((gg - 1) * M * M * M + 2 * rp * M) * YS] = lo;
          y1o[((gg - 1) * M * M * M + (2 * rp + 1) * M) * YS] = hi;
        }
        if constexpr (M & 1) {
          constexpr int r = M - 1;
          float accf = gg < NA ? yg[gg - 1][r] : 0.f;
#pragma unroll
          for (int a = 1; a < NA; ++a) {
            const int b = gg - a;
            if (b < 0 || b >= NA) continue;
#pragma unroll
            for (int i = 0; i < M; ++i) accf = fmaf(co.gy[b][r * 4 + i], sa[a - 1][i], accf);
          }
          y1o[((gg - 1) * M * M * M + r * M) * YS] = accf;
        }
      }
    }
    __syncthreads();
    // ---- z-pass: remainder form on Y_0 (the output's main part exact), FP32 for Y_1, Y_2 ----
    if (p > 0) {
      const H *c0 = sY0 + (p & 1) * Sh::SY0, *p0 = sY0 + ((p - 1) & 1) * Sh::SY0;
      const float *c1 = sY1 + (p & 1) * Sh::SY1, *p1 = sY1 + ((p - 1) & 1) * Sh::SY1;
#pragma unroll
      for (int k = 0; k < ZPT; ++k) {
        if (zxy[k] < 0) continue;
        unsigned long long z0p[2][M];      // grade-0 z-results per input field (exact pairs)
        float zf[2][3][M];                 // [fi][c][r]: c = 0 collapsed, c >= 1 FP32
#pragma unroll
        for (int fi = 0; fi < 2; ++fi) {
          H L0[M], R0[M];
          float mx = 0.f;
#pragma unroll
          for (int iz = 0; iz < M; ++iz) {
            const int q = zs[k] + (fi * M + iz) * M * M * YS;
            L0[iz] = p0[q];
            R0[iz] = c0[q];
            mx = fmaxf(mx, fmaxf(fabsf(L0[iz].hi), fabsf(R0[iz].hi)));
          }
          const float C = grid_constant<kRemBitsIn>(mx);
          unsigned long long Lp[M], Rp[M], rho[M];
          float Lf[M], rf[M];
#pragma unroll
          for (int i = 0; i < M; ++i) {
            Lp[i] = grid_split(L0[i].hi, L0[i].lo, C);
            Rp[i] = grid_split(R0[i].hi, R0[i].lo, C);
            Lf[i] = L0[i].hi + L0[i].lo;
          }
          rem_edge<M>(Lp, Rp, co.edge2, co.ts02, rho, z0p[fi]);
          rem_add_rr0<M>(co.rr[2][0], rho, z0p[fi], rf);
          float zg[NA > 1 ? NA - 1 : 1][M];
          rem_grades<M, NA>(co.ts[2], co.rr[2], co.rr2[2], co.scale[2], Lf, rf, zg);
#pragma unroll
          for (int r = 0; r < M; ++r) {
            float h, l;
            unpack2f(z0p[fi][r], h, l);
            zf[fi][0][r] = h + l;
#pragma unroll
            for (int c = 1; c < 3; ++c) zf[fi][c][r] = c < NA ? zg[c - 1][r] : 0.f;
          }
        }
        float s1[2][2][M];
        unsigned long long sd1[2][2][M];  // (sum, difference) butterfly pairs of Y_1, Y_2
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int iz = 0; iz < M; ++iz)
#pragma unroll
            for (int gm = 0; gm < 2; ++gm) {
              const int q1 = zs[k] + ((f * 2 + gm) * M + iz) * M * M * YS;
              const float Lf = p1[q1], Rf = c1[q1];
              s1[f][gm][iz] = (iz & 1) ? Rf - Lf : Rf + Lf;
              sd1[f][gm][iz] = pack2f(s1[f][gm][iz], (iz & 1) ? Rf + Lf : Rf - Lf);
            }
        double *o = out + (size_t)(z0 + p - 1) * pxy + zxy[k] + (size_t)zcomp[k] * plane;
        // Kz[g >= 1] on the y-results of grade >= 1, rows (2 rp, 2 rp + 1) in one fma.rn.f32x2
        float yres[2][M];
#pragma unroll
        for (int fo = 0; fo < 2; ++fo) {
#pragma unroll
          for (int rp = 0; rp < M / 2; ++rp) {
            unsigned long long acc2 = 0ull;
#pragma unroll
            for (int fi = 0; fi < 2; ++fi)
#pragma unroll
              for (int gm = 0; gm < 2; ++gm)
#pragma unroll
                for (int i = 0; i < M; ++i) acc2 = fma2f(co.kz2[fo][fi][gm][rp][i], sd1[fi][gm][i], acc2);
            unpack2f(acc2, yres[fo][2 * rp], yres[fo][2 * rp + 1]);
          }
          if constexpr (M & 1) {
            constexpr int r = M - 1;
            float t = 0.f;
#pragma unroll
            for (int fi = 0; fi < 2; ++fi)
#pragma unroll
              for (int gm = 0; gm < 2; ++gm)
#pragma unroll
                for (int i = 0; i < M; ++i) t = fmaf(co.kz[fo][fi][gm + 1][r * 4 + i], s1[fi][gm][i], t);
            yres[fo][r] = t;
          }
        }
#pragma unroll
        for (int fo = 0; fo < 2; ++fo)
#pragma unroll
          for (int r = 0; r < M; ++r) {
            // beta_0[fo][fo] = 1: the exact pair of the own field.  The other
            // field's grade-0 term (tau Z_0[v] in the u update; beta_0 = 0 in the
            // v update) is added as a double-float product: when |v| >> |u| its
            // FP32 rounding would dominate the error of u.  Everything else
            // (grades >= 1, small against the result) in FP32.
            float h, l;
            unpack2f(z0p[fo][r], h, l);
            df32 acc{h, l};
            const float bx = co.beta[fo][1 - fo][0];
            if (bx != 0.f) {
              float hx, lx;
              unpack2f(z0p[1 - fo][r], hx, lx);
              const float p = bx * hx;
              const float e = fmaf(bx, hx, -p);   // exact product error
              const df32 t = df_two_sum(acc.hi, p);
              acc = df_fast_two_sum(t.hi, t.lo + (acc.lo + fmaf(bx, lx, e)));
            }
            float accf = yres[fo][r];
#pragma unroll
            for (int fi = 0; fi < 2; ++fi)
#pragma unroll
              for (int c = 1; c < 3; ++c) accf = fmaf(co.beta[fo][fi][c], zf[fi][c][r], accf);
            state_store(g, out, &o[(size_t)((fo * M + r) * M * M) * plane], f2d_exact(acc.hi) + f2d_exact(acc.lo + accf));
          }
      }
    }
  }
}

template <int M, int TX, int TY, int NT, int MINB = 1>
cudaError_t launch_rem_cfg(const double *in, double *out, const Geom &g, const RemCoeffs &co, int zchunk,
                           cudaStream_t st) {
  using Sh = HybridShape<M, TX, TY>;
  auto kern = rem_step_kernel<M, TX, TY, NT, MINB>;
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
