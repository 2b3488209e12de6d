// Split pair of the half step (Sec. 3.1 + Sec. 3.2, the two-kernel design):
//   interp_kernel  -- Alg. 2: Ru = (H (x) H (x) H) u_loc for every cell of a
//                     z-slab, written to a workspace Ru[f][jz][jy][jx][cell];
//   evolve_kernel  -- Alg. 4 with q stages (the Horner form of the Taylor
//                     series; q = 4 equals classical RK4 here) for the
//                     wave operator L(u, v) = (v, c^2 Delta u), Delta built
//                     from Alg. 3 applied twice per dimension, then truncation
//                     to the node data of the dual node (Sec. 2).
// The interpolation stages the node planes in shared memory and marches along
// x3 like the fused kernel: H along x1 on x-edges, along x2 on xy-faces, along
// x3 per cell, each with the even/odd butterfly of H's right block.
#include <cuda_runtime.h>

#include "fused.cuh"
#include "hermite_impl.h"

namespace hermite {

template <typename TC, int M, int TX, int TY>
struct InterpShape {
  static constexpr int P = 2 * M;
  static constexpr int NC = M * M * M;
  static constexpr int NXN = TX + 1, NYN = TY + 1, NODES = NXN * NYN;
  static constexpr int SN = 2 * NC * NODES;
  static constexpr int SX = 2 * M * M * P * NYN * TX;  // [f][iz][iy][jx][ey][ex]
  static constexpr int SY = 2 * M * P * P * TY * TX;   // [f][iz][jy][jx][fy][fx]
  static constexpr size_t SMEM = (size_t)(SN + SX + SY) * sizeof(TC);
  static constexpr int ZITEMS = 2 * P * P * TX * TY;   // (f, jy, jx, cell)
};

template <typename TS, typename TC, int M, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
    interp_kernel(const TS *__restrict__ in, TC *__restrict__ ru, const Geom g, int zs0, int nzl,
                  int zchunk, const InterpCoeffs<TC> co) {
  using Sh = InterpShape<TC, M, TX, TY>;
  constexpr int P = Sh::P, NXN = Sh::NXN, NYN = Sh::NYN, NODES = Sh::NODES;
  constexpr int ZPT = (Sh::ZITEMS + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *sN = reinterpret_cast<TC *>(smem_raw);
  TC *sX = sN + Sh::SN;
  TC *sY = sX + Sh::SX;
  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const int tiles_x = (nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = zs0 + blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, zs0 + nzl);
  if (z0 >= z1) return;
  const size_t plane = (size_t)nx * ny * nz;
  const size_t slab = (size_t)nx * ny * nzl;

  TC prev[ZPT][M];
  for (int p = 0; p <= z1 - z0; ++p) {
    const int zn = wrap_index(z0 + s + p, nz);
    for (int e = threadIdx.x; e < Sh::SN; e += NT) {
      const int comp = e / NODES, r = e - comp * NODES;
      const int ly = r / NXN, lx = r - ly * NXN;
      const int gx = wrap_index(x0 + s + lx, nx), gy = wrap_index(y0 + s + ly, ny);
      sN[e] = (TC)__ldg(in + comp * plane + ((size_t)zn * ny + gy) * nx + gx);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * M * M * NYN * TX; e += NT) {  // H along x1
      int t = e;
      const int ex = t % TX; t /= TX;
      const int ey = t % NYN; t /= NYN;
      const int iy = t % M; t /= M;
      const int iz = t % M;
      const int f = t / M;
      const TC *nb = sN + ((f * M + iz) * M + iy) * M * NODES + ey * NXN + ex;
      TC sv[M], dv[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const TC L = nb[i * NODES], R = nb[i * NODES + 1];
        sv[i] = (i & 1) ? R - L : R + L;
        dv[i] = (i & 1) ? R + L : R - L;
      }
      TC *xo = sX + (((f * M + iz) * M + iy) * P) * NYN * TX + ey * TX + ex;
#pragma unroll
      for (int r = 0; r < P; ++r) {
        TC acc = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) acc = fma(co.hr[r][i], (r & 1) ? dv[i] : sv[i], acc);
        xo[r * NYN * TX] = acc;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * M * P * TY * TX; e += NT) {  // H along x2
      int t = e;
      const int fx = t % TX; t /= TX;
      const int fy = t % TY; t /= TY;
      const int jx = t % P; t /= P;
      const int iz = t % M;
      const int f = t / M;
      TC sv[M], dv[M];
#pragma unroll
      for (int iy = 0; iy < M; ++iy) {
        const TC *xi = sX + (((f * M + iz) * M + iy) * P + jx) * NYN * TX + fy * TX + fx;
        const TC L = xi[0], R = xi[TX];
        sv[iy] = (iy & 1) ? R - L : R + L;
        dv[iy] = (iy & 1) ? R + L : R - L;
      }
      TC *yo = sY + (((f * M + iz) * P) * P + jx) * TY * TX + fy * TX + fx;
#pragma unroll
      for (int r = 0; r < P; ++r) {
        TC acc = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) acc = fma(co.hr[r][i], (r & 1) ? dv[i] : sv[i], acc);
        yo[r * P * TY * TX] = acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ZPT; ++k) {  // H along x3, per cell
      const int item = threadIdx.x + k * NT;
      if (item < Sh::ZITEMS) {
        int t = item;
        const int cx = t % TX; t /= TX;
        const int cy = t % TY; t /= TY;
        const int jx = t % P; t /= P;
        const int jy = t % P;
        const int f = t / P;
        TC cur[M];
#pragma unroll
        for (int iz = 0; iz < M; ++iz)
          cur[iz] = sY[((((f * M + iz) * P + jy) * P + jx) * TY + cy) * TX + cx];
        if (p > 0) {
          const int ox = x0 + cx, oy = y0 + cy, oz = z0 + p - 1;
          if (ox < nx && oy < ny) {
            TC sv[M], dv[M];
#pragma unroll
            for (int iz = 0; iz < M; ++iz) {
              const TC L = prev[k][iz], R = cur[iz];
              sv[iz] = (iz & 1) ? R - L : R + L;
              dv[iz] = (iz & 1) ? R + L : R - L;
            }
            const size_t cell = ((size_t)(oz - zs0) * ny + oy) * nx + ox;
#pragma unroll
            for (int r = 0; r < P; ++r) {
              TC acc = 0;
#pragma unroll
              for (int i = 0; i < M; ++i) acc = fma(co.hr[r][i], (r & 1) ? dv[i] : sv[i], acc);
              ru[(size_t)(((f * P + r) * P + jy) * P + jx) * slab + cell] = acc;
            }
          }
        }
#pragma unroll
        for (int iz = 0; iz < M; ++iz) prev[k][iz] = cur[iz];
      }
    }
  }
}

// Evolution: CB cells per CTA, the coefficient tensors of each cell in shared
// memory; w <- Ru + (tau/k) L w for k = q..1 (Alg. 4), L w = (w_v, c^2 Delta w_u).
template <typename TS, typename TC, int M, int CB, int NT>
__global__ void __launch_bounds__(NT)
    evolve_kernel(const TC *__restrict__ ru, TS *__restrict__ out, const Geom g, int zs0, int nzl,
                  const EvolveParams ep) {
  constexpr int P = 2 * M, P3 = P * P * P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *yu = reinterpret_cast<TC *>(smem_raw);  // [CB][P3] each
  TC *yv = yu + CB * P3;
  TC *wu = yv + CB * P3;
  TC *wv = wu + CB * P3;
  TC *tv = wv + CB * P3;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t slab = (size_t)nx * ny * nzl;
  const size_t plane = (size_t)nx * ny * nz;
  const size_t c0 = (size_t)blockIdx.x * CB;
  const int ncell = (int)min((size_t)CB, slab - c0);
  for (int e = threadIdx.x; e < 2 * P3 * CB; e += NT) {
    const int cb = e % CB, comp = e / CB;
    TC v = 0;
    if (cb < ncell) v = ru[(size_t)comp * slab + c0 + cb];
    const int f = comp / P3, j = comp - f * P3;
    (f ? yv : yu)[cb * P3 + j] = v;
    (f ? wv : wu)[cb * P3 + j] = v;
  }
  __syncthreads();
  const TC c2h[3] = {(TC)ep.c2h[0], (TC)ep.c2h[1], (TC)ep.c2h[2]};
  for (int k = ep.q; k >= 1; --k) {
    const TC a = (TC)(ep.tau / k);
    for (int e = threadIdx.x; e < CB * P3; e += NT) {
      const int cb = e / P3, j = e - cb * P3;
      const int jx = j % P, jy = (j / P) % P, jz = j / (P * P);
      const TC *w = wu + cb * P3;
      TC lap = 0;
      if (jx + 2 < P) lap = fma(c2h[0] * (TC)((jx + 1) * (jx + 2)), w[j + 2], lap);
      if (jy + 2 < P) lap = fma(c2h[1] * (TC)((jy + 1) * (jy + 2)), w[j + 2 * P], lap);
      if (jz + 2 < P) lap = fma(c2h[2] * (TC)((jz + 1) * (jz + 2)), w[j + 2 * P * P], lap);
      tv[e] = fma(a, lap, yv[e]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CB * P3; e += NT) wu[e] = fma(a, wv[e], yu[e]);
    __syncthreads();
    TC *t = wv;
    wv = tv;
    tv = t;
  }
  for (int e = threadIdx.x; e < 2 * M * M * M * CB; e += NT) {
    const int cb = e % CB, comp = e / CB;
    if (cb >= ncell) continue;
    const int f = comp / (M * M * M), q = comp - f * M * M * M;
    const int ix = q % M, iy = (q / M) % M, iz = q / (M * M);
    const TC v = (f ? wv : wu)[cb * P3 + (iz * P + iy) * P + ix];
    const size_t cell = c0 + cb;
    const size_t ox = cell % nx, oy = (cell / nx) % ny, oz = zs0 + cell / ((size_t)nx * ny);
    out[(size_t)comp * plane + (oz * ny + oy) * nx + ox] = (TS)v;
  }
}

template <typename TS, typename TC, int M, int TX, int TY, int NT>
static cudaError_t launch_interp_cfg(const TS *in, TC *ru, const Geom &g, int z0, int nzl,
                                     const InterpCoeffs<TC> &co, cudaStream_t st) {
  using Sh = InterpShape<TC, M, TX, TY>;
  auto kern = interp_kernel<TS, TC, M, TX, TY, NT>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, Sh::SMEM); e != cudaSuccess) return e;
  const int zchunk = clamp_zchunk(nzl, 8);
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (nzl + zchunk - 1) / zchunk);
  kern<<<grid, NT, Sh::SMEM, st>>>(in, ru, g, z0, nzl, zchunk, co);
  return cudaGetLastError();
}

template <typename TS, typename TC, int M, int CB, int NT>
static cudaError_t launch_evolve_cfg(const TC *ru, TS *out, const Geom &g, int z0, int nzl,
                                     const EvolveParams &ep, cudaStream_t st) {
  constexpr size_t smem = (size_t)5 * CB * (2 * M) * (2 * M) * (2 * M) * sizeof(TC);
  auto kern = evolve_kernel<TS, TC, M, CB, NT>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, smem); e != cudaSuccess) return e;
  const size_t cells = (size_t)g.nx * g.ny * nzl;
  dim3 grid((unsigned)((cells + CB - 1) / CB));
  kern<<<grid, NT, smem, st>>>(ru, out, g, z0, nzl, ep);
  return cudaGetLastError();
}

template <typename TC>
static InterpCoeffs<TC> cast_interp(const InterpCoeffs<double> &in) {
  InterpCoeffs<TC> o;
  for (int r = 0; r < 8; ++r)
    for (int i = 0; i < 4; ++i) o.hr[r][i] = (TC)in.hr[r][i];
  return o;
}

template <typename TS, typename TC>
static cudaError_t interp_dispatch(int m, const void *in, void *ru, const Geom &g, int z0, int nzl,
                                   const InterpCoeffs<double> &co, cudaStream_t st) {
  const InterpCoeffs<TC> c = cast_interp<TC>(co);
  const TS *i = (const TS *)in;
  TC *r = (TC *)ru;
  switch (m) {
    case 1: return launch_interp_cfg<TS, TC, 2, 8, 8, 256>(i, r, g, z0, nzl, c, st);
    case 2: return launch_interp_cfg<TS, TC, 3, 4, 4, 256>(i, r, g, z0, nzl, c, st);
    case 3: return launch_interp_cfg<TS, TC, 4, 4, 4, 256>(i, r, g, z0, nzl, c, st);
  }
  return cudaErrorInvalidValue;
}

template <typename TS, typename TC>
static cudaError_t evolve_dispatch(int m, const void *ru, void *out, const Geom &g, int z0, int nzl,
                                   const EvolveParams &ep, cudaStream_t st) {
  const TC *r = (const TC *)ru;
  TS *o = (TS *)out;
  switch (m) {
    case 1: return launch_evolve_cfg<TS, TC, 2, 16, 256>(r, o, g, z0, nzl, ep, st);
    case 2: return launch_evolve_cfg<TS, TC, 3, 8, 256>(r, o, g, z0, nzl, ep, st);
    case 3: return launch_evolve_cfg<TS, TC, 4, 4, 256>(r, o, g, z0, nzl, ep, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_interp(int m, int state, int compute, const void *in, void *ru, const Geom &g,
                          int z0, int nzl, const InterpCoeffs<double> &co, cudaStream_t st) {
  if (compute == kF64) return interp_dispatch<double, double>(m, in, ru, g, z0, nzl, co, st);
  if (state == kF64) return interp_dispatch<double, float>(m, in, ru, g, z0, nzl, co, st);
  return interp_dispatch<float, float>(m, in, ru, g, z0, nzl, co, st);
}

cudaError_t launch_evolve(int m, int state, int compute, const void *ru, void *out, const Geom &g,
                          int z0, int nzl, const EvolveParams &ep, cudaStream_t st) {
  if (compute == kF64) return evolve_dispatch<double, double>(m, ru, out, g, z0, nzl, ep, st);
  if (state == kF64) return evolve_dispatch<double, float>(m, ru, out, g, z0, nzl, ep, st);
  return evolve_dispatch<float, float>(m, ru, out, g, z0, nzl, ep, st);
}

}  // namespace hermite
