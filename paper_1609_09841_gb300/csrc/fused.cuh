// Fused half-step kernel: interpolation (Sec. 3.1, Alg. 1/2), local evolution
// (Alg. 3/4 with the 4-term series of RK4) and truncation to dual-node data
// (Sec. 2) for a tile of cells, without the cell polynomial ever leaving the
// SM (the monolithic design of Sec. 3.3).
//
// The half step of one cell is written as a Kronecker sum of 1-D factors
// (StepCoeffs in hermite_impl.h), applied dimension by dimension:
//   x-pass  on every x-edge (pair of x-neighbouring nodes) of the node plane:
//           X_a = Gx_a [left; right], a = 0..2            (shared by 4 cells)
//   y-pass  on every xy-face (pair of y-neighbouring edges):
//           Y_g = sum_{a+b=g} Gy_b X_a, g = 0..2          (shared by 2 cells)
//   z-pass  per cell, from the faces of planes z and z+1:
//           out_fo = sum_{fi, g} Kz[fo][fi][g] Y_g(fi)     (fields coupled here)
// Every factor is applied with the even/odd butterfly of its right block.
//
// A CTA owns TX x TY output nodes of the xy-plane and marches along x3 over
// `zchunk` cells (Sec. 3.1's marching along x3: each node plane is loaded and
// its x- and y-passes are done once; the previous plane's face results stay
// in registers for the z-pass of the next cell layer).
#pragma once

#include <cuda_runtime.h>

#include "hermite_impl.h"

namespace hermite {

template <typename TC, int M, int TX, int TY>
struct FusedShape {
  static constexpr int NC = M * M * M;                // components per field
  static constexpr int NXN = TX + 1, NYN = TY + 1;
  static constexpr int NODES = NXN * NYN;             // node plane of the tile (with halo)
  static constexpr int NA = (M == 2) ? 2 : 3;         // non-zero grades of G (G_2 = 0 for m = 1)
  static constexpr int SN = 2 * NC * NODES;           // node data
  static constexpr int SX = 2 * M * M * NA * M * NYN * TX;  // x-pass results per edge
  static constexpr int SY = 2 * 3 * M * M * M * TX * TY;    // y-pass results per face
  static constexpr size_t SMEM = (size_t)(SN + SX + SY) * sizeof(TC);
  static constexpr int ZITEMS = M * M * TX * TY;
};

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <typename TS, typename TC, int M, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
    fused_step_kernel(const TS *__restrict__ in, TS *__restrict__ out, const Geom g, int zchunk,
                      const StepCoeffs<TC> co) {
  using Sh = FusedShape<TC, M, TX, TY>;
  constexpr int NXN = Sh::NXN, NYN = Sh::NYN, NODES = Sh::NODES, NA = Sh::NA;
  constexpr int ZPT = (Sh::ZITEMS + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *sN = reinterpret_cast<TC *>(smem_raw);
  TC *sX = sN + Sh::SN;
  TC *sY = sX + Sh::SX;

  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const int tiles_x = (nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  if (z0 >= nz) return;
  const size_t plane = (size_t)nx * ny * nz;

  TC prev[ZPT][2][3][M];  // face results of the previous node plane, per z-item

  for (int p = 0; p <= z1 - z0; ++p) {
    const int zn = wrap_index(z0 + s + p, nz);
    // (a) node plane of the tile (with a one-node halo in x and y)
    for (int e = threadIdx.x; e < Sh::SN; e += NT) {
      const int comp = e / NODES, r = e - comp * NODES;
      const int ly = r / NXN, lx = r - ly * NXN;
      const int gx = wrap_index(x0 + s + lx, nx), gy = wrap_index(y0 + s + ly, ny);
      sN[e] = (TC)__ldg(in + comp * plane + ((size_t)zn * ny + gy) * nx + gx);
    }
    __syncthreads();
    // (b) x-pass on the TX x (TY+1) x-edges
    for (int e = threadIdx.x; e < 2 * M * M * NYN * TX; e += NT) {
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
      TC *xo = sX + ((((f * M + iz) * M + iy) * NA) * M) * NYN * TX + ey * TX + ex;
#pragma unroll
      for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int r = 0; r < M; ++r) {
          TC acc = 0;
#pragma unroll
          for (int i = 0; i < M; ++i) acc = fma(co.gx[a][r * 4 + i], (r & 1) ? dv[i] : sv[i], acc);
          xo[(a * M + r) * NYN * TX] = acc;
        }
    }
    __syncthreads();
    // (c) y-pass on the TX x TY xy-faces
    for (int e = threadIdx.x; e < 2 * M * M * TY * TX; e += NT) {
      int t = e;
      const int fx = t % TX; t /= TX;
      const int fy = t % TY; t /= TY;
      const int ixp = t % M; t /= M;
      const int iz = t % M;
      const int f = t / M;
      TC sv[NA][M], dv[NA][M];
#pragma unroll
      for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int iy = 0; iy < M; ++iy) {
          const TC *xi = sX + ((((f * M + iz) * M + iy) * NA + a) * M + ixp) * NYN * TX + fy * TX + fx;
          const TC L = xi[0], R = xi[TX];
          sv[a][iy] = (iy & 1) ? R - L : R + L;
          dv[a][iy] = (iy & 1) ? R + L : R - L;
        }
      TC *yo = sY + (size_t)(f * 3 * M + iz) * M * M * TY * TX + fy * TX + fx;
#pragma unroll
      for (int gg = 0; gg < 3; ++gg)
#pragma unroll
        for (int r = 0; r < M; ++r) {
          TC acc = 0;
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const int b = gg - a;
            if (b < 0 || b >= NA) continue;
#pragma unroll
            for (int i = 0; i < M; ++i)
              acc = fma(co.gy[b][r * 4 + i], (r & 1) ? dv[a][i] : sv[a][i], acc);
          }
          // layout [f][g][iz][iy'][ix'][fy][fx]
          yo[((gg * M * M * M) + r * M + ixp) * TY * TX] = acc;
        }
    }
    __syncthreads();
    // (d) z-pass: cell layer z0 + p - 1 from the faces of planes p - 1 and p
#pragma unroll
    for (int k = 0; k < ZPT; ++k) {
      const int item = threadIdx.x + k * NT;
      if (item < Sh::ZITEMS) {
        int t = item;
        const int cx = t % TX; t /= TX;
        const int cy = t % TY; t /= TY;
        const int ixp = t % M;
        const int iyp = t / M;
        TC cur[2][3][M];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int gg = 0; gg < 3; ++gg)
#pragma unroll
            for (int iz = 0; iz < M; ++iz)
              cur[f][gg][iz] =
                  sY[(((((f * 3 + gg) * M + iz) * M + iyp) * M + ixp) * TY + cy) * TX + cx];
        if (p > 0) {
          const int ox = x0 + cx, oy = y0 + cy, oz = z0 + p - 1;
          TC sv[2][3][M], dv[2][3][M];
#pragma unroll
          for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int gg = 0; gg < 3; ++gg)
#pragma unroll
              for (int iz = 0; iz < M; ++iz) {
                const TC L = prev[k][f][gg][iz], R = cur[f][gg][iz];
                sv[f][gg][iz] = (iz & 1) ? R - L : R + L;
                dv[f][gg][iz] = (iz & 1) ? R + L : R - L;
              }
          if (ox < nx && oy < ny) {
            const size_t node = ((size_t)oz * ny + oy) * nx + ox;
#pragma unroll
            for (int fo = 0; fo < 2; ++fo)
#pragma unroll
              for (int r = 0; r < M; ++r) {
                TC acc = 0;
#pragma unroll
                for (int fi = 0; fi < 2; ++fi)
#pragma unroll
                  for (int gg = 0; gg < 3; ++gg)
#pragma unroll
                    for (int i = 0; i < M; ++i)
                      acc = fma(co.kz[fo][fi][gg][r * 4 + i], (r & 1) ? dv[fi][gg][i] : sv[fi][gg][i],
                                acc);
                out[(size_t)(((fo * M + r) * M + iyp) * M + ixp) * plane + node] = (TS)acc;
              }
          }
        }
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int gg = 0; gg < 3; ++gg)
#pragma unroll
            for (int iz = 0; iz < M; ++iz) prev[k][f][gg][iz] = cur[f][gg][iz];
      }
    }
    // The next plane's (a) writes sN only, which (b) has finished reading; its
    // (c) writes sY after two more barriers, so no barrier is needed here.
  }
}

template <typename TS, typename TC, int M, int TX, int TY, int NT>
cudaError_t launch_fused_cfg(const TS *in, TS *out, const Geom &g, const StepCoeffs<TC> &co,
                             int zchunk, cudaStream_t st) {
  using Sh = FusedShape<TC, M, TX, TY>;
  auto kern = fused_step_kernel<TS, TC, M, TX, TY, NT>;
  static bool attr_set = false;  // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (zchunk <= 0) zchunk = 16;
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (g.nz + zchunk - 1) / zchunk);
  kern<<<grid, NT, Sh::SMEM, st>>>(in, out, g, zchunk, co);
  return cudaGetLastError();
}

}  // namespace hermite
