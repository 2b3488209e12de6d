// Fused half-step kernel: interpolation (Sec. 3.1, Alg. 1/2), local evolution
// (Alg. 3/4 with the 4-term series of RK4) and truncation to dual-node data
// (Sec. 2) for a tile of cells, without the cell polynomial ever leaving the
// SM (the monolithic design of Sec. 3.3).
//
// The half step of one cell is written as a Kronecker sum of 1-D factors
// (StepCoeffs in hermite_impl.h), applied dimension by dimension:
//   x-pass  on every x-edge (pair of x-neighbouring nodes) of a node plane:
//           X_a = Gx_a [left; right], a = 0..2            (shared by 4 cells)
//   y-pass  on every xy-face (pair of y-neighbouring edges):
//           Y_g = sum_{a+b=g} Gy_b X_a, g = 0..2          (shared by 2 cells)
//   z-pass  per cell, from the faces of planes z and z+1:
//           out_fo = sum_{fi, g} Kz[fo][fi][g] Y_g(fi)     (fields coupled here)
// Every factor is applied with the even/odd butterfly of its right block.
//
// A CTA owns TX x TY output nodes of the xy-plane and marches along x3 over
// `zchunk` cells (Sec. 3.1's marching along x3): per node plane the x-pass
// reads the node pairs straight from global memory (coalesced along x1, the
// right neighbour of one thread is the left of the next, an L1 hit; each
// thread issues all its loads of the plane before any arithmetic), writes
// its results to shared memory; the y-pass turns them into face results
// (one plane in shared memory); the z-pass adds each plane's share to the
// cell below it (completed and stored) and the cell above it (kept in
// registers until the next plane).  Two barriers per plane.  Every per-item
// index is computed once before the march.
//
// Staged schedules (ST) stage each node plane in shared memory first: one
// tiled bulk tensor copy (TMA) per plane brings the (TY + 1) x BW window of
// every coefficient row, issued by one thread right after the x-pass of the
// previous plane and completed on an mbarrier while that plane's y- and
// z-passes run; the x-pass then reads its node pairs from shared memory.
// Tiles whose window wraps around the periodic boundary, and grids whose row
// pitch the copy engine cannot address, fill the same buffer with plain loads.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "hermite_impl.h"
#include "packed_f32.cuh"
#include "tma_ptx.cuh"

namespace hermite {

// Staging of the x-pass input (ST schedules: ST buffers, 1 or 2).  U: state
// elements per 16 bytes (the copy engine's alignment of the innermost
// coordinate); the window of a tile starts at xa, x0 + s rounded down to a
// multiple of U, and is BW columns wide: TX + 1 nodes after an offset of at
// most U - 1, rounded up to a multiple of U.  With two buffers the copy of
// plane p + 2 goes into the buffer plane p has just left, so each copy has
// two planes' y- and z-passes to land.
template <typename TS, int M, int TX, int TY, int NB = 1>
struct StageShape {
  static constexpr int U = 16 / (int)sizeof(TS);
  static constexpr int BW = (TX + 2 * U - 1) / U * U;
  static constexpr int ROWS = TY + 1;
  static constexpr int NC = 2 * M * M * M;    // coefficient rows of both fields
  static constexpr int BCS = ROWS * BW;       // elements of one coefficient row's window
  static constexpr int ELEMS = NC * BCS;
  static constexpr size_t BYTES = ((size_t)ELEMS * sizeof(TS) + 127) / 128 * 128;  // one buffer
  static constexpr int STRIDE = (int)(BYTES / sizeof(TS));                          // between buffers
  static constexpr size_t TAB_BYTES = ((size_t)BCS * sizeof(int) + 15) / 16 * 16;
  // dynamic shared memory beyond the fused tile's: 128-byte alignment slack,
  // the buffers and the in-plane offsets of the plain-load fill
  static constexpr size_t EXTRA = 128 + NB * BYTES + TAB_BYTES;
};

template <typename TS>
struct StageArgs {
  const CUtensorMap *map;  // the input state as a tensor (valid if map_ok)
  TS *buf;                 // NB buffers of StageShape::STRIDE elements, 128-byte aligned
  int *tab;                // StageShape::BCS in-plane offsets (plain-load fill)
  uint64_t *mbar;          // one mbarrier per buffer: plane p completes phase p / NB of mbar[p % NB]
  int *status;             // bit 0 set when a copy did not complete in time
  int map_ok;
};

// Polls of a staged plane's mbarrier before the CTA gives up (each poll may
// suspend the thread for a while): far beyond any copy's latency.
constexpr uint32_t kStageMaxPolls = 1u << 21;

// L1 prefetch hint (PTX prefetch.global.L1): fetches the line holding p into
// L1 without a register result.  Callers pass addresses they later load.
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// G: largest total grade the kernel carries (2 for the 4-term series of RK4;
// 2m for longer series, whose higher grades the z-pass tables fold in).
template <typename TC, int M, int TX, int TY, int G = 2>
struct FusedShape {
  static constexpr int NYN = TY + 1;
  static constexpr int NA = (M - 1 < G ? M - 1 : G) + 1;   // grades a <= min(m, G) of the 1-D factors
  static constexpr int NG = (2 * (NA - 1) < G ? 2 * (NA - 1) : G) + 1;  // grades of the y-pass results
  // x-pass results [f][iz][iy][a][ix'][ey][ex], one block of XB words per (f, iz, iy).  For the
  // RK4 kernels XB is padded to NYN * TX modulo 32 words, so that a warp whose items run from
  // the last node rows of one block into the next one stores to consecutive banks (the longer
  // series' kernels, at lower occupancy, measured slower with the padding).
  static constexpr int XB0 = NA * M * NYN * TX;
  static constexpr int XPAD = G == 2 ? (((NYN * TX - XB0) % 32) + 32) % 32 : 0;  // (longer series: no gain)
  static constexpr int XB = XB0 + XPAD;
  static constexpr int SX = 2 * M * M * XB;
  static constexpr int SY = 2 * NG * M * M * M * TX * TY;   // y-pass results [f][g][iz][iy'][ix'][fy][fx]
  static constexpr size_t SMEM = (size_t)(SX + SY) * sizeof(TC);  // one plane of y-pass results
  static constexpr int XITEMS = 2 * M * M * NYN * TX;       // (f, iz, iy, edge)
  static constexpr int YITEMS = 2 * M * M * TY * TX;        // (f, iz, ix', face)
  static constexpr int ZITEMS = M * M * TX * TY;            // (iy', ix', cell)
};

// Packed FP32 pairs for fma.rn.f32x2 (two lane-wise fma.rn.f32 in one
// instruction, same rounding as two scalar FMAs).  In the FP32 kernels the
// passes pair outputs that share their input: rows (r, r+1) of the x- and
// y-pass factors act on the butterfly pair (sum, difference), and the two
// output fields of the z-pass act on the same y-pass value.
struct PackedCoeffs {
  unsigned long long gx[kMaxA][2][4];     // (gx[a][(2rp)*4+i], gx[a][(2rp+1)*4+i])
  unsigned long long gy[kMaxA][2][4];     // the same for gy
  unsigned long long kz[2][kMaxG][4][4];  // [f_in][g][r][iz]: (kz[0][f_in][g][r*4+iz], kz[1][f_in][g][r*4+iz])
};

inline PackedCoeffs pack_coeffs(const StepCoeffs<float> &c) {
  PackedCoeffs p{};
  for (int a = 0; a < kMaxA; ++a)
    for (int rp = 0; rp < 2; ++rp)
      for (int i = 0; i < 4; ++i) {
        p.gx[a][rp][i] = pack_pair_host(c.gx[a][(2 * rp) * 4 + i], c.gx[a][(2 * rp + 1) * 4 + i]);
        p.gy[a][rp][i] = pack_pair_host(c.gy[a][(2 * rp) * 4 + i], c.gy[a][(2 * rp + 1) * 4 + i]);
      }
  for (int fi = 0; fi < 2; ++fi)
    for (int g = 0; g < kMaxG; ++g)
      for (int r = 0; r < 4; ++r)
        for (int iz = 0; iz < 4; ++iz)
          p.kz[fi][g][r][iz] = pack_pair_host(c.kz[0][fi][g][r * 4 + iz], c.kz[1][fi][g][r * 4 + iz]);
  return p;
}

// Exact float -> double with integer operations (the hardware widening runs
// on the FP64 pipe at about 1.5 per clock per SM on GB300, so a kernel that
// stores an FP64 state from FP32 results would be bound by it).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u, a = b & 0x7FFFFFFFu;
  unsigned hi, lo;
  if (a >= 0x00800000u && a < 0x7F800000u) {  // normal: rebias the exponent by 1023 - 127
    hi = s | ((a >> 3) + 0x38000000u);
    lo = b << 29;
  } else if (a >= 0x7F800000u) {  // infinity, NaN (payload kept)
    hi = s | 0x7FF00000u | ((a & 0x7FFFFFu) >> 3);
    lo = b << 29;
  } else if (a == 0u) {
    hi = s;
    lo = 0u;
  } else {  // subnormal a * 2^-149: normalise
    const unsigned lz = __clz(a);          // 9..31
    const unsigned mm = (a << lz) << 1;    // mantissa without its leading one
    hi = s | ((905u - lz) << 20) | (mm >> 12);
    lo = mm << 20;
  }
  return __hiloint2double((int)hi, (int)lo);
}

template <typename TS>
__device__ __forceinline__ TS state_from_float(float v) {
  if constexpr (sizeof(TS) == 8)
    return f2d_exact(v);
  else
    return v;
}

// Conversion of a computed value to the state type: exact, and by integer
// operations when FP32 results go to an FP64 state.
template <typename TS, typename TC>
__device__ __forceinline__ TS to_state(TC v) {
  if constexpr (sizeof(TS) == 8 && sizeof(TC) == 4)
    return f2d_exact(v);
  else
    return (TS)v;
}

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One tile: output nodes [x0, x0+TX) x [y0, y0+TY) x [z0, z1) of one grid.
// sX, sY: shared memory of FusedShape<TC, M, TX, TY>::SX and ::SY elements.
// All NT threads of the CTA must call it; it starts and ends without a
// pending barrier (callers that reuse sX, sY or `co` for another tile must
// put a __syncthreads() between the calls).
// PK: FP32 passes with fma.rn.f32x2 on the packed tables `pc` (kernel
// parameters); bitwise the same results as the scalar FMAs.
// PF: prefetch the next plane's x-pass lines into L1 during the y- and
// z-passes.  The batched kernel uses it; the single-grid kernels measured
// slower with it (and with the same hint into L2) and do not.
// ST: staged x-pass input in ST buffers (StageArgs `stg`; 0: not staged);
// returns early, with bit 0 of *stg->status set, if a plane's copy does not
// complete within the poll limit.
template <typename TS, typename TC, int M, int TX, int TY, int NT, int G = 2, bool PK = false, bool PF = false,
          int ST = 0>
__device__ __forceinline__ void fused_tile(const TS *__restrict__ in, TS *__restrict__ out, const Geom &g,
                                           int x0, int y0, int z0, int z1, const StepCoeffs<TC> &co,
                                           TC *__restrict__ sX, TC *__restrict__ sY,
                                           const PackedCoeffs *pc = nullptr, const StageArgs<TS> *stg = nullptr) {
  using Sh = FusedShape<TC, M, TX, TY, G>;
  using Sg = StageShape<TS, M, TX, TY, ST == 2 ? 2 : 1>;
  constexpr int NB = ST == 2 ? 2 : 1;
  constexpr int NYN = Sh::NYN, NA = Sh::NA, NG = Sh::NG;
  constexpr int XPT = (Sh::XITEMS + NT - 1) / NT;
  constexpr int YPT = (Sh::YITEMS + NT - 1) / NT;
  constexpr int ZPT = (Sh::ZITEMS + NT - 1) / NT;
  constexpr int XS = NYN * TX;  // stride of one (f, iz, iy, a, ix') row of sX
  constexpr int YS = TY * TX;   // stride of one (f, g, iz, iy', ix') row of sY
  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const size_t pxy = (size_t)nx * ny;
  const size_t plane = pxy * nz;

  // Staged input window: first column xa (x0 + s rounded down to a multiple
  // of U) and the tile's offset in it; copied by the engine when the window
  // lies inside the grid, else filled with plain loads (wrapping).
  const int xs0 = x0 + s;
  const int xa = xs0 >= 0 ? xs0 / Sg::U * Sg::U : -((-xs0 + Sg::U - 1) / Sg::U) * Sg::U;
  bool use_tma = false;
  if constexpr (ST) use_tma = stg->map_ok && xa >= 0 && xa + Sg::BW <= nx && y0 + s >= 0 && y0 + s + TY < ny;
  // debug-build drill: no copy is issued, so every wait of a copied tile runs out
  const bool drill = kDebugBuild && g.drill != 0;
  const uint32_t polls = drill ? kDrillPolls : kStageMaxPolls;

  // x-items: source planes and in-plane offsets of the edge's two nodes
  // (staged: xl is the left node's place in the window, xr unused).
  const TS *xsrc[XPT];
  int xl[XPT], xr[XPT], xdst[XPT];
#pragma unroll
  for (int k = 0; k < XPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::XITEMS ? e : 0;
    const int ex = t % TX; t /= TX;
    const int ey = t % NYN; t /= NYN;
    const int iy = t % M; t /= M;
    const int iz = t % M;
    const int f = t / M;
    if constexpr (ST) {
      xsrc[k] = nullptr;
      xl[k] = ((((f * M + iz) * M + iy) * M) * Sg::ROWS + ey) * Sg::BW + (xs0 - xa) + ex;
      xr[k] = 0;
    } else {
      const int gy = wrap_index(y0 + s + ey, ny);
      xsrc[k] = in + (size_t)(((f * M + iz) * M + iy) * M) * plane;
      xl[k] = gy * nx + wrap_index(x0 + s + ex, nx);
      xr[k] = gy * nx + wrap_index(x0 + s + ex + 1, nx);
    }
    xdst[k] = e < Sh::XITEMS ? ((f * M + iz) * M + iy) * Sh::XB + ey * TX + ex : -1;
  }
  if constexpr (ST) {
    if (use_tma) {
      if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) tc::mbar_init(stg->mbar + b, 1);
        tma::fence_mbar_init();
        tma::prefetch_map(stg->map);
      }
    } else {
      // in-plane offsets of the window's (row, column) pairs, wrapped
      for (int q = threadIdx.x; q < Sg::BCS; q += NT)
        stg->tab[q] = wrap_index(y0 + s + q / Sg::BW, ny) * nx + wrap_index(xa + q % Sg::BW, nx);
    }
    __syncthreads();
  }
  // one thread starts the copy of plane pp's window into buffer pp % NB
  auto stage_issue = [&](int pp) {
    if constexpr (ST) {
      if (drill) return;
      uint64_t *mb = stg->mbar + pp % NB;
      tc::fence_async_smem();  // the x-pass's reads of the buffer come before the copy's writes
      tma::arrive_expect_tx(mb, (uint32_t)(Sg::ELEMS * sizeof(TS)));
      tma::load_4d(stg->buf + (pp % NB) * Sg::STRIDE, stg->map, xa, y0 + s, wrap_index(z0 + s + pp, nz), 0, mb);
    }
  };
  if constexpr (ST)
    if (use_tma && threadIdx.x == 0)
      for (int pp = 0; pp < NB && pp <= z1 - z0; ++pp) stage_issue(pp);
  // y-items: base of the two edges in sX and of the face in sY.
  int ysrc[YPT], ydst[YPT];
#pragma unroll
  for (int k = 0; k < YPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::YITEMS ? e : 0;
    // item order (fx, fy, ix') when a warp holds whole (f, iz, ix') rows of faces; for smaller
    // tiles (fx, ix', fy), so that the warp's sX reads (ix' stride XS) fall on distinct banks
    int fx, fy, ixp;
    if constexpr (TX * TY < 32) {
      fx = t % TX; t /= TX;
      ixp = t % M; t /= M;
      fy = t % TY; t /= TY;
    } else {
      fx = t % TX; t /= TX;
      fy = t % TY; t /= TY;
      ixp = t % M; t /= M;
    }
    const int iz = t % M;
    const int f = t / M;
    ysrc[k] = (f * M + iz) * M * Sh::XB + ixp * XS + fy * TX + fx;
    ydst[k] = e < Sh::YITEMS ? ((f * NG * M + iz) * M * M + ixp) * YS + fy * TX + fx : -1;
  }
  // z-items: base in sY and the output node's in-plane offset (-1 if outside).
  int zsrc[ZPT], zxy[ZPT], zcomp[ZPT];
#pragma unroll
  for (int k = 0; k < ZPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::ZITEMS ? e : 0;
    const int cx = t % TX; t /= TX;
    const int cy = t % TY; t /= TY;
    const int ixp = t % M;
    const int iyp = t / M;
    zsrc[k] = (iyp * M + ixp) * YS + cy * TX + cx;
    zcomp[k] = iyp * M + ixp;
    const int ox = x0 + cx, oy = y0 + cy;
    zxy[k] = (e < Sh::ZITEMS && ox < nx && oy < ny) ? oy * nx + ox : -1;
  }

  TC zacc[ZPT][2][M];  // pending cell of each z-item: [f_out][r]
  for (int p = 0; p <= z1 - z0; ++p) {
    const size_t zoff = (size_t)wrap_index(z0 + s + p, nz) * pxy;
    // x-pass on the TX x (TY+1) x-edges of node plane z0 + s + p
    TC Lv[XPT][M], Rv[XPT][M];
    bool stage_failed = false;
    if constexpr (ST) {
      TS *bp = stg->buf + (p % NB) * Sg::STRIDE;
      if (use_tma) {
        stage_failed = !tc::mbar_wait(stg->mbar + p % NB, (uint32_t)((p / NB) & 1), polls);
      } else {
        for (int e = threadIdx.x; e < Sg::ELEMS; e += NT)
          bp[e] = state_load(g, in, in + (size_t)(e / Sg::BCS) * plane + zoff + stg->tab[e % Sg::BCS]);
        __syncthreads();
      }
#pragma unroll
      for (int k = 0; k < XPT; ++k) {
        if (xdst[k] < 0) continue;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          Lv[k][i] = (TC)bp[xl[k] + i * Sg::BCS];
          Rv[k][i] = (TC)bp[xl[k] + i * Sg::BCS + 1];
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < XPT; ++k) {
        if (xdst[k] < 0) continue;
        const TS *src = xsrc[k] + zoff;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          Lv[k][i] = (TC)state_load(g, in, src + i * plane + xl[k]);
          Rv[k][i] = (TC)state_load(g, in, src + i * plane + xr[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < XPT; ++k) {
      if (xdst[k] < 0) continue;
      TC sv[M], dv[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const TC L = Lv[k][i], R = Rv[k][i];
        sv[i] = (i & 1) ? R - L : R + L;
        dv[i] = (i & 1) ? R + L : R - L;
      }
      TC *xo = sX + xdst[k];
      if constexpr (PK) {
        unsigned long long sd[M];
#pragma unroll
        for (int i = 0; i < M; ++i) sd[i] = pack2f(sv[i], dv[i]);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
#pragma unroll
          for (int rp = 0; rp < M / 2; ++rp) {
            unsigned long long acc = 0ull;
#pragma unroll
            for (int i = 0; i < M; ++i) acc = fma2f(pc->gx[a][rp][i], sd[i], acc);
            float lo, hi;
            unpack2f(acc, lo, hi);
            xo[(a * M + 2 * rp) * XS] = lo;
            xo[(a * M + 2 * rp + 1) * XS] = hi;
          }
          if constexpr (M & 1) {
            TC acc = 0;
#pragma unroll
            for (int i = 0; i < M; ++i) acc = fma(co.gx[a][(M - 1) * 4 + i], sv[i], acc);
            xo[(a * M + M - 1) * XS] = acc;
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int r = 0; r < M; ++r) {
            TC acc = 0;
#pragma unroll
            for (int i = 0; i < M; ++i) acc = fma(co.gx[a][r * 4 + i], (r & 1) ? dv[i] : sv[i], acc);
            xo[(a * M + r) * XS] = acc;
          }
      }
    }
    if constexpr (ST) {
      if (__syncthreads_or(stage_failed)) {  // a copy never completed: give up on the tile
        if (threadIdx.x == 0) {
          atomicOr(stg->status, 1);
          // copies may still land: one more bounded wait on each before the shared memory is released
          for (int q = p; q < p + NB && q <= z1 - z0; ++q)
            tc::mbar_wait(stg->mbar + q % NB, (uint32_t)((q / NB) & 1), polls);
        }
        __syncthreads();
        return;
      }
      if (use_tma && threadIdx.x == 0 && p + NB <= z1 - z0) stage_issue(p + NB);
    } else {
      __syncthreads();
    }
    if constexpr (PF) {
      // the next plane's x-pass lines into L1 while this plane's y- and
      // z-passes run (the left nodes cover all but one x-node per row)
      if (p < z1 - z0) {
        const size_t znext = (size_t)wrap_index(z0 + s + p + 1, nz) * pxy;
#pragma unroll
        for (int k = 0; k < XPT; ++k) {
          if (xdst[k] < 0) continue;
#pragma unroll
          for (int i = 0; i < M; ++i) prefetch_l1(xsrc[k] + znext + i * plane + xl[k]);
        }
      }
    }
    // y-pass on the TX x TY xy-faces, accumulated grade by grade
#pragma unroll
    for (int k = 0; k < YPT; ++k) {
      if (ydst[k] < 0) continue;
      TC *yo = sY + ydst[k];
      if constexpr (PK) {
        unsigned long long acc2[NG][M / 2 > 0 ? M / 2 : 1];
        TC accr[NG];  // row M - 1 when M is odd
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) {
#pragma unroll
          for (int rp = 0; rp < M / 2; ++rp) acc2[gg][rp] = 0ull;
          accr[gg] = TC(0);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int iy = 0; iy < M; ++iy) {
            const TC *xi = sX + ysrc[k] + iy * Sh::XB + a * M * XS;
            const TC L = xi[0], R = xi[TX];
            const TC sv = (iy & 1) ? R - L : R + L;
            const TC dv = (iy & 1) ? R + L : R - L;
            const unsigned long long sd = pack2f(sv, dv);
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) {
              const int b = gg - a;
              if (b < 0 || b >= NA) continue;
#pragma unroll
              for (int rp = 0; rp < M / 2; ++rp) acc2[gg][rp] = fma2f(pc->gy[b][rp][iy], sd, acc2[gg][rp]);
              if constexpr (M & 1) accr[gg] = fma(co.gy[b][(M - 1) * 4 + iy], sv, accr[gg]);
            }
          }
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) {
#pragma unroll
          for (int rp = 0; rp < M / 2; ++rp) {
            float lo, hi;
            unpack2f(acc2[gg][rp], lo, hi);
            yo[(gg * M * M * M + 2 * rp * M) * YS] = lo;
            yo[(gg * M * M * M + (2 * rp + 1) * M) * YS] = hi;
          }
          if constexpr (M & 1) yo[(gg * M * M * M + (M - 1) * M) * YS] = accr[gg];
        }
      } else {
        TC acc[NG][M];
#pragma unroll
        for (int gg = 0; gg < NG; ++gg)
#pragma unroll
          for (int r = 0; r < M; ++r) acc[gg][r] = TC(0);
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int iy = 0; iy < M; ++iy) {
            const TC *xi = sX + ysrc[k] + iy * Sh::XB + a * M * XS;
            const TC L = xi[0], R = xi[TX];
            const TC sv = (iy & 1) ? R - L : R + L;
            const TC dv = (iy & 1) ? R + L : R - L;
#pragma unroll
            for (int gg = 0; gg < NG; ++gg) {
              const int b = gg - a;
              if (b < 0 || b >= NA) continue;
#pragma unroll
              for (int r = 0; r < M; ++r) acc[gg][r] = fma(co.gy[b][r * 4 + iy], (r & 1) ? dv : sv, acc[gg][r]);
            }
          }
#pragma unroll
        for (int gg = 0; gg < NG; ++gg)
#pragma unroll
          for (int r = 0; r < M; ++r) yo[(gg * M * M * M + r * M) * YS] = acc[gg][r];
      }
    }
    __syncthreads();
    // z-pass.  Plane p is the upper face of cell z0 + p - 1 and the lower face
    // of cell z0 + p.  With E_r, O_r the sums over even and odd iz of
    // Kz[r][iz] Y_iz, the reflection symmetry G[r][(lower, iz)] =
    // (-1)^(r+iz) G[r][(upper, iz)] makes the plane's share of the cell below
    // E_r + O_r and of the cell above (-1)^r (E_r - O_r): the first completes
    // the pending cell, the second starts the next one (kept in registers).
    // The next plane's y-pass overwrites sY only after its x-pass barrier.
#pragma unroll
    for (int k = 0; k < ZPT; ++k) {
      if (zxy[k] < 0) continue;
      TC E[2][M], O[2][M];
      if constexpr (PK) {
        unsigned long long E2[M], O2[M];  // lanes: f_out = 0, 1
#pragma unroll
        for (int r = 0; r < M; ++r) E2[r] = O2[r] = 0ull;
#pragma unroll
        for (int fi = 0; fi < 2; ++fi)
#pragma unroll
          for (int gg = 0; gg < NG; ++gg)
#pragma unroll
            for (int iz = 0; iz < M; ++iz) {
              const TC y = sY[zsrc[k] + ((fi * NG + gg) * M + iz) * M * M * YS];
              const unsigned long long yy = pack2f(y, y);
#pragma unroll
              for (int r = 0; r < M; ++r) {
                if (iz & 1)
                  O2[r] = fma2f(pc->kz[fi][gg][r][iz], yy, O2[r]);
                else
                  E2[r] = fma2f(pc->kz[fi][gg][r][iz], yy, E2[r]);
              }
            }
#pragma unroll
        for (int r = 0; r < M; ++r) {
          unpack2f(E2[r], E[0][r], E[1][r]);
          unpack2f(O2[r], O[0][r], O[1][r]);
        }
      } else {
#pragma unroll
        for (int fo = 0; fo < 2; ++fo)
#pragma unroll
          for (int r = 0; r < M; ++r) E[fo][r] = O[fo][r] = TC(0);
#pragma unroll
        for (int fi = 0; fi < 2; ++fi)
#pragma unroll
          for (int gg = 0; gg < NG; ++gg)
#pragma unroll
            for (int iz = 0; iz < M; ++iz) {
              const TC y = sY[zsrc[k] + ((fi * NG + gg) * M + iz) * M * M * YS];
#pragma unroll
              for (int fo = 0; fo < 2; ++fo)
#pragma unroll
                for (int r = 0; r < M; ++r) {
                  const TC w = co.kz[fo][fi][gg][r * 4 + iz];
                  if (iz & 1)
                    O[fo][r] = fma(w, y, O[fo][r]);
                  else
                    E[fo][r] = fma(w, y, E[fo][r]);
                }
            }
      }
      if (p > 0) {
        TS *o = out + (size_t)(z0 + p - 1) * pxy + zxy[k] + (size_t)zcomp[k] * plane;
#pragma unroll
        for (int fo = 0; fo < 2; ++fo)
#pragma unroll
          for (int r = 0; r < M; ++r)
            state_store(g, out, &o[(size_t)((fo * M + r) * M * M) * plane],
                        to_state<TS>(zacc[k][fo][r] + (E[fo][r] + O[fo][r])));
      }
#pragma unroll
      for (int fo = 0; fo < 2; ++fo)
#pragma unroll
        for (int r = 0; r < M; ++r) zacc[k][fo][r] = (r & 1) ? O[fo][r] - E[fo][r] : E[fo][r] - O[fo][r];
    }
  }
}

// The packed tables travel as a kernel parameter of the FP32 kernels only.
struct NoPackedCoeffs {};
template <typename TC>
using PackedFor = typename std::conditional<std::is_same<TC, float>::value, PackedCoeffs, NoPackedCoeffs>::type;

#define HERMITE_FUSED_KERNEL_BODY                                                                   \
  using Sh = FusedShape<TC, M, TX, TY, G>;                                                          \
  extern __shared__ __align__(16) unsigned char smem_raw[];                                        \
  TC *sX = reinterpret_cast<TC *>(smem_raw);                                                       \
  TC *sY = sX + Sh::SX;                                                                            \
  const int tiles_x = (g.nx + TX - 1) / TX;                                                        \
  const int x0 = (blockIdx.x % tiles_x) * TX;                                                      \
  const int y0 = (blockIdx.x / tiles_x) * TY;                                                      \
  const int z0 = g.zlo + blockIdx.y * zchunk;                                                      \
  if (z0 >= g.zhi) return;                                                                         \
  constexpr bool PK = std::is_same<TC, float>::value;                                              \
  const PackedCoeffs *pp = nullptr;                                                                \
  if constexpr (PK) pp = &pc;                                                                      \
  fused_tile<TS, TC, M, TX, TY, NT, G, PK>(in, out, g, x0, y0, z0, min(z0 + zchunk, g.zhi), co, sX, sY, pp);

template <typename TS, typename TC, int M, int TX, int TY, int NT, int G = 2>
__global__ void __launch_bounds__(NT)
    fused_step_kernel(const TS *__restrict__ in, TS *__restrict__ out, const Geom g, int zchunk,
                      const StepCoeffs<TC> co, const PackedFor<TC> pc) {
  HERMITE_FUSED_KERNEL_BODY
}

// The same kernel with a register cap that lets MINB CTAs share an SM
// (spilling if needed).  Without a second __launch_bounds__ argument ptxas
// allocates fewer registers than with an explicit 1, so the plain kernel
// above is kept for MINB = 1.
template <typename TS, typename TC, int M, int TX, int TY, int NT, int G, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    fused_step_kernel_mb(const TS *__restrict__ in, TS *__restrict__ out, const Geom g, int zchunk,
                         const StepCoeffs<TC> co, const PackedFor<TC> pc) {
  HERMITE_FUSED_KERNEL_BODY
}

#undef HERMITE_FUSED_KERNEL_BODY

// Staged schedules: MINB CTAs per SM, the x-pass input staged in NB shared
// buffers (StageShape), `map` the tensor map of `in` when map_ok.
// Dynamic shared memory: [alignment slack][buffers][offset table][sX][sY].
template <typename TS, typename TC, int M, int TX, int TY, int NT, int G, int MINB, int NB>
__global__ void __launch_bounds__(NT, MINB)
    fused_step_kernel_st(const TS *__restrict__ in, TS *__restrict__ out, const Geom g, int zchunk,
                         const StepCoeffs<TC> co, const PackedFor<TC> pc, const __grid_constant__ CUtensorMap map,
                         int map_ok, int *status) {
  using Sh = FusedShape<TC, M, TX, TY, G>;
  using Sg = StageShape<TS, M, TX, TY, NB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t mbar[NB];
  unsigned char *base = smem_raw + ((128u - (tc::smem_addr(smem_raw) & 127u)) & 127u);
  const StageArgs<TS> sa{&map, reinterpret_cast<TS *>(base), reinterpret_cast<int *>(base + NB * Sg::BYTES), mbar,
                         status, map_ok};
  TC *sX = reinterpret_cast<TC *>(base + NB * Sg::BYTES + Sg::TAB_BYTES);
  TC *sY = sX + Sh::SX;
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = g.zlo + blockIdx.y * zchunk;
  if (z0 >= g.zhi) return;
  constexpr bool PK = std::is_same<TC, float>::value;
  const PackedCoeffs *pp = nullptr;
  if constexpr (PK) pp = &pc;
  fused_tile<TS, TC, M, TX, TY, NT, G, PK, false, NB>(in, out, g, x0, y0, z0, min(z0 + zchunk, g.zhi), co, sX, sY,
                                                       pp, &sa);
}

template <typename TS, typename TC, int M, int TX, int TY, int NT, int G = 2, int MINB = 1>
cudaError_t launch_fused_cfg(const TS *in, TS *out, const Geom &g, const StepCoeffs<TC> &co,
                             int zchunk, cudaStream_t st) {
  using Sh = FusedShape<TC, M, TX, TY, G>;
  auto kern = [] {
    if constexpr (MINB > 1)
      return fused_step_kernel_mb<TS, TC, M, TX, TY, NT, G, MINB>;
    else
      return fused_step_kernel<TS, TC, M, TX, TY, NT, G>;
  }();
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, Sh::SMEM); e != cudaSuccess) return e;
  if (zchunk <= 0) zchunk = 16;
  zchunk = clamp_zchunk(g.zhi - g.zlo, zchunk);
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (g.zhi - g.zlo + zchunk - 1) / zchunk);
  PackedFor<TC> pc{};
  if constexpr (std::is_same<TC, float>::value) pc = pack_coeffs(co);
  kern<<<grid, NT, Sh::SMEM, st>>>(in, out, g, zchunk, co, pc);
  return cudaGetLastError();
}

// Launch of a staged schedule; `status` receives bit 0 if a plane's copy timed
// out.  Two buffers when MINB CTAs with two still fit an SM's shared memory
// (228 KB, 1 KB of it reserved per CTA), else one.  Debug builds take the
// plain-load fill everywhere, so that every read of the state goes through
// the bounds check.
template <typename TS, typename TC, int M, int TX, int TY, int NT, int G, int MINB>
cudaError_t launch_fused_st_cfg(const TS *in, TS *out, const Geom &g, const StepCoeffs<TC> &co, int zchunk,
                                int *status, cudaStream_t st) {
  using Sh = FusedShape<TC, M, TX, TY, G>;
  constexpr int NB = (Sh::SMEM + StageShape<TS, M, TX, TY, 2>::EXTRA + 1024) * MINB <= 228 * 1024 ? 2 : 1;
  using Sg = StageShape<TS, M, TX, TY, NB>;
  constexpr size_t smem = Sh::SMEM + Sg::EXTRA;
  auto kern = fused_step_kernel_st<TS, TC, M, TX, TY, NT, G, MINB, NB>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, smem); e != cudaSuccess) return e;
  if (!status) return cudaErrorInvalidValue;
  if (zchunk <= 0) zchunk = 16;
  zchunk = clamp_zchunk(g.zhi - g.zlo, zchunk);
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (g.zhi - g.zlo + zchunk - 1) / zchunk);
  PackedFor<TC> pc{};
  if constexpr (std::is_same<TC, float>::value) pc = pack_coeffs(co);
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  // debug builds: plain loads (every read bounds-checked), except in a wait drill, where the map
  // is encoded so that the copied tiles wait (for copies that are never issued)
  const int map_ok = (!kDebugBuild || g.drill) &&
                     encode_state_map(&map, in, (int)sizeof(TS), g.nx, g.ny, g.nz, Sg::NC, Sg::BW, Sg::ROWS);
  kern<<<grid, NT, smem, st>>>(in, out, g, zchunk, co, pc, map, map_ok, status);
  return cudaGetLastError();
}

}  // namespace hermite
