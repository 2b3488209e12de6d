// Fused half step with the z-pass on the tensor cores (tcgen05).
//
// The half step of a cell is the Kronecker sum of fused.cuh: x-pass on the
// x-edges of a node plane, y-pass on its xy-faces, z-pass per cell.  The
// z-pass is a dense contraction: for every z-item (iy', ix', cell) of a plane
//   D[item][j] = sum_k Y[item][k] B[j][k],   k = (f_in, g, iz), K = 2 NG M,
// where columns j = 0..7 hold the plane's share of the cell below it
// (f_out, r) and j = 8..15 its share of the cell above it (the lower-face
// block of Kz, which equals (-1)^(r+iz) times the upper-face block by the
// reflection symmetry of Hermite interpolation).  This is the mode product of
// the 1-D evolution-and-truncation factor along x3 (Sec. 3.1's Alg. 1/2 and
// Sec. 3.2's evolution folded into Kz), applied to all cells of the tile at
// once as an (items x K) x (K x 16) GEMM.
//
// The x- and y-passes run on the FP32 pipes as in fused.cuh (packed
// fma.rn.f32x2).  The y-pass writes its results straight into the A operand
// of the z-GEMM in shared memory (canonical K-major layout, no swizzle), split
// into pieces of the tensor-core input type:
//   3xTF32:    y = a1 + a2 with a1 = tf32(y), a2 = tf32(y - a1);
//              D = a1 b1 + a1 b2 + a2 b1          (b = b1 + b2 likewise)
//   BF16 x 3:  y = a1 + a2 + a3 with bf16 pieces;
//              D = a1 b1 + a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1
// with FP32 accumulation in tensor memory.  One thread issues the MMAs of a
// plane; they run while the CTA loads and computes the next plane's x-pass;
// then every thread reads its row of D (tcgen05.ld) and completes or starts
// its cells as in fused.cuh.  Every wait on the MMA's mbarrier is bounded: a
// CTA that gives up sets bit 0 of *status, stops, and frees its tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fused.cuh"
#include "tc_ptx.cuh"

namespace hermite {

enum TcKind { kTc3xTF32 = 0, kTcBF16x3 = 1 };

// Polls of the MMA barrier before a CTA gives up (each poll may suspend the
// thread for a short hardware-defined time; this bounds the wait to well
// under a second on GB300, far above the microseconds an MMA group takes).
constexpr uint32_t kTcMaxPolls = 1u << 21;

template <int M, int TX, int TY, int KIND>
struct TcShape {
  using Base = FusedShape<float, M, TX, TY, 2>;
  static constexpr int NG = Base::NG;
  static constexpr int K = 2 * NG * M;                   // (f_in, g, iz)
  static constexpr int ESZ = KIND == kTc3xTF32 ? 4 : 2;  // bytes per input element
  static constexpr int E = 16 / ESZ;                     // elements per core-matrix row
  static constexpr int KSTEP = 2 * E;                    // K of one MMA instruction (32 bytes)
  static constexpr int KP = (K + KSTEP - 1) / KSTEP * KSTEP;
  static constexpr int KC = KP / E;                      // core matrices along K
  static constexpr int NKS = KP / KSTEP;                 // MMA instructions per product
  static constexpr int NC = TX * TY;
  static constexpr int ZROWS = M * M * NC;               // z-items (iy', ix', cell)
  static constexpr int NTILE = (ZROWS + 127) / 128;
  static constexpr int ROWS = NTILE * 128;
  static constexpr int PIECES = KIND == kTc3xTF32 ? 2 : 3;
  static constexpr int SBO = KC * 128;                   // bytes between 8-row groups
  static constexpr int APIECE = ROWS * KP * ESZ;         // bytes of one piece of A
  static constexpr int BPIECE = 16 * KP * ESZ;           // bytes of one piece of B
  static constexpr int TMEM_COLS = NTILE * 16 <= 32 ? 32 : 64;
  // x-pass results [f][iz][iy][a][ix'][ey][ex], one block of XB words per (f, iz, iy).  A warp of
  // y-items spans 8 cells (fx) x 4 iz (below), so that its 4-byte stores of the A pieces fall on
  // (row % 8) * 4 + k % 4: 32 distinct banks.  Its sX reads then differ by iz * M * XB + fx words,
  // and the x-items run (ex, ey, iz, iy, f).  For M = 4, XB = 6 modulo 32 puts all three on
  // distinct banks (M XB = 24 modulo 32 separates the four iz rows of a read, and consecutive
  // (ex, ey) blocks of a store fall 24 words apart).
  static constexpr int XB0 = Base::XB0;
  static constexpr int XB = M == 4 ? XB0 + ((6 - XB0 % 32) + 32) % 32 : Base::XB;
  static constexpr int SX = 2 * M * M * XB;
  static constexpr size_t XBYTES = (size_t)SX * sizeof(float);
  static constexpr size_t AOFF = (XBYTES + 127) / 128 * 128;
  static constexpr size_t BOFF = AOFF + (size_t)PIECES * APIECE;
  static constexpr size_t SMEM = BOFF + (size_t)PIECES * BPIECE;
  static_assert(NTILE * 16 <= 64, "tensor memory columns");
  static_assert(M * M * NC % 8 == 0 || NTILE * 128 > ZROWS, "row groups");
};

// Byte offset of element (row, k) in a canonical K-major, no-swizzle operand
// with `kc` core matrices along K.
__host__ __device__ constexpr int tc_offset(int row, int k, int kc, int e, int esz) {
  return ((row >> 3) * kc + k / e) * 128 + (row & 7) * 16 + (k % e) * esz;
}

// Writes y as its pieces into A (piece stride APIECE bytes) at byte offset off.
template <int KIND, int APIECE>
__device__ __forceinline__ void tc_put(unsigned char *sA, int off, float y) {
  if constexpr (KIND == kTc3xTF32) {
    const float a1 = tc::to_tf32(y);
    const float a2 = tc::to_tf32(y - a1);
    *reinterpret_cast<float *>(sA + off) = a1;
    *reinterpret_cast<float *>(sA + APIECE + off) = a2;
  } else {
    const __nv_bfloat16 a1 = __float2bfloat16_rn(y);
    const float r1 = y - __bfloat162float(a1);
    const __nv_bfloat16 a2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 a3 = __float2bfloat16_rn(r1 - __bfloat162float(a2));
    *reinterpret_cast<__nv_bfloat16 *>(sA + off) = a1;
    *reinterpret_cast<__nv_bfloat16 *>(sA + APIECE + off) = a2;
    *reinterpret_cast<__nv_bfloat16 *>(sA + 2 * APIECE + off) = a3;
  }
}

template <typename TS, int M, int TX, int TY, int NT, int KIND>
__global__ void __launch_bounds__(NT, 2)
    tc_step_kernel(const TS *__restrict__ in, TS *__restrict__ out, const Geom g, int zchunk,
                   const StepCoeffs<float> co, const PackedCoeffs pc, const TcBTable bt, int *status) {
  using Sh = FusedShape<float, M, TX, TY, 2>;
  using T = TcShape<M, TX, TY, KIND>;
  using TC = float;
  constexpr int NYN = Sh::NYN, NA = Sh::NA, NG = Sh::NG;
  constexpr int XPT = (Sh::XITEMS + NT - 1) / NT;
  constexpr int YPT = (Sh::YITEMS + NT - 1) / NT;
  constexpr int XS = NYN * TX;
  static_assert(NT == T::ROWS || NT >= T::ZROWS, "one thread per z-row");
  static_assert(NT % 128 == 0, "whole lane quarters");

  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  float *sX = reinterpret_cast<float *>(smem);
  unsigned char *sA = smem + T::AOFF;
  unsigned char *sB = smem + T::BOFF;

  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = g.zlo + blockIdx.y * zchunk;
  if (z0 >= g.zhi) return;  // uniform over the CTA, before any allocation
  const int z1 = min(z0 + zchunk, g.zhi);
  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const size_t pxy = (size_t)nx * ny;
  const size_t plane = pxy * nz;

  // B pieces, and zeros in the padded K columns of every A row (the y-pass
  // writes only k < K; a NaN left in the padding would poison the row).
  for (int i = threadIdx.x; i < T::PIECES * T::BPIECE / 16; i += NT) reinterpret_cast<uint4 *>(sB)[i] = bt.words[i];
  if constexpr (T::KP > T::K) {
    constexpr int PAD = T::KP - T::K;
    for (int i = threadIdx.x; i < T::PIECES * T::ROWS * PAD; i += NT) {
      const int p = i / (T::ROWS * PAD), rem = i - p * (T::ROWS * PAD);
      const int row = rem / PAD, k = T::K + rem % PAD;
      const int off = p * T::APIECE + tc_offset(row, k, T::KC, T::E, T::ESZ);
      if constexpr (T::ESZ == 4)
        *reinterpret_cast<float *>(sA + off) = 0.f;
      else
        *reinterpret_cast<unsigned short *>(sA + off) = 0;
    }
  }
  tc::fence_async_smem();
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&tslot, T::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  // x-items (as fused_tile)
  const TS *xsrc[XPT];
  int xl[XPT], xr[XPT], xdst[XPT];
#pragma unroll
  for (int k = 0; k < XPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::XITEMS ? e : 0;
    const int ex = t % TX; t /= TX;
    const int ey = t % NYN; t /= NYN;
    const int iz = t % M; t /= M;       // order (ex, ey, iz, iy, f): see TcShape::XB
    const int iy = t % M;
    const int f = t / M;
    const int gy = wrap_index(y0 + s + ey, ny);
    xsrc[k] = in + (size_t)(((f * M + iz) * M + iy) * M) * plane;
    xl[k] = gy * nx + wrap_index(x0 + s + ex, nx);
    xr[k] = gy * nx + wrap_index(x0 + s + ex + 1, nx);
    xdst[k] = e < Sh::XITEMS ? ((f * M + iz) * M + iy) * T::XB + ey * TX + ex : -1;
  }
  // y-items: base of the two edges in sX; byte offsets of the item's A row
  // (r = 0) and of its K column per grade
  int ysrc[YPT], yrow[YPT], ykoff[YPT][NG];
#pragma unroll
  for (int k = 0; k < YPT; ++k) {
    const int e = threadIdx.x + k * NT;
    int t = e < Sh::YITEMS ? e : 0;
    // item order (fx, iz, fy, ix', f): see TcShape::XB
    const int fx = t % TX; t /= TX;
    const int iz = t % M; t /= M;
    const int fy = t % TY; t /= TY;
    const int ixp = t % M;
    const int f = t / M;
    ysrc[k] = e < Sh::YITEMS ? (f * M + iz) * M * T::XB + ixp * XS + fy * TX + fx : -1;
    const int row0 = ixp * T::NC + fy * TX + fx;  // row of r = 0; r adds r * M * NC
    yrow[k] = row0;
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) ykoff[k][gg] = tc_offset(0, (f * NG + gg) * M + iz, T::KC, T::E, T::ESZ);
  }
  // z-row of this thread: (iy', ix', cell) and its output node (-1 outside)
  const int zrow = threadIdx.x;
  int zxy = -1, zcomp = 0;
  if (zrow < T::ZROWS) {
    const int cell = zrow % T::NC, ixp = (zrow / T::NC) % M, iyp = zrow / (T::NC * M);
    const int ox = x0 + cell % TX, oy = y0 + cell / TX;
    zcomp = iyp * M + ixp;
    if (ox < nx && oy < ny) zxy = oy * nx + ox;
  }
  const int warp = threadIdx.x / 32;
  const bool warp_has_rows = warp / 4 < T::NTILE;
  const uint32_t taddr = tmem + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(16 * (warp / 4));

  auto xpass = [&](int p) {
    const size_t zoff = (size_t)wrap_index(z0 + s + p, nz) * pxy;
    TC Lv[XPT][M], Rv[XPT][M];
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
      unsigned long long sd[M];
#pragma unroll
      for (int i = 0; i < M; ++i) sd[i] = pack2f(sv[i], dv[i]);
#pragma unroll
      for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int rp = 0; rp < M / 2; ++rp) {
          unsigned long long acc = 0ull;
#pragma unroll
          for (int i = 0; i < M; ++i) acc = fma2f(pc.gx[a][rp][i], sd[i], acc);
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
    }
  };

  auto ypass = [&]() {
#pragma unroll
    for (int k = 0; k < YPT; ++k) {
      if (ysrc[k] < 0) continue;
      unsigned long long acc2[NG][M / 2 > 0 ? M / 2 : 1];
      TC accr[NG];
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
          const TC *xi = sX + ysrc[k] + iy * T::XB + a * M * XS;
          const TC L = xi[0], R = xi[TX];
          const TC sv = (iy & 1) ? R - L : R + L;
          const TC dv = (iy & 1) ? R + L : R - L;
          const unsigned long long sd = pack2f(sv, dv);
#pragma unroll
          for (int gg = 0; gg < NG; ++gg) {
            const int b = gg - a;
            if (b < 0 || b >= NA) continue;
#pragma unroll
            for (int rp = 0; rp < M / 2; ++rp) acc2[gg][rp] = fma2f(pc.gy[b][rp][iy], sd, acc2[gg][rp]);
            if constexpr (M & 1) accr[gg] = fma(co.gy[b][(M - 1) * 4 + iy], sv, accr[gg]);
          }
        }
      const int rbase = (yrow[k] >> 3) * T::SBO + (yrow[k] & 7) * 16;
      constexpr int RSTEP = (M * T::NC / 8) * T::SBO;  // bytes from row (r, .) to (r + 1, .)
      static_assert((M * T::NC) % 8 == 0, "r rows start on a row group");
#pragma unroll
      for (int gg = 0; gg < NG; ++gg) {
#pragma unroll
        for (int rp = 0; rp < M / 2; ++rp) {
          float lo, hi;
          unpack2f(acc2[gg][rp], lo, hi);
          tc_put<KIND, T::APIECE>(sA, rbase + (2 * rp) * RSTEP + ykoff[k][gg], lo);
          tc_put<KIND, T::APIECE>(sA, rbase + (2 * rp + 1) * RSTEP + ykoff[k][gg], hi);
        }
        if constexpr (M & 1) tc_put<KIND, T::APIECE>(sA, rbase + (M - 1) * RSTEP + ykoff[k][gg], accr[gg]);
      }
    }
  };

  auto issue_mma = [&]() {
    constexpr uint32_t idesc = tc::instr_desc(KIND == kTc3xTF32 ? tc::kFmtTF32 : tc::kFmtBF16, 128, 16);
    const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
    // products (A piece, B piece), largest first
    constexpr int NPROD = KIND == kTc3xTF32 ? 3 : 6;
    constexpr int PA[6] = {0, 0, 1, 0, 1, 2}, PB[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
    for (int t = 0; t < T::NTILE; ++t) {
#pragma unroll
      for (int q = 0; q < NPROD; ++q)
#pragma unroll
        for (int ks = 0; ks < T::NKS; ++ks) {
          const uint64_t da = tc::smem_desc(a0 + PA[q] * T::APIECE + t * 16 * T::SBO + ks * 256, 128, T::SBO);
          const uint64_t db = tc::smem_desc(b0 + PB[q] * T::BPIECE + ks * 256, 128, T::SBO);
          if constexpr (KIND == kTc3xTF32)
            tc::mma_tf32(tmem + 16 * t, da, db, idesc, (q > 0 || ks > 0) ? 1u : 0u);
          else
            tc::mma_bf16(tmem + 16 * t, da, db, idesc, (q > 0 || ks > 0) ? 1u : 0u);
        }
    }
    tc::mma_commit(&mbar);
  };

  float zacc[2][M];
  const int np = z1 - z0 + 1;
  bool failed = false;
  uint32_t failed_phase = 0;
  // debug-build drill: no MMA is issued, so every wait runs out and takes the failure path
  const bool drill = kDebugBuild && g.drill != 0;
  const uint32_t polls = drill ? kDrillPolls : kTcMaxPolls;
  xpass(0);
  __syncthreads();
  for (int p = 0; p < np; ++p) {
    ypass();
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      if (!drill) issue_mma();
    }
    if (p + 1 < np) xpass(p + 1);  // overlaps the MMAs (they read A and B only)
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&mbar, (uint32_t)(p & 1), polls));
    tc::fence_after_sync();
    if (ok && warp_has_rows) {
      float v[16];
      tc::tmem_ld16(taddr, v);
      if (zxy >= 0) {
        if (p > 0) {
          TS *o = out + (size_t)(z0 + p - 1) * pxy + zxy + (size_t)zcomp * plane;
#pragma unroll
          for (int fo = 0; fo < 2; ++fo)
#pragma unroll
            for (int r = 0; r < M; ++r)
              state_store(g, out, &o[(size_t)((fo * M + r) * M * M) * plane],
                          state_from_float<TS>(zacc[fo][r] + v[fo * 4 + r]));
        }
#pragma unroll
        for (int fo = 0; fo < 2; ++fo)
#pragma unroll
          for (int r = 0; r < M; ++r) zacc[fo][r] = v[8 + fo * 4 + r];
      }
    }
    tc::fence_before_sync();
    if (__syncthreads_or(!ok)) {
      failed = true;
      failed_phase = (uint32_t)(p & 1);
      break;
    }
  }
  if (failed) {
    if (threadIdx.x == 0) atomicOr(status, 1);
    // give the MMAs in flight one more bounded chance to finish before the
    // tensor memory they write is released
    tc::mbar_wait(&mbar, failed_phase, polls);
    __syncthreads();
  }
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem, T::TMEM_COLS);
}

template <typename TS, int M, int TX, int TY, int NT, int KIND>
cudaError_t launch_tc_cfg(const TS *in, TS *out, const Geom &g, const StepCoeffs<float> &co, const TcBTable &bt,
                          int zchunk, int *status, cudaStream_t st) {
  using T = TcShape<M, TX, TY, KIND>;
  auto kern = tc_step_kernel<TS, M, TX, TY, NT, KIND>;
  static SmemAttrOnce smem_once;
  if (cudaError_t e = raise_smem_limit(smem_once, kern, T::SMEM); e != cudaSuccess) return e;
  if (zchunk <= 0) zchunk = 16;
  zchunk = clamp_zchunk(g.zhi - g.zlo, zchunk);
  const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  dim3 grid(tiles, (g.zhi - g.zlo + zchunk - 1) / zchunk);
  const PackedCoeffs pc = pack_coeffs(co);
  kern<<<grid, NT, T::SMEM, st>>>(in, out, g, zchunk, co, pc, bt, status);
  return cudaGetLastError();
}

}  // namespace hermite
