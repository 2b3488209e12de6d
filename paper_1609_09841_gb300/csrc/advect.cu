// Advection half step kernels (Eq. 1 with a constant velocity; Sec. 2,
// Sec. 3.1, Alg. 4).  See advect.h for the factorisation.
//
// adv_kron_kernel applies a Kronecker product Gz (x) Gy (x) Gx of R x P
// factors to the 2 x 2 x 2 corner data of every cell:
//   * a CTA owns TX x TY cells in (x1, x2) and walks `zchunk` cells along x3,
//     streaming node layers: each layer of nodes is read from HBM once;
//   * x-pass, per (x1-edge, node row, i3, i2): R outputs from the P values of
//     the two x1-neighbours (coalesced along x1), into shared memory;
//   * y-pass, per (cell column, i3, r1): R outputs from the two node rows,
//     into one of two layer buffers;
//   * z-pass, per (cell, r2, r1): R outputs from the two layer buffers, to
//     the output state (R = M, fused half step) or to the split workspace
//     (R = P, interpolation only).
// Every periodic index is wrapped once: a cell index c < n gives node
// indices c + s + side in [-1, n].
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "advect.h"
#include "packed_f32.cuh"

namespace hermite {

namespace {

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename TS, typename TC, int M, int R, int TX, int TY>
struct KronShape {
  static constexpr int P = 2 * M;
  static constexpr int SX = (TY + 1) * M * M * R * TX;  // [node row][i3][i2][r1][x]
  static constexpr int SY = TY * M * R * R * TX;        // [row][i3][r2][r1][x], two layers
  static constexpr size_t BYTES = ((size_t)SX + 2 * SY) * sizeof(TC);
};

template <typename TS, typename TC, int M, int R, int TX, int TY, int NT, bool WS>
__global__ void __launch_bounds__(NT)
    adv_kron_kernel(const TS *__restrict__ in, void *__restrict__ out_, Geom g, KronCoeffs<TC> co, int zchunk,
                    int z0ws, int nzlws) {
  using S = KronShape<TS, TC, M, R, TX, TY>;
  constexpr int P = S::P;
  constexpr int XI = (TY + 1) * M * M * TX;  // x-pass items per layer: (node row, i3, i2, x)
  constexpr int IT = (XI + NT - 1) / NT;     // per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *sX = reinterpret_cast<TC *>(smem_raw);
  TC *sY = sX + S::SX;
  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const size_t N = (size_t)nx * ny * nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = g.zlo + blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, g.zhi);
  if (zb >= ze) return;  // uniform over the CTA
  const int nl = ze - zb + 1;
  // The x-pass inputs of one node layer, held in registers: the loads of
  // layer L+1 are issued before the y- and z-passes of layer L so that their
  // latency overlaps that work.
  TS pre[IT][P];
  auto load = [&](int L) {
    const int zn = wrap1(zb + s + L, nz);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int e = threadIdx.x + it * NT;
      const int xc = e % TX;
      int t = e / TX;
      const int i2 = t % M;
      t /= M;
      const int i3 = t % M;
      const int yn = t / M;
      if (e >= XI || x0 + xc >= nx || y0 + yn > ny) continue;
      const int yg = wrap1(y0 + yn + s, ny);
      const int xl = wrap1(x0 + xc + s, nx), xr = wrap1(x0 + xc + s + 1, nx);
      const TS *base = in + (size_t)(i3 * M + i2) * M * N + ((size_t)zn * ny + yg) * nx;
#pragma unroll
      for (int i1 = 0; i1 < M; ++i1) {
        pre[it][i1] = __ldg(base + (size_t)i1 * N + xl);
        pre[it][M + i1] = __ldg(base + (size_t)i1 * N + xr);
      }
    }
  };
  load(0);
  for (int L = 0; L < nl; ++L) {
    // x-pass from the registers
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int e = threadIdx.x + it * NT;
      const int xc = e % TX;
      int t = e / TX;
      const int i2 = t % M;
      t /= M;
      const int i3 = t % M;
      const int yn = t / M;
      if (e >= XI || x0 + xc >= nx || y0 + yn > ny) continue;
      TC *dst = sX + ((yn * M + i3) * M + i2) * R * TX + xc;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        TC acc = co.g[0][r][0] * (TC)pre[it][0];
#pragma unroll
        for (int c = 1; c < P; ++c) acc = fma(co.g[0][r][c], (TC)pre[it][c], acc);
        dst[r * TX] = acc;
      }
    }
    if (L + 1 < nl) load(L + 1);
    __syncthreads();
    // y-pass into layer buffer L & 1
    TC *sYL = sY + (L & 1) * S::SY;
    for (int e = threadIdx.x; e < TY * M * R * TX; e += NT) {
      const int xc = e % TX;
      int t = e / TX;
      const int r1 = t % R;
      t /= R;
      const int i3 = t % M;
      const int yc = t / M;
      if (x0 + xc >= nx || y0 + yc >= ny) continue;
      TC v[P];
#pragma unroll
      for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int i2 = 0; i2 < M; ++i2) v[side * M + i2] = sX[((((yc + side) * M + i3) * M + i2) * R + r1) * TX + xc];
      TC *dst = sYL + ((yc * M + i3) * R * R + r1) * TX + xc;
#pragma unroll
      for (int r2 = 0; r2 < R; ++r2) {
        TC acc = co.g[1][r2][0] * v[0];
#pragma unroll
        for (int c = 1; c < P; ++c) acc = fma(co.g[1][r2][c], v[c], acc);
        dst[r2 * R * TX] = acc;
      }
    }
    __syncthreads();
    if (L == 0) continue;
    // z-pass of cell layer zb + L - 1 (layers L - 1 and L)
    const TC *lo = sY + ((L - 1) & 1) * S::SY;
    const int zc = zb + L - 1;
    for (int e = threadIdx.x; e < TY * R * R * TX; e += NT) {
      const int xc = e % TX;
      int t = e / TX;
      const int r1 = t % R;
      t /= R;
      const int r2 = t % R;
      const int yc = t / R;
      const int gx = x0 + xc, gy = y0 + yc;
      if (gx >= nx || gy >= ny) continue;
      TC v[P];
#pragma unroll
      for (int i3 = 0; i3 < M; ++i3) {
        const int o = (((yc * M + i3) * R + r2) * R + r1) * TX + xc;
        v[i3] = lo[o];
        v[M + i3] = sYL[o];
      }
#pragma unroll
      for (int r3 = 0; r3 < R; ++r3) {
        TC acc = co.g[2][r3][0] * v[0];
#pragma unroll
        for (int c = 1; c < P; ++c) acc = fma(co.g[2][r3][c], v[c], acc);
        if constexpr (WS) {
          const size_t slab = (size_t)nzlws * ny * nx;
          reinterpret_cast<TC *>(out_)[(size_t)((r3 * P + r2) * P + r1) * slab +
                                       ((size_t)(zc - z0ws) * ny + gy) * nx + gx] = acc;
        } else {
          reinterpret_cast<TS *>(out_)[(size_t)((r3 * M + r2) * M + r1) * N + ((size_t)zc * ny + gy) * nx + gx] =
              (TS)acc;
        }
      }
    }
  }
}

template <typename TS, typename TC, int M, int R, int TX, int TY, int NT, bool WS>
cudaError_t launch_kron(const TS *in, void *out, const Geom &g, const KronCoeffs<TC> &co, int zchunk, int z0ws,
                        int nzlws, cudaStream_t st) {
  using S = KronShape<TS, TC, M, R, TX, TY>;
  constexpr size_t smem = S::BYTES;
  static_assert(smem <= 227 * 1024, "shared memory of the tile");
  auto kern = adv_kron_kernel<TS, TC, M, R, TX, TY, NT, WS>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, smem); e != cudaSuccess) return e;
  const int nzc = g.zhi - g.zlo;
  int zc = zchunk < 1 ? 1 : zchunk;
  if ((nzc + zc - 1) / zc > 65535) zc = (nzc + 65534) / 65535;  // gridDim.z limit
  if (nzc <= 0 || g.nx <= 0 || g.ny <= 0) return cudaSuccess;
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (nzc + zc - 1) / zc);
  kern<<<grid, NT, smem, st>>>(in, out, g, co, zc, z0ws, nzlws);
  return cudaGetLastError();
}

// Fused half step (R = M), the hot advection kernel.  Same three passes as
// adv_kron_kernel, but
//   * one y-pass layer in shared memory: each node layer is the upper face of
//     the cell below it and the lower face of the cell above it, so the
//     z-pass finishes the pending cell (upper-face columns of Gz) and starts
//     the next one (lower-face columns) from the same layer, keeping the
//     partial sums of its column in registers;
//   * NT = TY * M * TX threads: in the y- and z-passes a thread owns one
//     (row, component, x) column for the whole walk along x3, so its indices
//     are computed once, and loops over the last component index.
template <typename TS, typename TC, int M, int TX, int TY>
struct FusedAdvShape {
  static constexpr int P = 2 * M;
  static constexpr int NT = TY * M * TX;
  static constexpr int SX = (TY + 1) * M * M * M * TX;  // [node row][i3][i2][r1][x]
  static constexpr int SY = TY * M * M * M * TX;        // [row][i3][r2][r1][x], one layer
  static constexpr size_t BYTES = ((size_t)SX + SY) * sizeof(TC);
};

// FP32 kernels: the 1-D factors as duplicated pairs (g, g), so that one
// fma.rn.f32x2 applies a coefficient to two independent inputs (two x-pass
// items, or two r1 rows of the y- and z-passes).
struct AdvPacked {
  unsigned long long g[3][kAdvMaxP][kAdvMaxP];
};
struct NoAdvPacked {};
template <typename TC>
using AdvPackedFor = typename std::conditional<std::is_same<TC, float>::value, AdvPacked, NoAdvPacked>::type;

inline AdvPacked pack_adv(const KronCoeffs<float> &c) {
  AdvPacked p{};
  for (int k = 0; k < 3; ++k)
    for (int r = 0; r < kAdvMaxP; ++r)
      for (int q = 0; q < kAdvMaxP; ++q) p.g[k][r][q] = pack_pair_host(c.g[k][r][q], c.g[k][r][q]);
  return p;
}

template <typename TS, typename TC, int M, int TX, int TY, int XC>
__global__ void __launch_bounds__(TY * M * TX)
    adv_fused_kernel(const TS *__restrict__ in, TS *__restrict__ out, Geom g, KronCoeffs<TC> co, int zchunk,
                     const AdvPackedFor<TC> pk) {
  using S = FusedAdvShape<TS, TC, M, TX, TY>;
  constexpr bool PKA = std::is_same<TC, float>::value;  // packed f32x2 passes
  constexpr int P = S::P, NT = S::NT;
  constexpr int XI = (TY + 1) * M * M * TX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *sX = reinterpret_cast<TC *>(smem_raw);
  TC *sY = sX + S::SX;
  const int nx = g.nx, ny = g.ny, nz = g.nz, s = g.s;
  const size_t N = (size_t)nx * ny * nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = g.zlo + blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, g.zhi);
  if (zb >= ze) return;  // uniform over the CTA
  const int nl = ze - zb + 1;
  // this thread's column: x = xc, row = yc, and component k (i3 in the
  // y-pass, r2 in the z-pass)
  const int xc = threadIdx.x % TX;
  const int k = (threadIdx.x / TX) % M;
  const int yc = threadIdx.x / (TX * M);
  const bool live = x0 + xc < nx && y0 + yc < ny;
  const size_t out_col = (size_t)(k * M) * N + (size_t)(y0 + yc) * nx + (x0 + xc);  // r2 = k
  // NT is a multiple of TX, so every x-pass item of this thread has x = xc
  constexpr int IT = (XI + NT - 1) / NT;
  const bool xin = x0 + xc < nx;
  const int xl = wrap1(x0 + xc + s, nx), xr = wrap1(x0 + xc + s + 1, nx);
  TC acc[M][M];  // pending cell: [r1][r3]
  unsigned long long accp[M / 2 > 0 ? M / 2 : 1][M];  // FP32: rows (2 r1p, 2 r1p + 1) packed
  for (int L = 0; L < nl; ++L) {
    const int zn = wrap1(zb + s + L, nz);
    // x-pass: items (node row, i3, i2, x), IT per thread, taken in chunks of
    // XC items whose loads are all issued before the first product
#pragma unroll
    for (int i0 = 0; i0 < IT; i0 += XC) {
      TS v[XC][P] = {};
#pragma unroll
      for (int j = 0; j < XC; ++j) {
        const int e = threadIdx.x + (i0 + j) * NT;
        const int t = e / TX;
        const int i2 = t % M, i3 = (t / M) % M, yn = t / (M * M);
        if (i0 + j >= IT || e >= XI || !xin || y0 + yn > ny) continue;
        const int yg = wrap1(y0 + yn + s, ny);
        const TS *base = in + (size_t)(i3 * M + i2) * M * N + ((size_t)zn * ny + yg) * nx;
#pragma unroll
        for (int i1 = 0; i1 < M; ++i1) {
          v[j][i1] = __ldg(base + (size_t)i1 * N + xl);
          v[j][M + i1] = __ldg(base + (size_t)i1 * N + xr);
        }
      }
      if constexpr (PKA && XC == 2) {  // the two items on the packed lanes
        bool ok[2];
        int doff[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int e = threadIdx.x + (i0 + j) * NT;
          const int t = e / TX;
          const int i2 = t % M, i3 = (t / M) % M, yn = t / (M * M);
          ok[j] = i0 + j < IT && e < XI && xin && y0 + yn <= ny;
          doff[j] = ((yn * M + i3) * M + i2) * M * TX + xc;
        }
        unsigned long long vv[P];
#pragma unroll
        for (int c = 0; c < P; ++c) vv[c] = pack2f((TC)v[0][c], (TC)v[1][c]);
#pragma unroll
        for (int r = 0; r < M; ++r) {
          unsigned long long a = mul2f(pk.g[0][r][0], vv[0]);
#pragma unroll
          for (int c = 1; c < P; ++c) a = fma2f(pk.g[0][r][c], vv[c], a);
          float lo, hi;
          unpack2f(a, lo, hi);
          if (ok[0]) sX[doff[0] + r * TX] = lo;
          if (ok[1]) sX[doff[1] + r * TX] = hi;
        }
      } else {
#pragma unroll
        for (int j = 0; j < XC; ++j) {
          const int e = threadIdx.x + (i0 + j) * NT;
          const int t = e / TX;
          const int i2 = t % M, i3 = (t / M) % M, yn = t / (M * M);
          if (i0 + j >= IT || e >= XI || !xin || y0 + yn > ny) continue;
          TC *dst = sX + ((yn * M + i3) * M + i2) * M * TX + xc;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            TC a = co.g[0][r][0] * (TC)v[j][0];
#pragma unroll
            for (int c = 1; c < P; ++c) a = fma(co.g[0][r][c], (TC)v[j][c], a);
            dst[r * TX] = a;
          }
        }
      }
    }
    __syncthreads();
    // y-pass: column (yc, i3 = k, x), loop over r1
    if (live) {
      constexpr int RP1 = PKA ? M / 2 : 0;  // r1 pairs on the packed lanes
      if constexpr (PKA) {
#pragma unroll
        for (int rp = 0; rp < RP1; ++rp) {
          unsigned long long vv[P];
#pragma unroll
          for (int side = 0; side < 2; ++side)
#pragma unroll
            for (int i2 = 0; i2 < M; ++i2) {
              const TC *src = sX + ((((yc + side) * M + k) * M + i2) * M + 2 * rp) * TX + xc;
              vv[side * M + i2] = pack2f(src[0], src[TX]);
            }
          TC *dst = sY + ((yc * M + k) * M * M + 2 * rp) * TX + xc;
#pragma unroll
          for (int r2 = 0; r2 < M; ++r2) {
            unsigned long long a = mul2f(pk.g[1][r2][0], vv[0]);
#pragma unroll
            for (int c = 1; c < P; ++c) a = fma2f(pk.g[1][r2][c], vv[c], a);
            float lo, hi;
            unpack2f(a, lo, hi);
            dst[r2 * M * TX] = lo;
            dst[r2 * M * TX + TX] = hi;
          }
        }
      }
#pragma unroll
      for (int r1 = 2 * RP1; r1 < M; ++r1) {
        TC v[P];
#pragma unroll
        for (int side = 0; side < 2; ++side)
#pragma unroll
          for (int i2 = 0; i2 < M; ++i2) v[side * M + i2] = sX[((((yc + side) * M + k) * M + i2) * M + r1) * TX + xc];
        TC *dst = sY + ((yc * M + k) * M * M + r1) * TX + xc;
#pragma unroll
        for (int r2 = 0; r2 < M; ++r2) {
          TC a = co.g[1][r2][0] * v[0];
#pragma unroll
          for (int c = 1; c < P; ++c) a = fma(co.g[1][r2][c], v[c], a);
          dst[r2 * M * TX] = a;
        }
      }
    }
    __syncthreads();
    // z-pass: column (yc, r2 = k, x), loop over r1; this layer is the upper
    // face of cell zb + L - 1 and the lower face of cell zb + L
    if (live) {
      const size_t zoff = (size_t)(zb + L - 1) * ny * nx;
      constexpr int RP1 = PKA ? M / 2 : 0;
      if constexpr (PKA) {
#pragma unroll
        for (int rp = 0; rp < RP1; ++rp) {
          unsigned long long vv[M];
#pragma unroll
          for (int i3 = 0; i3 < M; ++i3) {
            const TC *src = sY + (((yc * M + i3) * M + k) * M + 2 * rp) * TX + xc;
            vv[i3] = pack2f(src[0], src[TX]);
          }
          if (L > 0) {
#pragma unroll
            for (int r3 = 0; r3 < M; ++r3) {
              unsigned long long a = accp[rp][r3];
#pragma unroll
              for (int i3 = 0; i3 < M; ++i3) a = fma2f(pk.g[2][r3][M + i3], vv[i3], a);
              float lo, hi;
              unpack2f(a, lo, hi);
              const size_t o = out_col + (size_t)(r3 * M * M + 2 * rp) * N + zoff;
              out[o] = (TS)lo;
              out[o + N] = (TS)hi;
            }
          }
#pragma unroll
          for (int r3 = 0; r3 < M; ++r3) {
            unsigned long long a = mul2f(pk.g[2][r3][0], vv[0]);
#pragma unroll
            for (int i3 = 1; i3 < M; ++i3) a = fma2f(pk.g[2][r3][i3], vv[i3], a);
            accp[rp][r3] = a;
          }
        }
      }
#pragma unroll
      for (int r1 = 2 * RP1; r1 < M; ++r1) {
        TC v[M];
#pragma unroll
        for (int i3 = 0; i3 < M; ++i3) v[i3] = sY[(((yc * M + i3) * M + k) * M + r1) * TX + xc];
        if (L > 0) {
#pragma unroll
          for (int r3 = 0; r3 < M; ++r3) {
            TC a = acc[r1][r3];
#pragma unroll
            for (int i3 = 0; i3 < M; ++i3) a = fma(co.g[2][r3][M + i3], v[i3], a);
            out[out_col + (size_t)(r3 * M * M + r1) * N + zoff] = (TS)a;
          }
        }
#pragma unroll
        for (int r3 = 0; r3 < M; ++r3) {
          TC a = co.g[2][r3][0] * v[0];
#pragma unroll
          for (int i3 = 1; i3 < M; ++i3) a = fma(co.g[2][r3][i3], v[i3], a);
          acc[r1][r3] = a;
        }
      }
    }
    // the next x-pass writes sX (read by this y-pass: behind the barrier
    // above) and the next y-pass writes sY after the next barrier
  }
}

template <typename TS, typename TC, int M, int TX, int TY, int XC>
cudaError_t launch_fused_adv(const TS *in, TS *out, const Geom &g, const KronCoeffs<TC> &co, int zchunk,
                             cudaStream_t st) {
  using S = FusedAdvShape<TS, TC, M, TX, TY>;
  constexpr size_t smem = S::BYTES;
  static_assert(smem <= 227 * 1024, "shared memory of the tile");
  static_assert(S::NT <= 1024, "threads per CTA");
  auto kern = adv_fused_kernel<TS, TC, M, TX, TY, XC>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, smem); e != cudaSuccess) return e;
  const int nzc = g.zhi - g.zlo;
  int zc = zchunk < 1 ? 1 : zchunk;
  if ((nzc + zc - 1) / zc > 65535) zc = (nzc + 65534) / 65535;  // gridDim.z limit
  if (nzc <= 0 || g.nx <= 0 || g.ny <= 0) return cudaSuccess;
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (nzc + zc - 1) / zc);
  AdvPackedFor<TC> pk{};
  if constexpr (std::is_same<TC, float>::value) pk = pack_adv(co);
  kern<<<grid, S::NT, smem, st>>>(in, out, g, co, zc, pk);
  return cudaGetLastError();
}

}  // namespace

namespace {

// Alg. 4 on the cell polynomials of a slab, CB cells per CTA, then the
// truncation to orders <= m (Sec. 2).  A thread owns one row (cell, jz, jy)
// of P coefficients along x1 in registers (with the row of Ru), so the
// x1-derivative of a stage uses its own registers; the x2- and x3-derivatives
// read the neighbouring rows (jy + 1, jz + 1) from one shared-memory copy of
// the iterate, [jz][jy][jx][cell].  NT = CB * P^2 threads.
template <typename TS, typename TC, int M, int CB>
__global__ void __launch_bounds__(CB * 4 * M * M)
    adv_evolve_kernel(const TC *__restrict__ ws, TS *__restrict__ out, Geom g, int z0, int nzl, TC tau, TC ah0,
                      TC ah1, TC ah2, int q) {
  constexpr int P = 2 * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC *w = reinterpret_cast<TC *>(smem_raw);  // [jz][jy][jx][k]
  const size_t ncell = (size_t)nzl * g.ny * g.nx;
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const int k = threadIdx.x % CB;
  const int row = threadIdx.x / CB;  // jz * P + jy
  const int jy = row % P, jz = row / P;
  const size_t c = (size_t)blockIdx.x * CB + k;
  const bool live = c < ncell;
  TC base[P], cur[P];
#pragma unroll
  for (int jx = 0; jx < P; ++jx) {
    base[jx] = live ? ws[(size_t)(row * P + jx) * ncell + c] : TC(0);
    cur[jx] = base[jx];
  }
  for (int stage = q; stage >= 1; --stage) {  // w <- Ru + (tau / k) L w
    const TC f = tau / (TC)stage;
    const TC f0 = f * ah0, f1 = f * ah1, f2 = f * ah2;
#pragma unroll
    for (int jx = 0; jx < P; ++jx) w[(row * P + jx) * CB + k] = cur[jx];
    __syncthreads();
    TC nxt[P];
#pragma unroll
    for (int jx = 0; jx < P; ++jx) {
      TC d = jx + 1 < P ? f0 * (TC)(jx + 1) * cur[jx + 1] : TC(0);
      if (jy + 1 < P) d = fma(f1 * (TC)(jy + 1), w[((row + 1) * P + jx) * CB + k], d);
      if (jz + 1 < P) d = fma(f2 * (TC)(jz + 1), w[((row + P) * P + jx) * CB + k], d);
      nxt[jx] = base[jx] + d;
    }
    __syncthreads();
#pragma unroll
    for (int jx = 0; jx < P; ++jx) cur[jx] = nxt[jx];
  }
  if (!live || jy > M - 1 || jz > M - 1) return;
#pragma unroll
  for (int i1 = 0; i1 < M; ++i1)
    out[(size_t)((jz * M + jy) * M + i1) * N + (size_t)z0 * g.ny * g.nx + c] = (TS)cur[i1];
}

template <typename TS, typename TC, int M, int CB>
cudaError_t launch_evolve_adv(const TC *ws, TS *out, const Geom &g, int z0, int nzl, const AdvEvolveParams &ep,
                              cudaStream_t st) {
  constexpr int P = 2 * M, NT = CB * P * P;
  static_assert(NT <= 1024, "threads per CTA");
  constexpr size_t smem = (size_t)P * P * P * CB * sizeof(TC);
  auto kern = adv_evolve_kernel<TS, TC, M, CB>;
  static SmemAttrOnce smem_once;  // per instantiation, per device
  if (cudaError_t e = raise_smem_limit(smem_once, kern, smem); e != cudaSuccess) return e;
  const size_t ncell = (size_t)nzl * g.ny * g.nx;
  if (ncell == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((ncell + CB - 1) / CB);
  kern<<<blocks, NT, smem, st>>>(ws, out, g, z0, nzl, (TC)ep.tau, (TC)ep.ah[0], (TC)ep.ah[1], (TC)ep.ah[2], ep.q);
  return cudaGetLastError();
}

// Tile tables (TX x TY cells per CTA), three shapes per order and precision
// for the fused kernel (the plan's schedule picks one) and one for the
// interpolation kernel; every shape stays within 227 KB of shared memory
// (checked at compile time).
template <typename TS, typename TC, int XC>
cudaError_t fused_dispatch_xc(int m, bool b, const TS *i, TS *o, const Geom &g, const KronCoeffs<TC> &co, int zchunk,
                              cudaStream_t st) {
  constexpr bool d = sizeof(TC) == 8;
  // TY rows per CTA (threads TY * M * 32): FP32 8|16, 4|8, 2|4; FP64 4|8, 2|4, 1|2 (m = 1, 2, 3)
  switch (m) {
    case 1:
      return b ? launch_fused_adv<TS, TC, 2, 32, d ? 8 : 16, XC>(i, o, g, co, zchunk, st)
               : launch_fused_adv<TS, TC, 2, 32, d ? 4 : 8, XC>(i, o, g, co, zchunk, st);
    case 2:
      return b ? launch_fused_adv<TS, TC, 3, 32, d ? 4 : 8, XC>(i, o, g, co, zchunk, st)
               : launch_fused_adv<TS, TC, 3, 32, d ? 2 : 4, XC>(i, o, g, co, zchunk, st);
    case 3:
      return b ? launch_fused_adv<TS, TC, 4, 32, d ? 2 : 4, XC>(i, o, g, co, zchunk, st)
               : launch_fused_adv<TS, TC, 4, 32, d ? 1 : 2, XC>(i, o, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

// Shapes whose x-pass items, (TY + 1) M^2 TX of them, split evenly over the
// TY M TX threads: TY divides M, so no thread is left with a partial last
// chunk while the rest of the CTA waits at the barrier.  TY = 2 and 3 for
// m = 1 and 2; for m = 3 the even shapes not in the table above (FP32 one
// row, FP64 four).
template <typename TS, typename TC, int XC>
cudaError_t fused_dispatch_even(int m, const TS *i, TS *o, const Geom &g, const KronCoeffs<TC> &co, int zchunk,
                                cudaStream_t st) {
  constexpr bool d = sizeof(TC) == 8;
  switch (m) {
    case 1: return launch_fused_adv<TS, TC, 2, 32, 2, XC>(i, o, g, co, zchunk, st);
    case 2: return launch_fused_adv<TS, TC, 3, 32, 3, XC>(i, o, g, co, zchunk, st);
    case 3: return launch_fused_adv<TS, TC, 4, 32, d ? 4 : 1, XC>(i, o, g, co, zchunk, st);
  }
  return cudaErrorInvalidValue;
}

// tile 0-3 = 2 * (loads of two x-pass items in flight) + (taller CTA);
// tiles 4, 5 = the even shapes with one or two items in flight
template <typename TS, typename TC>
cudaError_t fused_dispatch(int m, int tile, const void *in, void *out, const Geom &g, const KronCoeffs<TC> &co,
                           int zchunk, cudaStream_t st) {
  const TS *i = static_cast<const TS *>(in);
  TS *o = static_cast<TS *>(out);
  if (tile >= 4)
    return tile == 5 ? fused_dispatch_even<TS, TC, 2>(m, i, o, g, co, zchunk, st)
                     : fused_dispatch_even<TS, TC, 1>(m, i, o, g, co, zchunk, st);
  const bool b = (tile & 1) != 0;
  return tile >= 2 ? fused_dispatch_xc<TS, TC, 2>(m, b, i, o, g, co, zchunk, st)
                   : fused_dispatch_xc<TS, TC, 1>(m, b, i, o, g, co, zchunk, st);
}

template <typename TS, typename TC>
cudaError_t interp_dispatch(int m, const void *in, void *ws, const Geom &g, int z0, int nzl, const KronCoeffs<TC> &co,
                            cudaStream_t st) {
  const TS *i = static_cast<const TS *>(in);
  constexpr bool d = sizeof(TC) == 8;
  Geom gs = g;
  gs.zlo = z0;
  gs.zhi = z0 + nzl;
  const int zc = nzl < 16 ? nzl : 16;
  switch (m) {
    case 1: return launch_kron<TS, TC, 2, 4, 32, 4, 256, true>(i, ws, gs, co, zc, z0, nzl, st);
    case 2: return launch_kron<TS, TC, 3, 6, 32, 2, 256, true>(i, ws, gs, co, zc, z0, nzl, st);
    case 3: return launch_kron<TS, TC, 4, 8, d ? 16 : 32, 1, 256, true>(i, ws, gs, co, zc, z0, nzl, st);
  }
  return cudaErrorInvalidValue;
}

template <typename TS, typename TC>
cudaError_t evolve_dispatch(int m, const void *ws, void *out, const Geom &g, int z0, int nzl,
                            const AdvEvolveParams &ep, cudaStream_t st) {
  const TC *w = static_cast<const TC *>(ws);
  TS *o = static_cast<TS *>(out);
  switch (m) {
    case 1: return launch_evolve_adv<TS, TC, 2, 32>(w, o, g, z0, nzl, ep, st);
    case 2: return launch_evolve_adv<TS, TC, 3, 16>(w, o, g, z0, nzl, ep, st);
    case 3: return launch_evolve_adv<TS, TC, 4, 16>(w, o, g, z0, nzl, ep, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_adv_fused(int m, int tile, int state, int compute, const void *in, void *out, const Geom &g,
                             const KronCoeffs<double> &cd, const KronCoeffs<float> &cf, int zchunk, cudaStream_t st) {
  if (compute == kF64) return fused_dispatch<double, double>(m, tile, in, out, g, cd, zchunk, st);
  if (state == kF64) return fused_dispatch<double, float>(m, tile, in, out, g, cf, zchunk, st);
  return fused_dispatch<float, float>(m, tile, in, out, g, cf, zchunk, st);
}

cudaError_t launch_adv_interp(int m, int state, int compute, const void *in, void *ws, const Geom &g, int z0, int nzl,
                              const KronCoeffs<double> &cd, const KronCoeffs<float> &cf, cudaStream_t st) {
  if (compute == kF64) return interp_dispatch<double, double>(m, in, ws, g, z0, nzl, cd, st);
  if (state == kF64) return interp_dispatch<double, float>(m, in, ws, g, z0, nzl, cf, st);
  return interp_dispatch<float, float>(m, in, ws, g, z0, nzl, cf, st);
}

cudaError_t launch_adv_evolve(int m, int state, int compute, const void *ws, void *out, const Geom &g, int z0,
                              int nzl, const AdvEvolveParams &ep, cudaStream_t st) {
  if (compute == kF64) return evolve_dispatch<double, double>(m, ws, out, g, z0, nzl, ep, st);
  if (state == kF64) return evolve_dispatch<double, float>(m, ws, out, g, z0, nzl, ep, st);
  return evolve_dispatch<float, float>(m, ws, out, g, z0, nzl, ep, st);
}

// Host tables.  Shift(sigma) maps the monomial coefficients b_j of p(xi) to
// those of p(xi + sigma): sum_{j >= r} C(j, r) sigma^(j - r) b_j (binomial
// expansion); the fused factor keeps the rows r <= m.
void build_adv_coeffs(int m, const double h[3], const double a[3], double tau, KronCoeffs<double> *fused,
                      KronCoeffs<double> *interp) {
  const int M = m + 1, P = 2 * M;
  double H[64];
  build_H(m, H);
  *fused = KronCoeffs<double>{};
  *interp = KronCoeffs<double>{};
  for (int k = 0; k < 3; ++k) {
    const long double sigma = (long double)a[k] * tau / h[k];
    for (int r = 0; r < M; ++r)
      for (int c = 0; c < P; ++c) {
        long double acc = 0.0L, binom = 1.0L, pw = 1.0L;  // C(j, r), sigma^(j - r) at j = r
        for (int j = r; j < P; ++j) {
          acc += binom * pw * (long double)H[j * P + c];
          binom = binom * (j + 1) / (j + 1 - r);
          pw *= sigma;
        }
        fused->g[k][r][c] = (double)acc;
      }
    for (int r = 0; r < P; ++r)
      for (int c = 0; c < P; ++c) interp->g[k][r][c] = H[r * P + c];
  }
}

}  // namespace hermite
