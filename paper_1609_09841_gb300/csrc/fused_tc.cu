// Instantiations of the tensor-core fused half step (fused_tc.cuh) and the
// host construction of its z-pass B operand.  One tile shape per order:
// 8 x 4 cells for m = 1 (128 z-rows), 8 x 2 for m = 2 (144 rows, two MMA row
// tiles) and m = 3 (256 rows), 256 threads, two CTAs per SM.
#include <cmath>
#include <cstring>

#include "fused_tc.cuh"

namespace hermite {
namespace {

// x rounded to nearest (ties to even) with `bits` significant bits.
double round_sig(double x, int bits) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  int e = 0;
  const double f = std::frexp(x, &e);  // x = f 2^e, 0.5 <= |f| < 1
  return std::ldexp(std::nearbyint(std::ldexp(f, bits)), e - bits);
}

template <int M, int TX, int TY, int KIND>
TcBTable make_btable(const StepCoeffs<double> &co) {
  using T = TcShape<M, TX, TY, KIND>;
  static_assert(T::PIECES * T::BPIECE <= (int)sizeof(TcBTable), "B table size");
  TcBTable bt;
  std::memset(&bt, 0, sizeof bt);
  unsigned char *bytes = reinterpret_cast<unsigned char *>(bt.words);
  const int sig = KIND == kTc3xTF32 ? 11 : 8;  // significant bits of TF32 / BF16
  for (int half = 0; half < 2; ++half)
    for (int fo = 0; fo < 2; ++fo)
      for (int r = 0; r < M; ++r) {
        const int j = half * 8 + fo * 4 + r;
        for (int fi = 0; fi < 2; ++fi)
          for (int gg = 0; gg < T::NG; ++gg)
            for (int iz = 0; iz < M; ++iz) {
              const int k = (fi * T::NG + gg) * M + iz;
              double b = co.kz[fo][fi][gg][r * 4 + iz];
              if (half && ((r + iz) & 1)) b = -b;  // lower-face block: the reflection of the upper one
              double rest = b;
              for (int p = 0; p < T::PIECES; ++p) {
                const double piece = round_sig(rest, sig);
                rest -= piece;
                const float pf = (float)piece;  // exact: at most 11 significant bits
                const int off = p * T::BPIECE + tc_offset(j, k, T::KC, T::E, T::ESZ);
                if (KIND == kTc3xTF32) {
                  std::memcpy(bytes + off, &pf, 4);
                } else {
                  unsigned u;
                  std::memcpy(&u, &pf, 4);
                  const unsigned short h = (unsigned short)(u >> 16);  // exact: 8 significant bits
                  std::memcpy(bytes + off, &h, 2);
                }
              }
            }
      }
  return bt;
}

template <int KIND>
TcBTable btable_kind(int m, const StepCoeffs<double> &co) {
  switch (m) {
    case 1: return make_btable<2, 8, 4, KIND>(co);
    case 2: return make_btable<3, 8, 2, KIND>(co);
    default: return make_btable<4, 8, 2, KIND>(co);
  }
}

template <typename TS, int KIND>
cudaError_t dispatch_tc(int m, const TS *in, TS *out, const Geom &g, const StepCoeffs<float> &co,
                        const TcBTable &bt, int zchunk, int *status, cudaStream_t st) {
  switch (m) {
    case 1: return launch_tc_cfg<TS, 2, 8, 4, 256, KIND>(in, out, g, co, bt, zchunk, status, st);
    case 2: return launch_tc_cfg<TS, 3, 8, 2, 256, KIND>(in, out, g, co, bt, zchunk, status, st);
    case 3: return launch_tc_cfg<TS, 4, 8, 2, 256, KIND>(in, out, g, co, bt, zchunk, status, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

TcBTable build_tc_btable(int m, int kind, const StepCoeffs<double> &co) {
  return kind == kTc3xTF32 ? btable_kind<kTc3xTF32>(m, co) : btable_kind<kTcBF16x3>(m, co);
}

cudaError_t launch_fused_tc(int kind, int m, int state, const void *in, void *out, const Geom &g,
                            const StepCoeffs<float> &co, const TcBTable &bt, int zchunk, int *status,
                            cudaStream_t st) {
  if (state == kF64) {
    const double *i = (const double *)in;
    double *o = (double *)out;
    return kind == kTc3xTF32 ? dispatch_tc<double, kTc3xTF32>(m, i, o, g, co, bt, zchunk, status, st)
                             : dispatch_tc<double, kTcBF16x3>(m, i, o, g, co, bt, zchunk, status, st);
  }
  const float *i = (const float *)in;
  float *o = (float *)out;
  return kind == kTc3xTF32 ? dispatch_tc<float, kTc3xTF32>(m, i, o, g, co, bt, zchunk, status, st)
                           : dispatch_tc<float, kTcBF16x3>(m, i, o, g, co, bt, zchunk, status, st);
}

}  // namespace hermite
