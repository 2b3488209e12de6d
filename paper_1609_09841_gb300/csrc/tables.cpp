// Host construction of the 1-D operators in exact rational arithmetic.
//
// H (Sec. 3.1) maps the data of a cell edge -- [left node: scaled derivatives
// i = 0..m, right node: i = 0..m] with the nodes at xi = -1/2 and +1/2 -- to
// the P = 2m+2 monomial coefficients of the interpolant in xi = (x - x_c)/h
// (Eq. 3).  The node data of p(xi) = sum c_j xi^j are
// (1/i!) p^(i)(xi0) = sum_j C(j, i) xi0^(j-i) c_j (Eq. 2 in the scaled
// variable); H is the inverse of that matrix, computed here by Gauss-Jordan
// elimination on fractions of 128-bit integers and rounded to double once.
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "hermite_impl.h"

namespace hermite {
namespace {

using i128 = __int128;

i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Q {
  i128 n = 0, d = 1;
  Q() = default;
  Q(i128 num, i128 den = 1) : n(num), d(den) { norm(); }
  void norm() {
    if (d < 0) {
      n = -n;
      d = -d;
    }
    i128 g = gcd128(n, d);
    if (g > 1) {
      n /= g;
      d /= g;
    }
  }
  double to_double() const { return (double)((long double)n / (long double)d); }
};
Q operator-(const Q &a, const Q &b) { return Q(a.n * b.d - b.n * a.d, a.d * b.d); }
Q operator*(const Q &a, const Q &b) { return Q(a.n * b.n, a.d * b.d); }
Q operator/(const Q &a, const Q &b) { return Q(a.n * b.d, a.d * b.n); }

i128 binom(int n, int k) {
  i128 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Exact H for order m, H[j][col], P x P.
void exact_H(int m, Q H[8][8]) {
  const int M = m + 1, P = 2 * m + 2;
  Q A[8][16];
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < 2 * P; ++c) A[r][c] = Q(0);
  for (int side = 0; side < 2; ++side) {
    const Q xi0(side == 0 ? -1 : 1, 2);
    for (int i = 0; i < M; ++i)
      for (int j = i; j < P; ++j) {
        Q p(1);
        for (int e = 0; e < j - i; ++e) p = p * xi0;
        A[side * M + i][j] = Q(binom(j, i)) * p;
      }
  }
  for (int r = 0; r < P; ++r) A[r][P + r] = Q(1);
  for (int col = 0; col < P; ++col) {
    int piv = col;
    while (A[piv][col].n == 0) ++piv;
    if (piv != col)
      for (int c = 0; c < 2 * P; ++c) {
        Q t = A[col][c];
        A[col][c] = A[piv][c];
        A[piv][c] = t;
      }
    const Q p = A[col][col];
    for (int c = 0; c < 2 * P; ++c) A[col][c] = A[col][c] / p;
    for (int r = 0; r < P; ++r) {
      if (r == col || A[r][col].n == 0) continue;
      const Q f = A[r][col];
      for (int c = 0; c < 2 * P; ++c) A[r][c] = A[r][c] - f * A[col][c];
    }
  }
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c) H[r][c] = A[r][P + c];
}

}  // namespace

void build_H(int m, double *H) {
  const int P = 2 * m + 2;
  Q Hq[8][8];
  exact_H(m, Hq);
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c) H[r * P + c] = Hq[r][c].to_double();
}

void build_interp_coeffs(int m, InterpCoeffs<double> *out) {
  const int M = m + 1, P = 2 * m + 2;
  Q Hq[8][8];
  exact_H(m, Hq);
  for (int r = 0; r < 8; ++r)
    for (int i = 0; i < 4; ++i) out->hr[r][i] = (r < P && i < M) ? Hq[r][M + i].to_double() : 0.0;
}

// G_a[r][col] = (r+2a)!/r! H[r+2a][col] (zero when r + 2a > 2m+1): the
// coefficients of order r <= m of d^{2a}/dxi^{2a} applied to the interpolant
// (Alg. 3 twice per power of the Laplacian, then truncation of Sec. 2).
void build_step_coeffs(int m, const double h[3], double c, double tau, int mode, int q,
                       StepCoeffs<double> *out) {
  const bool adjoint = mode == kAdjoint;
  const int M = m + 1, P = 2 * m + 2;
  Q Hq[8][8];
  exact_H(m, Hq);
  // G_a = lam^(2a)/a! T1 (d^2/dxi^2)^a H for a <= m (higher powers vanish on
  // degree 2m+1), per dimension.
  double G[3][kMaxA][4][8];  // [dim][a][r][col]
  for (int k = 0; k < 3; ++k) {
    const double lam2 = (c * tau / h[k]) * (c * tau / h[k]);
    double scale = 1.0;  // lam2^a / a!
    for (int a = 0; a < kMaxA; ++a) {
      if (a > 0) scale *= lam2 / a;
      for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 8; ++col) {
          double v = 0.0;
          if (r < M && col < P && r + 2 * a < P) {
            i128 fac = 1;
            for (int qq = r + 1; qq <= r + 2 * a; ++qq) fac *= qq;
            v = (Q(fac) * Hq[r + 2 * a][col]).to_double() * scale;
          }
          G[k][a][r][col] = v;
        }
    }
  }
  // Right block (forward) or transposed left block (adjoint).
  double GR[3][kMaxA][16];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < kMaxA; ++a)
      for (int r = 0; r < 4; ++r)
        for (int i = 0; i < 4; ++i) {
          double v = 0.0;
          if (r < M && i < M) v = adjoint ? G[k][a][i][r] : G[k][a][r][M + i];
          GR[k][a][r * 4 + i] = v;
        }
  // Field coupling of the q-term Taylor series E = sum_{k<=q} (tau L)^k / k!,
  // L = [[0, I], [c^2 Delta, 0]], L^2 = c^2 Delta on both fields, written per
  // grade s of Lambda^s = (tau^2 c^2 Delta)^s = s! sum_{a+b+c=s} prod_k
  // (lam_k^2 d^2/dxi_k^2)^{a_k} / a_k!:
  //   E_uu = E_vv = sum_{2s <= q} Lambda^s / (2s)!
  //   E_uv = tau sum_{2s+1 <= q} Lambda^s / (2s+1)!
  //   E_vu = tau^-1 sum_{1 <= s, 2s-1 <= q} Lambda^s / (2s-1)!
  // so beta_s = s! times those coefficients.  (q = 4: uu = (1, 1/2, 1/12),
  // uv = tau (1, 1/6), vu = (0, 1, 1/3) / tau.)
  const int A = m < 3 ? m : 3;                 // largest grade per dimension
  int S = (q + 1) / 2;                         // largest total grade with a non-zero beta
  if (S > 3 * A) S = 3 * A;
  double beta[2][2][3 * kMaxA];
  for (int s = 0; s < 3 * kMaxA; ++s) {
    double fs = 1.0;  // s!
    for (int t = 2; t <= s; ++t) fs *= t;
    auto inv_fact = [](int n) {
      double v = 1.0;
      for (int t = 2; t <= n; ++t) v /= t;
      return v;
    };
    const double uu = (s <= S && 2 * s <= q) ? fs * inv_fact(2 * s) : 0.0;
    const double uv = (s <= S && 2 * s + 1 <= q) ? tau * fs * inv_fact(2 * s + 1) : 0.0;
    const double vu = (s >= 1 && s <= S && 2 * s - 1 <= q) ? fs * inv_fact(2 * s - 1) / tau : 0.0;
    beta[0][0][s] = uu;
    beta[1][1][s] = uu;
    beta[0][1][s] = adjoint ? vu : uv;
    beta[1][0][s] = adjoint ? uv : vu;
  }
  // Every term of grade s carries prod_k lam_k^(2 a_k), proportional to
  // c^(2s); beta does not depend on c.  Hence dS/dc is the same sum with
  // beta_s replaced by (2 s / c) beta_s.
  if (mode == kDc)
    for (int fo = 0; fo < 2; ++fo)
      for (int fi = 0; fi < 2; ++fi)
        for (int s = 0; s < 3 * kMaxA; ++s) beta[fo][fi][s] *= 2.0 * s / c;
  for (int a = 0; a < kMaxA; ++a)
    for (int qq = 0; qq < 16; ++qq) {
      out->gx[a][qq] = GR[0][a][qq];
      out->gy[a][qq] = GR[1][a][qq];
    }
  // y-pass results of grade g <= min(2A, S) exist; fold the z factors of
  // grade c <= min(A, S - g) into Kz[g].
  for (int fo = 0; fo < 2; ++fo)
    for (int fi = 0; fi < 2; ++fi)
      for (int g = 0; g < kMaxG; ++g)
        for (int qq = 0; qq < 16; ++qq) {
          double v = 0.0;
          if (g <= 2 * A && g <= S)
            for (int cz = 0; cz <= A && g + cz <= S; ++cz) v += beta[fo][fi][g + cz] * GR[2][cz][qq];
          out->kz[fo][fi][g][qq] = v;
        }
}

// Remainder form of the 1-D factors (remainder.cuh).  With p_L(xi) =
// sum_j L_j (xi + 1/2)^j the left node's Taylor polynomial of degree m, whose
// data at the right node are sum_j C(j, i) L_j, linearity and the exactness of
// Hermite interpolation on polynomials of degree <= 2m+1 give
// G_a [L; R] = G_a [L; T L] + G_a [0; rho] = ts_a L + rr_a rho, where
//   ts_a[r][j] = j!/(j-2a)! C(j-2a, r) 2^-(j-2a-r)   (coefficient of xi^r of
//                (d/dxi)^(2a) p_L; zero unless j >= r + 2a)
//   rr_a[r][i] = a!/lam^(2a) G_a[r][right node, i]
// and scale_a = lam^(2a)/a!.  ts and rr are dyadic rationals, exact in float.
void build_rem_coeffs(int m, const double h[3], double c, double tau, const StepCoeffs<float> &f32,
                      RemCoeffs *out) {
  const int M = m + 1, P = 2 * m + 2;
  Q Hq[8][8];
  exact_H(m, Hq);
  *out = RemCoeffs{};
  for (int d = 0; d < 3; ++d) {
    const double lam2 = (c * tau / h[d]) * (c * tau / h[d]);
    double scale = 1.0;
    for (int a = 0; a < 3; ++a) {
      if (a > 0) scale *= lam2 / a;
      for (int r = 0; r < M; ++r) {
        for (int i = 0; i < M; ++i) {
          double v = 0.0;
          if (r + 2 * a < P) {
            i128 fac = 1;
            for (int qq = r + 1; qq <= r + 2 * a; ++qq) fac *= qq;
            v = (Q(fac) * Hq[r + 2 * a][M + i]).to_double();
          }
          out->rr[d][a][r][i] = (float)v;
        }
        for (int j = 0; j < M; ++j) {
          double v = 0.0;
          if (j >= r + 2 * a) {
            i128 fac = 1;
            for (int qq = j - 2 * a + 1; qq <= j; ++qq) fac *= qq;   // j!/(j-2a)!
            v = (Q(fac * binom(j - 2 * a, r), (i128)1 << (j - 2 * a - r))).to_double();
          }
          out->ts[d][a][r][j] = (float)v;
        }
      }
      out->scale[d][a] = (float)scale;
    }
  }
  // RK4 (the 4-term series): uu = vv = (1, 1/2, 1/12), uv = tau (1, 1/6, 0), vu = (0, 1, 1/3) / tau
  const double b_uu[3] = {1.0, 0.5, 1.0 / 12}, b_uv[3] = {tau, tau / 6, 0.0}, b_vu[3] = {0.0, 1.0 / tau, 1.0 / (3 * tau)};
  for (int k = 0; k < 3; ++k) {
    out->beta[0][0][k] = (float)b_uu[k];
    out->beta[1][1][k] = (float)b_uu[k];
    out->beta[0][1][k] = (float)b_uv[k];
    out->beta[1][0][k] = (float)b_vu[k];
  }
  for (int b = 0; b < 3; ++b)
    for (int qq = 0; qq < 16; ++qq) out->gy[b][qq] = f32.gy[b][qq];
  for (int fo = 0; fo < 2; ++fo)
    for (int fi = 0; fi < 2; ++fi)
      for (int g = 0; g < 3; ++g)
        for (int qq = 0; qq < 16; ++qq) out->kz[fo][fi][g][qq] = f32.kz[fo][fi][g][qq];
  auto pair = [](float lo, float hi) {
    unsigned a, b;
    std::memcpy(&a, &lo, 4);
    std::memcpy(&b, &hi, 4);
    return ((unsigned long long)b << 32) | a;
  };
  for (int rp = 0; rp < 2; ++rp)
    for (int i = 0; i < 4; ++i) {
      for (int b = 0; b < 3; ++b) out->gy2[b][rp][i] = pair(out->gy[b][2 * rp * 4 + i], out->gy[b][(2 * rp + 1) * 4 + i]);
      for (int fo = 0; fo < 2; ++fo)
        for (int fi = 0; fi < 2; ++fi)
          for (int g = 1; g < 3; ++g)
            out->kz2[fo][fi][g - 1][rp][i] =
                pair(out->kz[fo][fi][g][2 * rp * 4 + i], out->kz[fo][fi][g][(2 * rp + 1) * 4 + i]);
      for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a) out->rr2[d][a][rp][i] = pair(out->rr[d][a][2 * rp][i], out->rr[d][a][2 * rp + 1][i]);
    }
  // the remainder rho_i = R_i - sum_{j>=i} C(j, i) L_j and the Taylor shift to the
  // cell centre, sum_{j>r} C(j, r) 2^-(j-r) L_j (the coefficient of xi^r of (xi + 1/2)^j)
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      long long bc = 1;  // C(j, i)
      for (int k = 1; k <= i; ++k) bc = bc * (j - i + k) / k;
      const float nb = j >= i ? -(float)bc : 0.f;
      const float ts = j > i ? (float)bc / (float)(1 << (j - i)) : 0.f;
      out->edge2[i][j] = pair(nb, nb);
      out->ts02[i][j] = pair(ts, ts);
    }
}

}  // namespace hermite
