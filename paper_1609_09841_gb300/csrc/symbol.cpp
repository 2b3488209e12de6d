// Fourier symbol of the half step and the largest stable time step, computed
// by the library (Sec. 2: Hermite methods are stable while waves do not
// travel from the cell boundary to the cell centre in a half step; for a given
// order, series length and grid the precise bound is where the spectral
// radius of the half step's symbol reaches one).
//
// For a Fourier mode exp(i theta . x / h) the 8 corners of a cell sit at
// offsets (side - 1/2) from the output node, so the 1-D factors of the half
// step become M x M complex matrices; their Kronecker products give the
// symbol, a 2M^3 x 2M^3 (wave equation) or M^3 x M^3 (advection) complex
// matrix.  Its eigenvalues come from a complex Hessenberg reduction
// (Householder reflections) and the shifted QR iteration with Wilkinson
// shifts and deflation (Francis; Golub and Van Loan, "Matrix Computations",
// Sec. 7.4-7.5), eigenvalues only.  Host code only: no GPU is used.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/hermite.h"
#include "advect.h"
#include "hermite_impl.h"

namespace hermite {
int fail(int code, const char *fmt, ...);
}

using namespace hermite;

namespace {

using cplx = std::complex<double>;

// Eigenvalues of the n x n complex matrix A (row-major, destroyed).  Returns
// false if the QR iteration did not converge within 60 n sweeps.
bool eigenvalues(std::vector<cplx> &A, int n, std::vector<cplx> &ev) {
  auto at = [&](int i, int j) -> cplx & { return A[(size_t)i * n + j]; };
  ev.assign(n, cplx(0));
  // Hessenberg reduction: for each column k, a reflection I - 2 v v^H that
  // zeroes the entries below the subdiagonal.
  std::vector<cplx> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0;
    for (int i = k + 1; i < n; ++i) xn += std::norm(at(i, k));
    xn = std::sqrt(xn);
    if (xn == 0) continue;
    const cplx x0 = at(k + 1, k);
    const cplx alpha = (std::abs(x0) > 0 ? -x0 / std::abs(x0) : cplx(-1)) * xn;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) {
      v[i] = at(i, k) - (i == k + 1 ? alpha : cplx(0));
      vn += std::norm(v[i]);
    }
    vn = std::sqrt(vn);
    if (vn == 0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    for (int j = k; j < n; ++j) {  // A <- (I - 2 v v^H) A
      cplx d = 0;
      for (int i = k + 1; i < n; ++i) d += std::conj(v[i]) * at(i, j);
      for (int i = k + 1; i < n; ++i) at(i, j) -= 2.0 * v[i] * d;
    }
    for (int i = 0; i < n; ++i) {  // A <- A (I - 2 v v^H)
      cplx d = 0;
      for (int j = k + 1; j < n; ++j) d += at(i, j) * v[j];
      for (int j = k + 1; j < n; ++j) at(i, j) -= 2.0 * d * std::conj(v[j]);
    }
    for (int i = k + 2; i < n; ++i) at(i, k) = 0;
  }
  // Shifted QR on the active window [lo, hi] of the Hessenberg matrix.  A
  // subdiagonal entry is dropped when it is below eps times its diagonal
  // neighbours or below eps times the largest entry of the matrix (the
  // latter settles eigenvalues near zero of defective blocks, whose
  // subdiagonals shrink only linearly; the perturbation stays eps ||H||).
  const double eps = 2.220446049250313e-16;
  double anorm = 0;
  for (const cplx &x : A) anorm = std::max(anorm, std::abs(x));
  std::vector<double> cs(n);
  std::vector<cplx> sn(n);
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev[0] = at(0, 0);
      break;
    }
    int lo = hi;
    while (lo > 0) {
      const double scale = std::abs(at(lo, lo)) + std::abs(at(lo - 1, lo - 1));
      if (std::abs(at(lo, lo - 1)) <= eps * std::max(scale, anorm)) {
        at(lo, lo - 1) = 0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // a 1 x 1 block has split off
      ev[hi] = at(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    ++iter;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its
    // last diagonal entry; an exceptional shift every 10 sweeps.
    const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    cplx mu;
    if (iter % 10 == 0) {
      mu = d + 0.75 * std::abs(c);
    } else {
      const cplx half = 0.5 * (a - d);
      const cplx disc = std::sqrt(half * half + b * c);
      const cplx m1 = d + half + disc, m2 = d + half - disc;  // (a + d)/2 +- disc
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    for (int k = lo; k <= hi; ++k) at(k, k) -= mu;
    // H - mu I = Q R by Givens rotations G_k on rows (k, k+1) ...
    for (int k = lo; k < hi; ++k) {
      const cplx x = at(k, k), y = at(k + 1, k);
      const double r = std::hypot(std::abs(x), std::abs(y));
      double cc;
      cplx ss;
      if (r == 0) {
        cc = 1;
        ss = 0;
      } else if (std::abs(x) == 0) {
        cc = 0;
        ss = std::conj(y) / std::abs(y);
      } else {
        cc = std::abs(x) / r;
        ss = (x / std::abs(x)) * std::conj(y) / r;
      }
      cs[k] = cc;
      sn[k] = ss;
      for (int j = k; j <= hi; ++j) {
        const cplx p = at(k, j), q = at(k + 1, j);
        at(k, j) = cc * p + ss * q;
        at(k + 1, j) = -std::conj(ss) * p + cc * q;
      }
    }
    // ... then R Q: columns (k, k+1) by G_k^H, and the shift back.
    for (int k = lo; k < hi; ++k) {
      const double cc = cs[k];
      const cplx ss = sn[k];
      const int rmax = std::min(k + 2, hi);
      for (int i = lo; i <= rmax; ++i) {
        const cplx p = at(i, k), q = at(i, k + 1);
        at(i, k) = p * cc + q * std::conj(ss);
        at(i, k + 1) = -p * ss + q * cc;
      }
    }
    for (int k = lo; k <= hi; ++k) at(k, k) += mu;
  }
  return true;
}

double spectral_radius(std::vector<cplx> &A, int n, bool *ok) {
  std::vector<cplx> ev;
  *ok = eigenvalues(A, n, ev);
  double r = 0;
  for (const cplx &e : ev) r = std::max(r, std::abs(e));
  return r;
}

// Phase of entry (r, i) of a right block: the left block is (-1)^(r+i) times
// it, at offset -1/2 instead of +1/2.
inline cplx phase(int r, int i, double th) {
  return ((r + i) & 1) ? cplx(0.0, 2.0 * std::sin(0.5 * th)) : cplx(2.0 * std::cos(0.5 * th), 0.0);
}

// Wave equation: S[(fo, r3, r2, r1)][(fi, i3, i2, i1)] =
//   sum_g Kz[fo][fi][g](theta3) (sum_{a+b=g} Gy_b(theta2) (x) Gx_a(theta1)),
// from the kernels' own tables (every grade; grades the series does not
// reach have zero tables).
void wave_symbol(int m, const StepCoeffs<double> &co, const double th[3], std::vector<cplx> &S) {
  const int M = m + 1, n = 2 * M * M * M;
  S.assign((size_t)n * n, cplx(0));
  cplx X[kMaxA][4][4], Y[kMaxA][4][4], Z[2][2][kMaxG][4][4];
  for (int a = 0; a < kMaxA; ++a)
    for (int r = 0; r < M; ++r)
      for (int i = 0; i < M; ++i) {
        X[a][r][i] = co.gx[a][r * 4 + i] * phase(r, i, th[0]);
        Y[a][r][i] = co.gy[a][r * 4 + i] * phase(r, i, th[1]);
      }
  for (int fo = 0; fo < 2; ++fo)
    for (int fi = 0; fi < 2; ++fi)
      for (int g = 0; g < kMaxG; ++g)
        for (int r = 0; r < M; ++r)
          for (int i = 0; i < M; ++i) Z[fo][fi][g][r][i] = co.kz[fo][fi][g][r * 4 + i] * phase(r, i, th[2]);
  std::vector<cplx> YX((size_t)kMaxG * M * M * M * M);  // [g][r2][r1][i2][i1]
  for (int g = 0; g < kMaxG; ++g)
    for (int r2 = 0; r2 < M; ++r2)
      for (int r1 = 0; r1 < M; ++r1)
        for (int i2 = 0; i2 < M; ++i2)
          for (int i1 = 0; i1 < M; ++i1) {
            cplx acc = 0;
            for (int a = 0; a < kMaxA; ++a)
              if (g - a >= 0 && g - a < kMaxA) acc += Y[g - a][r2][i2] * X[a][r1][i1];
            YX[(((size_t)(g * M + r2) * M + r1) * M + i2) * M + i1] = acc;
          }
  for (int fo = 0; fo < 2; ++fo)
    for (int r3 = 0; r3 < M; ++r3)
      for (int r2 = 0; r2 < M; ++r2)
        for (int r1 = 0; r1 < M; ++r1) {
          const int o = ((fo * M + r3) * M + r2) * M + r1;
          for (int fi = 0; fi < 2; ++fi)
            for (int i3 = 0; i3 < M; ++i3)
              for (int i2 = 0; i2 < M; ++i2)
                for (int i1 = 0; i1 < M; ++i1) {
                  cplx acc = 0;
                  for (int g = 0; g < kMaxG; ++g)
                    acc += Z[fo][fi][g][r3][i3] * YX[(((size_t)(g * M + r2) * M + r1) * M + i2) * M + i1];
                  S[(size_t)o * n + ((fi * M + i3) * M + i2) * M + i1] = acc;
                }
        }
}

// Advection: the per-cell matrix W (M^3 x P^3) of interpolation (Sec. 3.1),
// the q-stage loop of Alg. 4 and truncation, column by column.
void adv_cell_matrix(int m, int q, const double a[3], const double h[3], double tau, std::vector<double> &W) {
  const int M = m + 1, P = 2 * M, P3 = P * P * P, M3 = M * M * M;
  double H[64];
  build_H(m, H);
  const double ah[3] = {a[0] / h[0], a[1] / h[1], a[2] / h[2]};
  W.assign((size_t)M3 * P3, 0.0);
  std::vector<double> base(P3), w(P3), nw(P3);
  for (int tz = 0; tz < P; ++tz)
    for (int ty = 0; ty < P; ++ty)
      for (int tx = 0; tx < P; ++tx) {
        const int t = (tz * P + ty) * P + tx;
        for (int jz = 0; jz < P; ++jz)
          for (int jy = 0; jy < P; ++jy)
            for (int jx = 0; jx < P; ++jx)
              base[(jz * P + jy) * P + jx] = H[jz * P + tz] * H[jy * P + ty] * H[jx * P + tx];
        w = base;
        for (int k = q; k >= 1; --k) {
          const double f = tau / k;
          for (int jz = 0; jz < P; ++jz)
            for (int jy = 0; jy < P; ++jy)
              for (int jx = 0; jx < P; ++jx) {
                const int j = (jz * P + jy) * P + jx;
                double d = 0;
                if (jx + 1 < P) d += ah[0] * (jx + 1) * w[j + 1];
                if (jy + 1 < P) d += ah[1] * (jy + 1) * w[j + P];
                if (jz + 1 < P) d += ah[2] * (jz + 1) * w[j + P * P];
                nw[j] = base[j] + f * d;
              }
          w.swap(nw);
        }
        for (int i3 = 0; i3 < M; ++i3)
          for (int i2 = 0; i2 < M; ++i2)
            for (int i1 = 0; i1 < M; ++i1)
              W[(size_t)((i3 * M + i2) * M + i1) * P3 + t] = w[(i3 * P + i2) * P + i1];
      }
}

void adv_symbol(int m, const std::vector<double> &W, const double th[3], std::vector<cplx> &S) {
  const int M = m + 1, P = 2 * M, P3 = P * P * P, n = M * M * M;
  S.assign((size_t)n * n, cplx(0));
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const cplx e = std::exp(cplx(0.0, th[0] * (cx - 0.5) + th[1] * (cy - 0.5) + th[2] * (cz - 0.5)));
        for (int o = 0; o < n; ++o)
          for (int i3 = 0; i3 < M; ++i3)
            for (int i2 = 0; i2 < M; ++i2)
              for (int i1 = 0; i1 < M; ++i1) {
                const int t = ((cz * M + i3) * P + (cy * M + i2)) * P + (cx * M + i1);
                S[(size_t)o * n + (i3 * M + i2) * M + i1] += W[(size_t)o * P3 + t] * e;
              }
      }
}

// Largest spectral radius over the npts^3 grid of theta in [0, pi]^3 (the
// symbol at -theta is the complex conjugate), on up to 16 host threads.  With
// `limit` > 0 the search stops at the first radius above it.
template <typename Build>
double max_radius(int n, int npts, double limit, const Build &build, bool *ok) {
  const int total = npts * npts * npts;
  std::atomic<int> next(0);
  std::atomic<bool> stop(false), bad(false);
  unsigned nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  nthreads = std::min<unsigned>(nthreads, (unsigned)total);
  std::vector<double> best(nthreads, 0.0);
  auto work = [&](unsigned id) {
    std::vector<cplx> S;
    for (int t = next++; t < total && !stop; t = next++) {
      double th[3];
      int u = t;
      for (int k = 0; k < 3; ++k) {
        th[k] = npts > 1 ? M_PI * (u % npts) / (npts - 1) : 0.0;
        u /= npts;
      }
      build(th, S);
      bool good;
      const double r = spectral_radius(S, n, &good);
      if (!good) bad = true;
      best[id] = std::max(best[id], r);
      if (limit > 0 && r > limit) stop = true;
    }
  };
  std::vector<std::thread> pool;
  for (unsigned k = 1; k < nthreads; ++k) pool.emplace_back(work, k);
  work(0);
  for (auto &th : pool) th.join();
  *ok = !bad;
  return *std::max_element(best.begin(), best.end());
}

// The largest dt with max radius <= 1 + 1e-10 at every dt' <= dt: the set of
// stable steps need not be an interval (m = 3 with the whole series is weakly
// unstable, rho - 1 ~ 1e-7, for c tau / h in about (0.373, 0.39) and stable
// again at 0.40), so the steps dt_hi k / 60, k = 1, 2, ... are scanned
// upwards to the first unstable one and that bracket is bisected to 1e-4
// relative.  A window of instability narrower than dt_hi / 60 can be missed.
template <typename Radius>
int first_unstable_dt(double dt_hi, const Radius &radius_at, double *dt_out) {
  const double thresh = 1.0 + 1e-10;
  constexpr int kScan = 60;
  bool ok = true;
  double lo = 0, hi = -1;
  for (int k = 1; k <= kScan; ++k) {
    const double d = dt_hi * k / kScan;
    const double r = radius_at(d, thresh, &ok);
    if (!ok) return fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
    if (r > thresh) {
      hi = d;
      break;
    }
    lo = d;
  }
  if (hi < 0) {  // stable over the whole scan
    *dt_out = lo;
    return HERMITE_OK;
  }
  for (int it = 0; it < 60 && hi - lo > 1e-4 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double r = radius_at(mid, thresh, &ok);
    if (!ok) return fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
    (r <= thresh ? lo : hi) = mid;
  }
  *dt_out = lo;
  return HERMITE_OK;
}

bool valid_h(const double h[3]) {
  for (int k = 0; k < 3; ++k)
    if (!(h[k] > 0.0) || !std::isfinite(h[k])) return false;
  return true;
}

}  // namespace

extern "C" {

int hermite_symbol_radius(int m, int q, double c, const double h[3], double dt, const double theta[3],
                          double *rho) {
  if (m < 1 || m > 3 || !h || !theta || !rho || !valid_h(h) || !(c > 0) || !(dt >= 0) || !std::isfinite(dt))
    return fail(HERMITE_EINVAL, "bad argument to hermite_symbol_radius");
  if (q < 4 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 4..%d", q, 3 * (2 * m + 1));
  StepCoeffs<double> co;
  build_step_coeffs(m, h, c, 0.5 * dt, kForward, q, &co);
  std::vector<cplx> S;
  wave_symbol(m, co, theta, S);
  bool ok;
  *rho = spectral_radius(S, 2 * (m + 1) * (m + 1) * (m + 1), &ok);
  return ok ? HERMITE_OK : fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
}

int hermite_max_dt(int m, int q, double c, const double h[3], int npts, double *dt) {
  if (m < 1 || m > 3 || !h || !dt || !valid_h(h) || !(c > 0) || !std::isfinite(c) || npts < 2 || npts > 64)
    return fail(HERMITE_EINVAL, "bad argument to hermite_max_dt");
  if (q < 4 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 4..%d", q, 3 * (2 * m + 1));
  const int n = 2 * (m + 1) * (m + 1) * (m + 1);
  const double hmin = std::min(h[0], std::min(h[1], h[2]));
  auto radius_at = [&](double d, double limit, bool *ok) {
    StepCoeffs<double> co;
    build_step_coeffs(m, h, c, 0.5 * d, kForward, q, &co);
    return max_radius(n, npts, limit, [&](const double th[3], std::vector<cplx> &S) { wave_symbol(m, co, th, S); },
                      ok);
  };
  return first_unstable_dt(2.0 * 0.6 * hmin / c, radius_at, dt);
}

int hermite_max_radius(int m, int q, double c, const double h[3], double dt, int npts, double *rho) {
  if (m < 1 || m > 3 || !h || !rho || !valid_h(h) || !(c > 0) || !(dt >= 0) || !std::isfinite(dt) || npts < 1 ||
      npts > 64)
    return fail(HERMITE_EINVAL, "bad argument to hermite_max_radius");
  if (q < 4 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 4..%d", q, 3 * (2 * m + 1));
  StepCoeffs<double> co;
  build_step_coeffs(m, h, c, 0.5 * dt, kForward, q, &co);
  bool ok;
  *rho = max_radius(2 * (m + 1) * (m + 1) * (m + 1), npts, 0.0,
                    [&](const double th[3], std::vector<cplx> &S) { wave_symbol(m, co, th, S); }, &ok);
  return ok ? HERMITE_OK : fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
}

int hermite_adv_max_radius(int m, int q, const double a[3], const double h[3], double dt, int npts, double *rho) {
  if (m < 1 || m > 3 || !a || !h || !rho || !valid_h(h) || !(dt >= 0) || !std::isfinite(dt) || npts < 1 ||
      npts > 64)
    return fail(HERMITE_EINVAL, "bad argument to hermite_adv_max_radius");
  if (q == 0) q = 3 * (2 * m + 1);
  if (q < 1 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 1..%d", q, 3 * (2 * m + 1));
  std::vector<double> W;
  adv_cell_matrix(m, q, a, h, 0.5 * dt, W);
  bool ok;
  *rho = max_radius((m + 1) * (m + 1) * (m + 1), npts, 0.0,
                    [&](const double th[3], std::vector<cplx> &S) { adv_symbol(m, W, th, S); }, &ok);
  return ok ? HERMITE_OK : fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
}

int hermite_adv_symbol_radius(int m, int q, const double a[3], const double h[3], double dt,
                              const double theta[3], double *rho) {
  if (m < 1 || m > 3 || !a || !h || !theta || !rho || !valid_h(h) || !(dt >= 0) || !std::isfinite(dt))
    return fail(HERMITE_EINVAL, "bad argument to hermite_adv_symbol_radius");
  if (q == 0) q = 3 * (2 * m + 1);
  if (q < 1 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 1..%d", q, 3 * (2 * m + 1));
  std::vector<double> W;
  adv_cell_matrix(m, q, a, h, 0.5 * dt, W);
  std::vector<cplx> S;
  adv_symbol(m, W, theta, S);
  bool ok;
  *rho = spectral_radius(S, (m + 1) * (m + 1) * (m + 1), &ok);
  return ok ? HERMITE_OK : fail(HERMITE_ENOCONV, "eigenvalue iteration did not converge");
}

int hermite_adv_max_dt(int m, int q, const double a[3], const double h[3], int npts, double *dt) {
  if (m < 1 || m > 3 || !a || !h || !dt || !valid_h(h) || npts < 2 || npts > 64)
    return fail(HERMITE_EINVAL, "bad argument to hermite_adv_max_dt");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(a[k])) return fail(HERMITE_EINVAL, "velocity a[%d] is not finite", k);
  if (q == 0) q = 3 * (2 * m + 1);
  if (q < 1 || q > 3 * (2 * m + 1)) return fail(HERMITE_EINVAL, "q = %d outside 1..%d", q, 3 * (2 * m + 1));
  double speed = 0;  // max_k |a_k| / h_k
  for (int k = 0; k < 3; ++k) speed = std::max(speed, std::fabs(a[k]) / h[k]);
  if (speed == 0) return fail(HERMITE_EINVAL, "a = 0: every step is stable");
  const int n = (m + 1) * (m + 1) * (m + 1);
  auto radius_at = [&](double d, double limit, bool *ok) {
    std::vector<double> W;
    adv_cell_matrix(m, q, a, h, 0.5 * d, W);
    return max_radius(n, npts, limit, [&](const double th[3], std::vector<cplx> &S) { adv_symbol(m, W, th, S); },
                      ok);
  };
  return first_unstable_dt(2.0 * 0.6 / speed, radius_at, dt);
}

}  // extern "C"
