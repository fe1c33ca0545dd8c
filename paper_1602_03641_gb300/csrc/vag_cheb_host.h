// Arithmetic of the Chebyshev-Jacobi preconditioner: the interval from the
// Lanczos tridiagonal of a few Jacobi-CG steps, the coefficient table of the
// Chebyshev recurrence (Saad, Iterative Methods for Sparse Linear Systems,
// 2nd ed., Sec. 6.7.3 and Alg. 12.1), and the per-row update of one step,
// which the device kernel calls.  Compiles without CUDA, so that it can be
// checked on its own.
#pragma once

#include <cmath>
#include <vector>

#ifdef __CUDACC__
#define VAG_CHEB_HD __host__ __device__
#else
#define VAG_CHEB_HD
#endif

namespace vag {

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a and
// off-diagonal e, by bisection on the Sturm count (the number of negative
// pivots of T - x I, which is the number of eigenvalues below x).
inline double tridiag_max_eig(const std::vector<double> &a, const std::vector<double> &e) {
  const int m = (int)a.size();
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < m; ++i) {   // Gershgorin discs
    const double rad = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
    lo = std::fmin(lo, a[i] - rad);
    hi = std::fmax(hi, a[i] + rad);
  }
  auto below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      q = (a[i] - x) - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-13 * std::fmax(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= m) hi = mid;
    else lo = mid;
  }
  return hi;
}

// Upper end of the interval: `safety` x the largest eigenvalue of the Lanczos
// tridiagonal that m preconditioned-CG steps define (T_jj = 1/alpha_j +
// beta_{j-1}/alpha_{j-1}, T_j,j+1 = sqrt(beta_j)/alpha_j); 2 when m = 0 or
// the value is not a positive number.
inline double cheb_upper_bound(const double *alpha, const double *beta, int m, double safety) {
  if (m <= 0) return 2.0;
  std::vector<double> d(m), e(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j + 1 < m) e[j] = std::sqrt(beta[j]) / alpha[j];
  }
  const double b = safety * tridiag_max_eig(d, e);
  return (b > 0.0 && std::isfinite(b)) ? b : 2.0;
}

// Coefficients of `degree` steps of Chebyshev acceleration on [a, b]:
// theta = (b + a)/2, delta = (b - a)/2, sigma = theta/delta, rho_0 = 1/sigma,
// rho_j = 1/(2 sigma - rho_{j-1}); c[0] = 1/theta, and for j = 1..degree-1
// c[2j] = rho_j rho_{j-1}, c[2j+1] = 2 rho_j / delta (c[1] unused, 0).
inline void cheb_table(double a, double b, int degree, double *c) {
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  c[0] = 1.0 / theta;
  c[1] = 0.0;
  double rho_prev = 1.0 / sigma;
  for (int j = 1; j < degree; ++j) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    c[2 * j] = rho * rho_prev;
    c[2 * j + 1] = 2.0 * rho / delta;
    rho_prev = rho;
  }
}

// Step j >= 1 of the recurrence for one row, given the row's residual entry
// r_i, the product (A z_in)_i, D^-1_ii and the previous direction and iterate
// (d_in_i, z_in_i): with s = c[0] on the first step (its inputs are the
// unscaled w = D^-1 r) and 1 after it,
//   res = r_i - s (A z_in)_i,  d_out = c[2j] s d_in + c[2j+1] D^-1_ii res,
//   z_out = s z_in + d_out.
VAG_CHEB_HD inline void cheb_row_step(const double *c, int j, double ri, double Az, double dinv_i, double d_in,
                                      double z_in, double *d_out, double *z_out) {
  const double s_in = j == 1 ? c[0] : 1.0;
  const double res = fma(-s_in, Az, ri);
  const double di = fma(c[2 * j] * s_in, d_in, c[2 * j + 1] * (dinv_i * res));
  *d_out = di;
  *z_out = fma(s_in, z_in, di);
}

}  // namespace vag
