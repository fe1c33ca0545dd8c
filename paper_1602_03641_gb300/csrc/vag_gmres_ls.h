// The small least-squares problem of GMRES (Saad & Schultz 1986): each new
// Hessenberg column is reduced by the Givens rotations of the previous
// columns and one new rotation, which also rotates the right-hand side g
// (|g_{j+1}| is then the residual norm); at the end of a cycle R y = g is
// solved by back substitution.  Host and device code (the GMRES kernels call
// it per system in one thread; it compiles without CUDA for checking on the
// CPU).
#pragma once

#include <cfloat>
#include <math.h>

#ifdef __CUDACC__
#define VAG_HD __host__ __device__
#else
#define VAG_HD
#endif

namespace vag {

// c[0..j+1]: column j of the Hessenberg matrix on entry, of R on exit
// (c[j+1] = 0).  cs, sn: rotations 0..j-1 on entry, j added; g: rotated
// right-hand side, entries j and j+1 updated.  Returns false (nothing
// changed past the previous rotations) if the column is degenerate: its
// rotated diagonal pair has no positive finite norm.
VAG_HD inline bool gm_rotate_column(int j, double *c, double *cs, double *sn, double *g) {
  for (int q = 0; q < j; ++q) {
    const double a0 = c[q], a1 = c[q + 1];
    c[q] = cs[q] * a0 + sn[q] * a1;
    c[q + 1] = -sn[q] * a0 + cs[q] * a1;
  }
  const double rho = hypot(c[j], c[j + 1]);
  if (!(rho > 0.0 && rho <= DBL_MAX)) return false;
  cs[j] = c[j] / rho;
  sn[j] = c[j + 1] / rho;
  c[j] = rho;
  c[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  return true;
}

// y[0..k) with R y = g, R upper triangular stored by columns: R[l * ld + i]
// is row i of column l.
VAG_HD inline void gm_back_substitute(int k, const double *R, int ld, const double *g, double *y) {
  for (int i = k - 1; i >= 0; --i) {
    double a = g[i];
    for (int l = i + 1; l < k; ++l) a = fma(-R[l * ld + i], y[l], a);
    y[i] = a / R[i * ld + i];
  }
}

}  // namespace vag
