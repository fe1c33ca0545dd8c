// Krylov solve of the cell-eliminated system (Sec. 4.2, Eq. eqschur).
//
// The system is the Galerkin form restricted to the non-Dirichlet unknowns,
// hence symmetric positive definite: conjugate gradients with a Jacobi
// preconditioner (or a general one, z = M r: Chebyshev-Jacobi or aggregation
// AMG, further below).  A solve handles a batch of independent systems at once
// (a single system is a batch of one): every kernel runs one thread block per
// row tile of some system, and each system keeps its own CG scalars.  Per
// iteration three kernels:
//   k_spmv      q = A p (sliced ELL, one thread per row) fused with the partial p.q; the
//               last tile of a system to finish computes its alpha;
//   k_update    x += alpha p, r -= alpha q, partial r.z and r.r (z = D^-1 r);
//               the last tile computes beta and the convergence flag;
//   k_pdir      p = z + beta p.
// A converged system's tiles return at entry.  Reductions are deterministic
// and depend only on the system itself (its tiles cover its own rows only),
// so a system gives bitwise the same iterates alone or in a batch.
// Iterations are captured in a CUDA graph of `chunk` iterations; the host
// polls one counter (systems done) between graph launches.
#include <cmath>
#include <cstdio>
#include <vector>

#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int NT = 256;

// q = A p in the sliced-ELL layout, one thread per row: exactly one FMA per
// stored entry, in the row's CSR order.
template <int U>
__global__ void __launch_bounds__(NT) k_spmv(const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                             const int *__restrict__ scol, const double *__restrict__ sval,
                                             const double *__restrict__ x, double *__restrict__ y, Tiles tl,
                                             double *partials, unsigned *counter, KrylovScalars *ks, int *n_done,
                                             int with_dot) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  pdl_wait();
  pdl_trigger();
  if (with_dot && ks[sys].done) return;
  double dp = 0.0;
  for (int row = r0 + threadIdx.x; row < r1; row += NT) {
    const double s = sell_row<double, U>(row, rowptr, slice_ptr, scol, sval, x);
    y[row] = s;
    dp = fma(x[row], s, dp);
  }
  if (!with_dot) return;
  double v[1] = {dp}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.pq = out[0];
    if (!(out[0] > 0.0)) {
      k.breakdown = 1;
      k.alpha = 0.0;
      if (!k.done) { k.done = 1; atomicAdd(n_done, 1); }
    } else {
      k.alpha = k.rz / out[0];
    }
  }
}

__global__ void __launch_bounds__(NT) k_init(const double *__restrict__ b, const double *__restrict__ dinv,
                                             double *__restrict__ x, double *__restrict__ r, double *__restrict__ p,
                                             Tiles tl, double *partials, unsigned *counter, KrylovScalars *ks,
                                             int *n_done, double rtol, int maxit) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rz = 0.0, rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double bi = b[i];
    const double zi = dinv[i] * bi;
    x[i] = 0.0;
    r[i] = bi;
    p[i] = zi;
    rz = fma(bi, zi, rz);
    rr = fma(bi, bi, rr);
  }
  double v[2] = {rz, rr}, out[2];
  if (seg_sum<NT, 2>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.rz = out[0];
    k.rr = out[1];
    k.bb = out[1];
    k.tol2 = rtol * rtol * out[1];
    k.iter = 0;
    k.maxit = maxit;
    k.breakdown = 0;
    k.stalled = 0;
    k.inner_total = 0;
    k.beta = 0.0;
    k.done = (out[1] <= k.tol2) ? 1 : 0;
    if (k.done) atomicAdd(n_done, 1);
  }
}

__global__ void __launch_bounds__(NT) k_update(double *__restrict__ x, double *__restrict__ r,
                                               const double *__restrict__ p, const double *__restrict__ q,
                                               const double *__restrict__ dinv, Tiles tl, double *partials,
                                               unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double alpha = ks[sys].alpha;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rz = 0.0, rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rz = fma(ri, dinv[i] * ri, rz);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {rz, rr}, out[2];
  if (seg_sum<NT, 2>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    k.rr = out[1];
    k.iter += 1;
    bool fin = out[1] <= k.tol2 || k.iter >= k.maxit;
    if (!(out[1] == out[1])) { k.breakdown = 1; fin = true; }
    if (fin) { k.done = 1; atomicAdd(n_done, 1); }
  }
}

__global__ void __launch_bounds__(NT) k_pdir(double *__restrict__ p, const double *__restrict__ r,
                                             const double *__restrict__ dinv, Tiles tl, const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double beta = ks[sys].beta;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0 + threadIdx.x; i < r1; i += NT) p[i] = fma(beta, p[i], dinv[i] * r[i]);
}

// Restart from the current iterate with the true residual: r = b - A x,
// p = z = D^-1 r.  A system whose true residual already meets the tolerance
// stays done.
__global__ void __launch_bounds__(NT) k_restart(const double *__restrict__ b, const double *__restrict__ Ax,
                                                const double *__restrict__ dinv, double *__restrict__ r,
                                                double *__restrict__ p, Tiles tl, double *partials, unsigned *counter,
                                                KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rz = 0.0, rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double ri = b[i] - Ax[i];
    const double zi = dinv[i] * ri;
    r[i] = ri;
    p[i] = zi;
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {rz, rr}, out[2];
  if (seg_sum<NT, 2>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.rz = out[0];
    k.rr = out[1];
    k.beta = 0.0;
    k.done = (out[1] <= k.tol2 || k.iter >= k.maxit || k.breakdown || k.stalled) ? 1 : 0;
    if (k.done) atomicAdd(n_done, 1);
  }
}

// --- preconditioned by a general operator z = M r (AMG) -------------------

// x = 0, r = b, partial b.b (scalars set by k_rz_start)
__global__ void __launch_bounds__(NT) k_init_m(const double *__restrict__ b, double *__restrict__ x,
                                               double *__restrict__ r, Tiles tl, double *partials,
                                               unsigned *counter, KrylovScalars *ks, double rtol, int maxit) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double bb = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    bb = fma(bi, bi, bb);
  }
  double v[1] = {bb}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.bb = out[0];
    k.rr = out[0];
    k.tol2 = rtol * rtol * out[0];
    k.iter = 0;
    k.maxit = maxit;
    k.breakdown = 0;
    k.stalled = 0;
    k.inner_total = 0;
    k.beta = 0.0;
    k.done = 0;
  }
}

// p = z, rz = r.z; done if r.r already meets the tolerance (or the system is
// done for another reason)
__global__ void __launch_bounds__(NT) k_rz_start(const double *__restrict__ r, const double *__restrict__ z,
                                                 double *__restrict__ p, Tiles tl, double *partials,
                                                 unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rz = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double zi = z[i];
    p[i] = zi;
    rz = fma(r[i], zi, rz);
  }
  double v[1] = {rz}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.rz = out[0];
    k.beta = 0.0;
    const bool fin = k.rr <= k.tol2 || k.iter >= k.maxit || k.breakdown || k.stalled;
    k.done = fin ? 1 : 0;
    if (fin) atomicAdd(n_done, 1);
    else if (!(out[0] > 0.0)) { k.breakdown = 1; k.done = 1; atomicAdd(n_done, 1); }
  }
}

// x += alpha p, r -= alpha q, partial r.r; the last tile counts the iteration
// and tests convergence
// With sinv0 set, also the first sweep of the AMG V-cycle from zero,
// t0 = omega D_l1^-1 r (the same product the V-cycle would form).
__global__ void __launch_bounds__(NT) k_update_m(double *__restrict__ x, double *__restrict__ r,
                                                 const double *__restrict__ p, const double *__restrict__ q, Tiles tl,
                                                 double *partials, unsigned *counter, KrylovScalars *ks, int *n_done,
                                                 const double *__restrict__ sinv0, double *__restrict__ t0,
                                                 double omega) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  pdl_wait();
  pdl_trigger();
  if (ks[sys].done) return;
  const double alpha = ks[sys].alpha;
  double rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    if (sinv0) t0[i] = omega * sinv0[i] * ri;
    rr = fma(ri, ri, rr);
  }
  double v[1] = {rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.rr = out[0];
    k.iter += 1;
    bool fin = out[0] <= k.tol2 || k.iter >= k.maxit;
    if (!(out[0] == out[0])) { k.breakdown = 1; fin = true; }
    if (fin) { k.done = 1; atomicAdd(n_done, 1); }
  }
}

// beta = (r.z)_new / (r.z)_old and p = z + beta p in one pass: each tile
// first needs the system's new r.z, so this kernel only reduces; k_pdir_z
// applies it
__global__ void __launch_bounds__(NT) k_rz(const double *__restrict__ r, const double *__restrict__ z, Tiles tl,
                                           double *partials, unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  pdl_wait();
  pdl_trigger();
  if (ks[sys].done) return;
  double rz = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) rz = fma(r[i], z[i], rz);
  double v[1] = {rz}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    if (!(out[0] > 0.0)) { k.breakdown = 1; k.done = 1; atomicAdd(n_done, 1); }
  }
}

__global__ void __launch_bounds__(NT) k_pdir_z(double *__restrict__ p, const double *__restrict__ z, Tiles tl,
                                               const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  pdl_wait();
  pdl_trigger();
  if (ks[sys].done) return;
  const double beta = ks[sys].beta;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) p[i] = fma(beta, p[i], z[i]);
}

// restart for the general preconditioner: r = b - A x and r.r
__global__ void __launch_bounds__(NT) k_restart_m(const double *__restrict__ b, const double *__restrict__ Ax,
                                                  double *__restrict__ r, Tiles tl, double *partials,
                                                  unsigned *counter, KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double v[1] = {rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) ks[sys].rr = out[0];
}

__global__ void __launch_bounds__(NT) k_resid2(const double *__restrict__ b, const double *__restrict__ Ax, Tiles tl,
                                               double *partials, unsigned *counter, KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double s = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double d = b[i] - Ax[i];
    s = fma(d, d, s);
  }
  double v[1] = {s}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) ks[sys].res2 = out[0];
}

// u over [nodes | ffaces | cells]: Krylov rows, then Dirichlet values.
__global__ void k_scatter_rows(int n_rows, const int *__restrict__ dof_of_row, const double *__restrict__ x,
                               double *__restrict__ u) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rows) u[dof_of_row[r]] = x[r];
}
__global__ void k_scatter_dir(int nd, const int *__restrict__ dn, const double *__restrict__ dv, double *__restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nd) u[dn[i]] = dv[i];
}

Tiles tiles_of(const System *s) {
  return Tiles{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0, s->seg.sys_grp0,
               s->seg.n_tiles, s->seg.n_sys};
}

// ------------------------------------------------------------- BiCGStab ----
// Right-preconditioned BiCGStab (van der Vorst 1992), the Krylov method the
// paper's experiments use (§5.3), with the same per-system tiles and
// deterministic reductions as CG.  Per iteration, with p^ = M p, s^ = M s:
//   v = A p^, alpha = rho / (r0^.v), s = r - alpha v, t = A s^,
//   omega = (t.s)/(t.t), x += alpha p^ + omega s^, r = s - omega t,
//   rho' = r0^.r, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).

// r0^ = p = r (after k_init_m: x = 0, r = b); rho = r.r = b.b
__global__ void __launch_bounds__(NT) k_bi_start(const double *__restrict__ r, double *__restrict__ r0,
                                                 double *__restrict__ p, Tiles tl, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int r0i = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0i + threadIdx.x; i < r1; i += NT) {
    r0[i] = r[i];
    p[i] = r[i];
  }
  if (t == tl.sys_tile0[sys] && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.rz = k.bb;
    k.omega = 1.0;
    k.half = 0;
    const bool fin = k.rr <= k.tol2 || k.maxit <= 0;
    k.done = fin ? 1 : 0;
    if (fin) atomicAdd(n_done, 1);
  }
}

// z = D^-1 x (Jacobi preconditioner of BiCGStab)
__global__ void __launch_bounds__(NT) k_bi_jacobi(const double *__restrict__ x, const double *__restrict__ dinv,
                                                  double *__restrict__ z, Tiles tl, const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) z[i] = dinv[i] * x[i];
}

// alpha = rho / (r0^.v)
__global__ void __launch_bounds__(NT) k_bi_alpha(const double *__restrict__ r0, const double *__restrict__ v, Tiles tl,
                                                 double *partials, unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  double d = 0.0;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) d = fma(r0[i], v[i], d);
  double in[1] = {d}, out[1];
  if (seg_sum<NT, 1>(in, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.pq = out[0];
    if (!(out[0] != 0.0) || !(k.rz == k.rz)) {
      k.breakdown = 1;
      k.done = 1;
      atomicAdd(n_done, 1);
    } else {
      k.alpha = k.rz / out[0];
    }
  }
}

// s = r - alpha v, and s.s (a converged s ends the iteration with omega = 0)
__global__ void __launch_bounds__(NT) k_bi_s(const double *__restrict__ r, const double *__restrict__ v,
                                             double *__restrict__ sv, Tiles tl, double *partials, unsigned *counter,
                                             KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double alpha = ks[sys].alpha;
  double ss = 0.0;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    const double si = fma(-alpha, v[i], r[i]);
    sv[i] = si;
    ss = fma(si, si, ss);
  }
  double in[1] = {ss}, out[1];
  if (seg_sum<NT, 1>(in, partials, counter, tl, t, sys, out) && threadIdx.x == 0)
    ks[sys].half = out[0] <= ks[sys].tol2 ? 1 : 0;
}

// omega = (t.s)/(t.t) (0 when s already met the tolerance)
__global__ void __launch_bounds__(NT) k_bi_omega(const double *__restrict__ tv, const double *__restrict__ sv, Tiles tl,
                                                 double *partials, unsigned *counter, KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  double ts = 0.0, tt = 0.0;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    ts = fma(tv[i], sv[i], ts);
    tt = fma(tv[i], tv[i], tt);
  }
  double in[2] = {ts, tt}, out[2];
  if (seg_sum<NT, 2>(in, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.omega = (k.half || !(out[1] > 0.0)) ? 0.0 : out[0] / out[1];
  }
}

// x += alpha p^ + omega s^, r = s - omega t, rho' = r0^.r and r.r; the last
// tile counts the iteration, tests convergence and forms beta
__global__ void __launch_bounds__(NT) k_bi_update(double *__restrict__ x, double *__restrict__ r,
                                                  const double *__restrict__ ph, const double *__restrict__ sh,
                                                  const double *__restrict__ sv, const double *__restrict__ tv,
                                                  const double *__restrict__ r0, Tiles tl, double *partials,
                                                  unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double alpha = ks[sys].alpha, omega = ks[sys].omega;
  double rho = 0.0, rr = 0.0;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
    const double ri = fma(-omega, tv[i], sv[i]);
    r[i] = ri;
    rho = fma(r0[i], ri, rho);
    rr = fma(ri, ri, rr);
  }
  double in[2] = {rho, rr}, out[2];
  if (seg_sum<NT, 2>(in, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.iter += 1;
    k.rr = out[1];
    bool fin = out[1] <= k.tol2 || k.half || k.iter >= k.maxit;
    if (!(out[1] == out[1])) { k.breakdown = 1; fin = true; }
    if (!fin && (!(out[0] != 0.0) || !(k.omega != 0.0))) { k.breakdown = 1; fin = true; }
    if (!fin) {
      k.beta = (out[0] / k.rz) * (k.alpha / k.omega);
      k.rz = out[0];
    }
    if (fin) { k.done = 1; atomicAdd(n_done, 1); }
  }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(NT) k_bi_pdir(double *__restrict__ p, const double *__restrict__ r,
                                                const double *__restrict__ v, Tiles tl, const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double beta = ks[sys].beta, omega = ks[sys].omega;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) p[i] = fma(beta, fma(-omega, v[i], p[i]), r[i]);
}

}  // namespace

// Rows per tile: 256, one row per thread.  (Tiles of up to 2048 rows, several
// rows per thread, cost the SpMV a third of its bandwidth at 128^3 on GB300:
// a thread's rows run one after the other, with fewer loads in flight; the
// price of small tiles, a longer list of partial sums for the last tile of a
// system to add, is a few microseconds.)  The tiling depends on the system
// alone.
static int tile_rows(int) { return 256; }

void build_tiles(System *s) {
  Segments &g = s->seg;
  std::vector<int> tsys, t0, t1, st(g.n_sys + 1);
  for (int i = 0; i < g.n_sys; ++i) {
    st[i] = (int)tsys.size();
    const int a = g.row_start[i], b = g.row_start[i + 1];
    const int T = tile_rows(b - a);
    int r = a;
    do {   // at least one (possibly empty) tile per system
      tsys.push_back(i);
      t0.push_back(r);
      t1.push_back(std::min(r + T, b));
      r += T;
    } while (r < b);
  }
  st[g.n_sys] = (int)tsys.size();
  g.n_tiles = (int)tsys.size();
  g.tile_start_h = st;
  std::vector<int> gr(g.n_sys + 1, 0);   // reduction groups of each system's tiles
  for (int i = 0; i < g.n_sys; ++i) gr[i + 1] = gr[i] + (st[i + 1] - st[i] + kSegGroup - 1) / kSegGroup;
  g.n_groups = gr[g.n_sys];
  g.sys_grp0 = sys_alloc<int>(s, g.n_sys + 1);
  g.tile_sys = sys_alloc<int>(s, g.n_tiles);
  g.tile_row0 = sys_alloc<int>(s, g.n_tiles);
  g.tile_row1 = sys_alloc<int>(s, g.n_tiles);
  g.sys_tile0 = sys_alloc<int>(s, g.n_sys + 1);
  cudaStream_t str = s->ctx->stream;
  VAG_CUDA(cudaMemcpyAsync(g.tile_sys, tsys.data(), sizeof(int) * g.n_tiles, cudaMemcpyHostToDevice, str));
  VAG_CUDA(cudaMemcpyAsync(g.tile_row0, t0.data(), sizeof(int) * g.n_tiles, cudaMemcpyHostToDevice, str));
  VAG_CUDA(cudaMemcpyAsync(g.tile_row1, t1.data(), sizeof(int) * g.n_tiles, cudaMemcpyHostToDevice, str));
  VAG_CUDA(cudaMemcpyAsync(g.sys_tile0, st.data(), sizeof(int) * (g.n_sys + 1), cudaMemcpyHostToDevice, str));
  VAG_CUDA(cudaMemcpyAsync(g.sys_grp0, gr.data(), sizeof(int) * (g.n_sys + 1), cudaMemcpyHostToDevice, str));
  VAG_CUDA(cudaStreamSynchronize(str));   // host vectors go out of scope
}

static void launch_spmv_u(System *s, int u, const double *x, double *y, int with_dot, cudaStream_t st) {
  auto kern = u == 2 ? k_spmv<2> : u == 8 ? k_spmv<8> : k_spmv<4>;
  launch_pdl(kern, s->seg.n_tiles, NT, 0, st, (const int *)s->rowptr, (const int *)s->slice_ptr,
             (const int *)s->scol, (const double *)s->sval, x, y, tiles_of(s), s->partials, s->counter, s->ks,
             s->n_done, with_dot);
  note_launches(1);
}

static void launch_spmv(System *s, const double *x, double *y, int with_dot, cudaStream_t st) {
  launch_spmv_u(s, s->sell_u ? s->sell_u : 4, x, y, with_dot, st);
}

// The autotuner of the sliced-ELL product: 2, 4 or 8 entries of a row in
// flight per thread, timed (CUDA events) on the system's own matrix the first
// time the context meets a matrix of this size class; later systems of the
// class reuse the choice.  The candidates take turns over four rounds of 10
// launches and each keeps its fastest round; 4 stays unless another is more
// than 2 % faster (at 128^3 the three are within a few per cent, single
// short timings picked each of them in different processes, and 4 is the
// best for the FP32 sweeps of the mixed path as well).  Every candidate
// performs the same FMAs in the same order, so the choice changes the time,
// never the result (a system stays bitwise the same alone or in a batch).
void tune_sell(System *s) {
  if (s->sell_u) return;
  int cls = 0;
  while ((2 << cls) <= s->n_rows && cls < 31) ++cls;
  int &slot = s->ctx->sell_unroll[cls];
  if (!slot) {
    ensure_krylov_buffers(s);
    cudaStream_t st = s->ctx->stream;
    VAG_CUDA(cudaMemsetAsync(s->kp, 0, sizeof(double) * s->n_rows, st));
    const int cand[3] = {4, 2, 8};
    float best[3] = {0.f, 0.f, 0.f};
    for (int round = 0; round < 4; ++round) {
      for (int c = 0; c < 3; ++c) {
        launch_spmv_u(s, cand[c], s->kp, s->kq, 0, st);
        VAG_CUDA(cudaEventRecord(s->ev0, st));
        for (int r = 0; r < 10; ++r) launch_spmv_u(s, cand[c], s->kp, s->kq, 0, st);
        VAG_CUDA(cudaEventRecord(s->ev1, st));
        VAG_CUDA(cudaEventSynchronize(s->ev1));
        float ms = 0.f;
        VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
        if (round == 0 || ms < best[c]) best[c] = ms;
      }
    }
    int pick = 0;   // 4
    for (int c = 1; c < 3; ++c)
      if (best[c] < 0.98f * best[0] && best[c] < best[pick]) pick = c;
    slot = cand[pick];
    if (trace_enabled()) std::fprintf(stderr, "[vag trace] SELL autotune: %d rows -> %d in flight\n", s->n_rows, slot);
  }
  s->sell_u = slot;
}

void ensure_krylov_buffers(System *s) {
  if (s->kx) return;
  const int ns = s->seg.n_sys;
  s->kx = sys_alloc<double>(s, s->n_rows);
  s->kr = sys_alloc<double>(s, s->n_rows);
  s->kp = sys_alloc<double>(s, s->n_rows);
  s->kq = sys_alloc<double>(s, s->n_rows);
  // tile partials, then group partials (two values each at most)
  s->partials = sys_alloc<double>(s, std::max<size_t>(2 * ((size_t)s->seg.n_tiles + s->seg.n_groups),
                                                      (size_t)kMaxRedBlocks));
  // per-system counters, one spare, then the group counters
  s->counter = sys_alloc<unsigned>(s, ns + 1 + s->seg.n_groups);
  s->ks = sys_alloc<KrylovScalars>(s, ns);
  s->n_done = sys_alloc<int>(s, 1);
  s->u = sys_alloc<double>(s, (size_t)s->n_cv);
  VAG_CUDA(cudaMemsetAsync(s->counter, 0, (ns + 1 + s->seg.n_groups) * sizeof(unsigned), s->ctx->stream));
  VAG_CUDA(cudaMemsetAsync(s->u, 0, sizeof(double) * s->n_cv, s->ctx->stream));
  if (!s->ks_host) VAG_CUDA(cudaMallocHost(&s->ks_host, sizeof(KrylovScalars) * ns));
  if (!s->n_done_host) VAG_CUDA(cudaMallocHost(&s->n_done_host, sizeof(int)));
}

void launch_spmv_plain(System *s, const double *x, double *y, cudaStream_t st) { launch_spmv(s, x, y, 0, st); }

void true_residual2(System *s, cudaStream_t st) {
  launch_spmv(s, s->kx, s->kq, 0, st);
  k_resid2<<<s->seg.n_tiles, NT, 0, st>>>(s->rhs, s->kq, tiles_of(s), s->partials, s->counter, s->ks);
  note_launches(1);
  VAG_CHECK_LAUNCH();
}

void spmv_f64(System *s, const double *x, double *y) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  launch_spmv(s, x, y, 0, s->ctx->stream);
  VAG_CHECK_LAUNCH();
}

double time_spmv(System *s, int reps) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  cudaStream_t st = s->ctx->stream;
  VAG_CUDA(cudaMemsetAsync(s->kp, 0, sizeof(double) * s->n_rows, st));
  launch_spmv(s, s->kp, s->kq, 0, st);   // warm-up
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  for (int r = 0; r < reps; ++r) launch_spmv(s, s->kp, s->kq, 0, st);
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  return (double)ms / reps;
}

static void pcg_iteration_amg(System *s, cudaStream_t st) {
  const Tiles tl = tiles_of(s);
  const int nt = s->seg.n_tiles;
  launch_spmv(s, s->kp, s->kq, 1, st);
  double *t0 = nullptr;
  double omega = 0.0;
  const double *sinv0 = amg_first_sweep_scale(s, t0, omega);
  launch_pdl(k_update_m, nt, NT, 0, st, s->kx, s->kr, (const double *)s->kp, (const double *)s->kq, tl, s->partials,
             s->counter, s->ks, s->n_done, sinv0, t0, omega);
  const bool rz_done = sinv0 ? amg_apply_cg(s, s->kr, s->kz, st) : (amg_apply(s, s->kr, s->kz, st), false);
  if (!rz_done) {
    launch_pdl(k_rz, nt, NT, 0, st, (const double *)s->kr, (const double *)s->kz, tl, s->partials, s->counter, s->ks,
               s->n_done);
    note_launches(1);
  }
  launch_pdl(k_pdir_z, nt, NT, 0, st, s->kp, (const double *)s->kz, tl, (const KrylovScalars *)s->ks);
  note_launches(2);
}

static void pcg_iteration(System *s, cudaStream_t st) {
  const Tiles tl = tiles_of(s);
  launch_spmv(s, s->kp, s->kq, 1, st);
  k_update<<<s->seg.n_tiles, NT, 0, st>>>(s->kx, s->kr, s->kp, s->kq, s->dinv, tl, s->partials, s->counter, s->ks,
                                          s->n_done);
  note_launches(1);
  k_pdir<<<s->seg.n_tiles, NT, 0, st>>>(s->kp, s->kr, s->dinv, tl, s->ks);
  note_launches(1);
}

// Chebyshev: the CG update also forms w = D^-1 r (the polynomial's first
// step), the remaining steps follow, the last one forming r.z and beta
static void pcg_iteration_cheb(System *s, cudaStream_t st) {
  const Tiles tl = tiles_of(s);
  const int nt = s->seg.n_tiles;
  launch_spmv(s, s->kp, s->kq, 1, st);
  launch_pdl(k_update_m, nt, NT, 0, st, s->kx, s->kr, (const double *)s->kp, (const double *)s->kq, tl, s->partials,
             s->counter, s->ks, s->n_done, (const double *)s->dinv, s->cw, 1.0);
  cheb_apply(s, s->kr, s->kz, st, true, true, true);
  launch_pdl(k_pdir_z, nt, NT, 0, st, s->kp, (const double *)s->kz, tl, (const KrylovScalars *)s->ks);
  note_launches(2);
}

void jacobi_cg_coefficients(System *s, const double *v, int m, std::vector<double> &alpha,
                            std::vector<double> &beta, std::vector<int> &steps) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  cudaStream_t st = s->ctx->stream;
  const int ns = s->seg.n_sys;
  VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
  // rtol 0: a system stops only on an exact zero residual, a breakdown or m
  k_init<<<s->seg.n_tiles, NT, 0, st>>>(v, s->dinv, s->kx, s->kr, s->kp, tiles_of(s), s->partials, s->counter, s->ks,
                                        s->n_done, 0.0, m);
  note_launches(1);
  alpha.assign((size_t)ns * m, 0.0);
  beta.assign((size_t)ns * m, 0.0);
  steps.assign(ns, 0);
  for (int j = 0; j < m; ++j) {
    pcg_iteration(s, st);
    VAG_CHECK_LAUNCH();
    VAG_CUDA(cudaMemcpyAsync(s->ks_host, s->ks, sizeof(KrylovScalars) * ns, cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < ns; ++i) {
      const KrylovScalars &k = s->ks_host[i];
      if (steps[i] != j || k.iter != j + 1 || k.breakdown) continue;
      if (!(k.alpha > 0.0) || !std::isfinite(k.alpha) || !(k.beta >= 0.0) || !std::isfinite(k.beta)) continue;
      alpha[(size_t)i * m + j] = k.alpha;
      beta[(size_t)i * m + j] = k.beta;
      steps[i] = j + 1;
    }
  }
}

void pcg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
  tune_sell(s);
  const bool amg = o->precond == VAG_PC_AMG || o->precond == VAG_PC_AMG_RS;
  const bool cheb = o->precond == VAG_PC_CHEBYSHEV;
  const bool general = amg || cheb;   // z = M r by a general operator
  const int ns = s->seg.n_sys;
  const int nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  float setup_ms = 0.f;
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  if (general) {
    if (!s->kz) s->kz = sys_alloc<double>(s, s->n_rows);
    if (amg) amg_setup(s, o->precision != VAG_FP64, o->precision == VAG_MIXED_F16, o->precond == VAG_PC_AMG_RS);
    else cheb_setup(s);
    trace_mark(st, amg ? "AMG setup" : "Chebyshev setup (Lanczos bounds)");
    VAG_CUDA(cudaEventRecord(s->ev1, st));
    VAG_CUDA(cudaEventSynchronize(s->ev1));
    cudaEventElapsedTime(&setup_ms, s->ev0, s->ev1);
  }
  auto apply_m = [&](const double *r, double *z) {
    if (amg) amg_apply(s, r, z, st);
    else cheb_apply(s, r, z, st, false, false, false);
  };
  VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
  if (general) {
    k_init_m<<<nt, NT, 0, st>>>(s->rhs, s->kx, s->kr, tl, s->partials, s->counter, s->ks, o->rtol, o->maxit);
    apply_m(s->kr, s->kz);
    k_rz_start<<<nt, NT, 0, st>>>(s->kr, s->kz, s->kp, tl, s->partials, s->counter, s->ks, s->n_done);
    note_launches(2);
  } else {
    k_init<<<nt, NT, 0, st>>>(s->rhs, s->dinv, s->kx, s->kr, s->kp, tl, s->partials, s->counter, s->ks,
                              s->n_done, o->rtol, o->maxit);
    note_launches(1);
  }
  VAG_CHECK_LAUNCH();
  trace_mark(st, "CG start (r0, z0)");
  const int chunk = 16;
  cudaGraphExec_t &gexec = amg ? s->pcg_graph_amg : cheb ? s->pcg_graph_cheb : s->pcg_graph;
  if (amg && gexec) {   // the hierarchy (and its pointers) is rebuilt every solve
    cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  if (!gexec) {
    cudaGraph_t graph;
    VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    for (int i = 0; i < chunk; ++i) {
      if (amg) pcg_iteration_amg(s, st);
      else if (cheb) pcg_iteration_cheb(s, st);
      else pcg_iteration(s, st);
    }
    set_capturing(false);
    VAG_CUDA(cudaStreamEndCapture(st, &graph));
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    VAG_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
    cudaGraphDestroy(graph);
    if (amg) s->amg_graph_nodes = nodes;
    if (cheb) s->cheb_graph_nodes = nodes;
    trace_mark(st, "graph capture + instantiate");
  }
  const unsigned long long per_launch = amg ? s->amg_graph_nodes : cheb ? s->cheb_graph_nodes : 3ull * chunk;
  const int max_chunks = (o->maxit + chunk - 1) / chunk;
  // The recursive residual can drift below the true one; after convergence
  // the true residual is recomputed and CG restarts from the current iterate
  // (a few times at most) for every system still above its tolerance whose
  // true residual still falls.
  std::vector<double> prev_res2;
  for (int attempt = 0;; ++attempt) {
    for (int c = 0; c < max_chunks + 1; ++c) {
      VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*s->n_done_host >= ns) break;
      VAG_CUDA(cudaGraphLaunch(gexec, st));
      note_launches(per_launch);
    }
    trace_mark(st, "CG iterations (graph chunks)");
    launch_spmv(s, s->kx, s->kq, 0, st);
    k_resid2<<<nt, NT, 0, st>>>(s->rhs, s->kq, tl, s->partials, s->counter, s->ks);
    note_launches(1);
    VAG_CHECK_LAUNCH();
    trace_mark(st, "true residual");
    if (attempt == 3) break;
    VAG_CUDA(cudaMemcpyAsync(s->ks_host, s->ks, sizeof(KrylovScalars) * ns, cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    bool again = false;
    prev_res2.resize(ns, INFINITY);
    for (int i = 0; i < ns; ++i) {
      const KrylovScalars &k = s->ks_host[i];
      const bool improving = k.res2 < 0.25 * prev_res2[i];
      again |= (k.res2 > k.tol2 && k.iter < k.maxit && !k.breakdown && improving);
      prev_res2[i] = k.res2;
      s->ks_host[i].stalled = !improving;
    }
    if (!again) break;
    // push the stall flags back before the restart kernels read them
    VAG_CUDA(cudaMemcpyAsync(s->ks, s->ks_host, sizeof(KrylovScalars) * ns, cudaMemcpyHostToDevice, st));
    VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
    if (general) {
      k_restart_m<<<nt, NT, 0, st>>>(s->rhs, s->kq, s->kr, tl, s->partials, s->counter, s->ks);
      apply_m(s->kr, s->kz);
      k_rz_start<<<nt, NT, 0, st>>>(s->kr, s->kz, s->kp, tl, s->partials, s->counter, s->ks, s->n_done);
      note_launches(2);
    } else {
      k_restart<<<nt, NT, 0, st>>>(s->rhs, s->kq, s->dinv, s->kr, s->kp, tl, s->partials, s->counter, s->ks,
                                   s->n_done);
      note_launches(1);
    }
  }
  finish_solve(s, info, false);
  info->ms_setup = setup_ms;
  info->ms_solve -= setup_ms;
}

void bicgstab_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
  tune_sell(s);
  const bool amg = o->precond == VAG_PC_AMG || o->precond == VAG_PC_AMG_RS;
  const bool cheb = o->precond == VAG_PC_CHEBYSHEV;
  const int nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  if (!s->b_r0) {
    s->b_r0 = sys_alloc<double>(s, s->n_rows);
    s->b_s = sys_alloc<double>(s, s->n_rows);
    s->b_sh = sys_alloc<double>(s, s->n_rows);
    s->b_t = sys_alloc<double>(s, s->n_rows);
    s->b_ph = sys_alloc<double>(s, s->n_rows);
  }
  float setup_ms = 0.f;
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  if (amg) {
    if (!s->kz) s->kz = sys_alloc<double>(s, s->n_rows);
    amg_setup(s, o->precision != VAG_FP64, o->precision == VAG_MIXED_F16, o->precond == VAG_PC_AMG_RS);
    VAG_CUDA(cudaEventRecord(s->ev1, st));
    VAG_CUDA(cudaEventSynchronize(s->ev1));
    cudaEventElapsedTime(&setup_ms, s->ev0, s->ev1);
  } else if (cheb) {
    cheb_setup(s);
    VAG_CUDA(cudaEventRecord(s->ev1, st));
    VAG_CUDA(cudaEventSynchronize(s->ev1));
    cudaEventElapsedTime(&setup_ms, s->ev0, s->ev1);
  }
  auto precond = [&](const double *in, double *out) {
    if (amg) {
      amg_apply(s, in, out, st);
    } else if (cheb) {
      cheb_apply(s, in, out, st, true, false, false);
    } else {
      k_bi_jacobi<<<nt, NT, 0, st>>>(in, s->dinv, out, tl, s->ks);
      note_launches(1);
    }
  };
  VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
  k_init_m<<<nt, NT, 0, st>>>(s->rhs, s->kx, s->kr, tl, s->partials, s->counter, s->ks, o->rtol, o->maxit);
  k_bi_start<<<nt, NT, 0, st>>>(s->kr, s->b_r0, s->kp, tl, s->ks, s->n_done);
  note_launches(2);
  VAG_CHECK_LAUNCH();
  // iterations in a CUDA graph of `chunk` iterations, rebuilt every solve
  // (the AMG hierarchy's buffers are new each time)
  const int chunk = 8;
  if (s->bicg_graph) {
    cudaGraphExecDestroy(s->bicg_graph);
    s->bicg_graph = nullptr;
  }
  cudaGraph_t graph;
  VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  for (int i = 0; i < chunk; ++i) {
    precond(s->kp, s->b_ph);
    launch_spmv(s, s->b_ph, s->kq, 0, st);   // v
    k_bi_alpha<<<nt, NT, 0, st>>>(s->b_r0, s->kq, tl, s->partials, s->counter, s->ks, s->n_done);
    k_bi_s<<<nt, NT, 0, st>>>(s->kr, s->kq, s->b_s, tl, s->partials, s->counter, s->ks);
    precond(s->b_s, s->b_sh);
    launch_spmv(s, s->b_sh, s->b_t, 0, st);  // t
    k_bi_omega<<<nt, NT, 0, st>>>(s->b_t, s->b_s, tl, s->partials, s->counter, s->ks);
    k_bi_update<<<nt, NT, 0, st>>>(s->kx, s->kr, s->b_ph, s->b_sh, s->b_s, s->b_t, s->b_r0, tl, s->partials,
                                   s->counter, s->ks, s->n_done);
    k_bi_pdir<<<nt, NT, 0, st>>>(s->kp, s->kr, s->kq, tl, s->ks);
    note_launches(5);
  }
  set_capturing(false);
  VAG_CUDA(cudaStreamEndCapture(st, &graph));
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  VAG_CUDA(cudaGraphInstantiate(&s->bicg_graph, graph, 0));
  cudaGraphDestroy(graph);
  const int ns = s->seg.n_sys;
  const int max_chunks = (o->maxit + chunk - 1) / chunk;
  for (int c = 0; c < max_chunks + 1; ++c) {
    VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (*s->n_done_host >= ns) break;
    VAG_CUDA(cudaGraphLaunch(s->bicg_graph, st));
    note_launches(nodes);
  }
  // the true residual decides the status
  launch_spmv(s, s->kx, s->kq, 0, st);
  k_resid2<<<nt, NT, 0, st>>>(s->rhs, s->kq, tl, s->partials, s->counter, s->ks);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  finish_solve(s, info, false);
  info->ms_setup = setup_ms;
  info->ms_solve -= setup_ms;
}

static vag_solve_info info_of(const KrylovScalars &k, bool mixed) {
  vag_solve_info o{};
  o.iterations = mixed ? k.inner_total : k.iter;
  o.outer = mixed ? k.iter : 1;
  o.rel_residual = k.bb > 0 ? sqrt(k.res2 / k.bb) : 0.0;
  o.status = k.breakdown ? VAG_EBREAKDOWN : (k.res2 > k.tol2 ? VAG_ENOTCONVERGED : VAG_OK);
  return o;
}

void finish_solve(System *s, vag_solve_info *info, bool mixed) {
  cudaStream_t st = s->ctx->stream;
  const int n = s->n_rows, ns = s->seg.n_sys;
  k_scatter_rows<<<grid_for(n, NT), NT, 0, st>>>(n, s->dof_of_row, s->kx, s->u);
  note_launches(1);
  k_scatter_dir<<<grid_for(s->nd, NT), NT, 0, st>>>(s->nd, s->dir_nodes, s->dir_vals, s->u);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  recover_cells_and_fluxes(s);
  trace_mark(st, "scatter + cell recovery + fluxes");
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaMemcpyAsync(s->ks_host, s->ks, sizeof(KrylovScalars) * ns, cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  // aggregate over the batch: most iterations, worst residual, worst status
  vag_solve_info agg{};
  agg.ms_solve = ms;
  agg.status = VAG_OK;
  for (int i = 0; i < ns; ++i) {
    const vag_solve_info o = info_of(s->ks_host[i], mixed);
    agg.iterations = std::max(agg.iterations, o.iterations);
    agg.outer = std::max(agg.outer, o.outer);
    agg.rel_residual = std::max(agg.rel_residual, o.rel_residual);
    if (o.status == VAG_EBREAKDOWN) agg.status = VAG_EBREAKDOWN;
    else if (o.status == VAG_ENOTCONVERGED && agg.status == VAG_OK) agg.status = VAG_ENOTCONVERGED;
  }
  *info = agg;
  s->solved = true;
  s->last_mixed = mixed;
}

void solve_infos(const System *s, vag_solve_info *infos) {
  for (int i = 0; i < s->seg.n_sys; ++i) infos[i] = info_of(s->ks_host[i], s->last_mixed);
}

}  // namespace vag
