// Chebyshev polynomial preconditioner of the Jacobi-scaled operator D^-1 A
// for the Krylov solve of the cell-eliminated system (Sec. 4.2, Eq. eqschur).
//
// z = M r is the iterate after kChebDegree steps of Chebyshev acceleration of
// the Jacobi iteration for A z = r from z = 0 on an interval [a, b] that
// should hold the spectrum of D^-1 A (Saad, Iterative Methods for Sparse
// Linear Systems, 2nd ed., Sec. 12.3, Alg. 12.1):
//   theta = (b + a)/2, delta = (b - a)/2, sigma = theta/delta, rho_0 = 1/sigma,
//   d_1 = D^-1 r / theta,  z_1 = d_1,
//   rho_j = 1/(2 sigma - rho_{j-1}),
//   d_{j+1} = rho_j rho_{j-1} d_j + (2 rho_j/delta) D^-1 (r - A z_j),
//   z_{j+1} = z_j + d_{j+1}.
// M = p(D^-1 A) D^-1 for a polynomial p, so M is symmetric.  The residual
// polynomial 1 - l p(l) = T_k((theta - l)/delta) / T_k(sigma) has modulus
// below 1 for 0 < l < b + a, so p > 0 there and M is positive definite
// whenever the spectrum of D^-1 A lies below b + a: CG may use it.
//
// Bounds: b = kChebSafety x the largest Ritz value of D^-1 A after
// kLanczosSteps steps of Jacobi-preconditioned CG from a pseudo-random start
// vector (CG's alpha_j, beta_j are the entries of the Lanczos tridiagonal,
// Saad Sec. 6.7.3); a = b / kChebRatio.  Every system of a batch has its own
// interval, start vector (a function of its local row index alone) and
// coefficient table, so a system is bitwise the same alone or in a batch.
//
// Per application: the first step (D^-1 r, folded into the CG update kernel
// inside the iteration), then kChebDegree - 1 fused sliced-ELL steps, the last
// of which also forms r.z for CG's beta.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "vag_cheb_host.h"
#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int NT = 256;
constexpr int kChebDegree = 4;
constexpr int kLanczosSteps = 10;
constexpr double kChebSafety = 1.2;
constexpr double kChebRatio = 100.0;
constexpr int kCoefStride = 2 * kChebDegree;

Tiles tiles_of(const System *s) {
  return Tiles{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0, s->seg.sys_grp0,
               s->seg.n_tiles, s->seg.n_sys};
}

// Pseudo-random start vector, uniform in [-1, 1): the SplitMix64 output
// function (Steele, Lea & Flood, OOPSLA 2014) of the row's index inside its
// own system.
__global__ void __launch_bounds__(NT) k_start_vector(Tiles tl, double *__restrict__ v) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int first = tl.row0[tl.sys_tile0[sys]];
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    uint64_t z = (uint64_t)(i - first + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

// w = D^-1 r (the first step before the 1/theta scale, which the next step
// applies)
__global__ void __launch_bounds__(NT) k_jacobi_scale(const double *__restrict__ r, const double *__restrict__ dinv,
                                                     double *__restrict__ w, Tiles tl) {
  const int t = blockIdx.x;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) w[i] = dinv[i] * r[i];
}

// Step j >= 1 of the recurrence, one thread per row.  For j = 1 the incoming
// d and z are both w = D^-1 r and carry the factor 1/theta (s_in), applied
// here.  d_in and d_out may be the same buffer (each row reads its own entry
// before writing it).  in_iter: inside a Krylov iteration, where systems
// already done return at entry.  with_rz: also r.z and, in the last tile of
// the system, beta = (r.z)' / (r.z), as k_rz does.
template <int U>
__global__ void __launch_bounds__(NT) k_cheb_step(const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                                  const int *__restrict__ scol, const double *__restrict__ sval,
                                                  const double *__restrict__ dinv, const double *__restrict__ r,
                                                  const double *__restrict__ coef, int j, const double *d_in,
                                                  const double *__restrict__ z_in, double *d_out,
                                                  double *__restrict__ z_out, Tiles tl, double *partials,
                                                  unsigned *counter, KrylovScalars *ks, int *n_done, int in_iter,
                                                  int with_rz) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int i = tl.row0[t] + threadIdx.x;
  const bool valid = i < tl.row1[t];
  const double *c = coef + (size_t)kCoefStride * sys;
  pdl_wait();
  pdl_trigger();
  if (in_iter && ks[sys].done) return;   // uniform in the block: one system per tile
  double rz = 0.0;
  if (valid) {
    const double ri = r[i];
    double di, zi;
    cheb_row_step(c, j, ri, sell_row<double, U>(i, rowptr, slice_ptr, scol, sval, z_in), dinv[i], d_in[i], z_in[i],
                  &di, &zi);
    if (d_out) d_out[i] = di;
    z_out[i] = zi;
    rz = ri * zi;
  }
  if (!with_rz) return;
  double v[1] = {rz}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    if (!(out[0] > 0.0)) { k.breakdown = 1; k.done = 1; atomicAdd(n_done, 1); }
  }
}

}  // namespace

void cheb_setup(System *s) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  const int ns = s->seg.n_sys;
  cudaStream_t st = s->ctx->stream;
  if (!s->cheb_coef) {
    s->cheb_coef = sys_alloc<double>(s, (size_t)kCoefStride * ns);
    s->cw = sys_alloc<double>(s, s->n_rows);
    s->cd = sys_alloc<double>(s, s->n_rows);
    s->cy = sys_alloc<double>(s, s->n_rows);
    if (!s->kz) s->kz = sys_alloc<double>(s, s->n_rows);
  }
  const Tiles tl = tiles_of(s);
  k_start_vector<<<s->seg.n_tiles, NT, 0, st>>>(tl, s->cy);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  std::vector<double> alpha, beta;
  std::vector<int> steps;
  jacobi_cg_coefficients(s, s->cy, kLanczosSteps, alpha, beta, steps);
  std::vector<double> coef((size_t)kCoefStride * ns, 0.0);
  s->cheb_bounds.assign(2 * (size_t)ns, 0.0);
  for (int sy = 0; sy < ns; ++sy) {
    // no Lanczos step (empty system or immediate breakdown): b = 2
    const double b = cheb_upper_bound(&alpha[(size_t)sy * kLanczosSteps], &beta[(size_t)sy * kLanczosSteps],
                                      steps[sy], kChebSafety);
    const double a = b / kChebRatio;
    cheb_table(a, b, kChebDegree, &coef[(size_t)kCoefStride * sy]);
    s->cheb_bounds[2 * sy] = a;
    s->cheb_bounds[2 * sy + 1] = b;
  }
  VAG_CUDA(cudaMemcpyAsync(s->cheb_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st));
  VAG_CUDA(cudaStreamSynchronize(st));   // the host table goes out of scope
  if (trace_enabled()) {
    for (int sy = 0; sy < ns && sy < 8; ++sy)
      std::fprintf(stderr, "[vag trace] Chebyshev system %d: %d Lanczos steps, interval [%.4g, %.4g]\n", sy,
                   steps[sy], s->cheb_bounds[2 * sy], s->cheb_bounds[2 * sy + 1]);
  }
}

void cheb_apply(System *s, const double *r, double *z, cudaStream_t st, bool in_iter, bool w_ready, bool rz) {
  const Tiles tl = tiles_of(s);
  const int nt = s->seg.n_tiles;
  if (!w_ready) {
    k_jacobi_scale<<<nt, NT, 0, st>>>(r, s->dinv, s->cw, tl);
    note_launches(1);
  }
  auto step = s->sell_u == 2 ? k_cheb_step<2> : s->sell_u == 8 ? k_cheb_step<8> : k_cheb_step<4>;
  const double *d_in = s->cw, *z_in = s->cw;
  for (int j = 1; j < kChebDegree; ++j) {
    const bool last = j == kChebDegree - 1;
    double *z_out = last ? z : (z_in == s->cy ? s->cw : s->cy);
    double *d_out = last ? nullptr : s->cd;
    launch_pdl(step, nt, NT, 0, st, (const int *)s->rowptr, (const int *)s->slice_ptr, (const int *)s->scol,
               (const double *)s->sval, (const double *)s->dinv, r, (const double *)s->cheb_coef, j, d_in, z_in,
               d_out, z_out, tl, s->partials, s->counter, s->ks, s->n_done, (int)in_iter, (int)(last && rz));
    note_launches(1);
    d_in = s->cd;
    z_in = z_out;
  }
}

}  // namespace vag
