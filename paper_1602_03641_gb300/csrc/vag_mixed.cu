// Mixed-precision solve of the eliminated system: FP64 iterative refinement
// around an FP32 conjugate-gradient inner solve.
//
// With s = D^{-1/2} (D the diagonal of A) the inner operator is the FP32 copy
// of S A S, which has a unit diagonal (the Jacobi preconditioner is folded
// in).  One refinement step, per system of the batch:
//   r = b - A x            FP64 SpMV (k_spmv of the FP64 path) and k_ir_resid
//   solve (S A S) y = S r  FP32 CG to ||res|| <= eta ||S r||
//   x += S y               FP64
// until ||r|| <= rtol ||b|| in FP64.  The inner loop reads 8 bytes per stored
// nonzero and runs on FP32 FMAs: on GB300 both halve the cost of an FP64
// iteration, whose SpMV is limited by the FP64 pipe.  Every reduction is per
// system and deterministic, as in the FP64 path.
//
// With the AMG preconditioner (mixed_amg_solve) the inner solve is FP32 CG on
// A itself, preconditioned by the FP32 V-cycle, on the normalised residual
// r / ||r||, to a per-system relative tolerance
//   eta = clamp(0.3 sqrt(tol^2 / ||r||^2), eta_min, 0.1)
// so that the last refinement step solves only as far as the outer tolerance
// needs; the correction is x += ||r|| y.  The inner product uses the
// difference form of A,
//   (A p)_i = sum_{j != i} a_ij (p_j - p_i) + (sum_j a_ij) p_i,
// with the off-diagonal entries in FP32 (0 in the diagonal slot) and the row
// sum (FP64, rounded once) in an array of its own: rounding each entry of a VAG row to FP32 would break
// its zero row sum by about 6e-8 |a_ii|, a spurious reaction term that, at
// fracture/matrix contrasts near 1e6, changes the smooth modes of the inner
// operator; in difference form constants are annihilated exactly and p_j -
// p_i of nearby FP32 values is exact (Sterbenz).
#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int NT = 256;
constexpr double kEta = 1e-6;      // inner relative tolerance (within FP32 reach on S A S)
// smallest inner tolerance of the AMG-preconditioned inner CG: the first
// refinement step solves as far as FP32 goes, the second the rest (measured
// on the 128^3 DFN at ratios 1e2 / 1e4 / 1e6: 1e-6 gave 74 / 88 / 100 ms,
// 1e-4 gave 76 / 98 / 104 ms, 1e-2 gave 75 / 93 / 109 ms)
constexpr double kEtaAmg = 1e-6;
constexpr int kMaxOuter = 40;

Tiles tiles_of(const System *s) {
  return Tiles{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0, s->seg.sys_grp0,
               s->seg.n_tiles, s->seg.n_sys};
}

__global__ void k_dscale(int n, const double *__restrict__ dinv, double *__restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sc[i] = sqrt(dinv[i]);
}

template <int U>
__global__ void __launch_bounds__(NT) k_spmv32(const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                               const int *__restrict__ scol, const float *__restrict__ sval,
                                               const float *__restrict__ x, float *__restrict__ y, Tiles tl,
                                               double *partials, unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ks[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float dp = 0.f;
  for (int row = r0 + threadIdx.x; row < r1; row += NT) {
    const float s = sell_row<float, U>(row, rowptr, slice_ptr, scol, sval, x);
    y[row] = s;
    dp = fmaf(x[row], s, dp);
  }
  double v[1] = {(double)dp}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.pq = out[0];
    if (!(out[0] > 0.0)) {
      k.breakdown = 1;
      k.alpha = 0.0;
      k.done = 1;
      atomicAdd(n_done, 1);
    } else {
      k.alpha = k.rz / out[0];
    }
  }
}

__global__ void __launch_bounds__(NT) k_upd32(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
                                              const float *__restrict__ q, Tiles tl, double *partials, unsigned *counter,
                                              KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const float a = (float)ks[sys].alpha;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rr = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    x[i] = fmaf(a, p[i], x[i]);
    const float ri = fmaf(-a, q[i], r[i]);
    r[i] = ri;
    rr = fmaf(ri, ri, rr);
  }
  double v[1] = {(double)rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    k.iter += 1;
    if (out[0] <= k.tol2 || k.iter >= k.maxit || !(out[0] == out[0])) {
      k.done = 1;
      atomicAdd(n_done, 1);
    }
  }
}

__global__ void __launch_bounds__(NT) k_pdir32(float *__restrict__ p, const float *__restrict__ r, Tiles tl,
                                               const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const float b = (float)ks[sys].beta;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0 + threadIdx.x; i < r1; i += NT) p[i] = fmaf(b, p[i], r[i]);
}

// x = 0, r = b; outer scalars: bb, tol2, done.
__global__ void __launch_bounds__(NT) k_ir_init(const double *__restrict__ b, double *__restrict__ x,
                                                double *__restrict__ r, Tiles tl, double *partials, unsigned *counter,
                                                KrylovScalars *ko, int *n_done, double rtol, int maxit) {
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
    KrylovScalars &k = ko[sys];
    k.bb = out[0];
    k.rr = out[0];
    k.res2 = out[0];
    k.tol2 = rtol * rtol * out[0];
    k.iter = 0;
    k.maxit = maxit;
    k.inner_total = 0;
    k.stalled = 0;
    k.breakdown = 0;
    k.done = out[0] <= k.tol2 ? 1 : 0;
    if (k.done) atomicAdd(n_done, 1);
  }
}

// inner right-hand side S r in FP32, x32 = 0, p32 = r32; inner scalars.
__global__ void __launch_bounds__(NT) k_ir_prep(const double *__restrict__ r, const double *__restrict__ sc,
                                                float *__restrict__ r32, float *__restrict__ x32,
                                                float *__restrict__ p32, Tiles tl, double *partials, unsigned *counter,
                                                const KrylovScalars *ko, KrylovScalars *ki, int *n_done_in,
                                                double eta, int maxit_in) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const bool outer_done = ko[sys].done;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rr = 0.f;
  if (!outer_done) {
    for (int i = r0 + threadIdx.x; i < r1; i += NT) {
      const float v = (float)(sc[i] * r[i]);
      r32[i] = v;
      p32[i] = v;
      x32[i] = 0.f;
      rr = fmaf(v, v, rr);
    }
  }
  double v[1] = {(double)rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ki[sys];
    k.rz = out[0];
    k.bb = out[0];
    k.tol2 = eta * eta * out[0];
    k.iter = 0;
    k.maxit = maxit_in;
    k.breakdown = 0;
    k.beta = 0.0;
    k.done = (outer_done || !(out[0] > 0.0)) ? 1 : 0;
    if (k.done) atomicAdd(n_done_in, 1);
  }
}

__global__ void __launch_bounds__(NT) k_ir_correct(double *__restrict__ x, const float *__restrict__ x32,
                                                   const double *__restrict__ sc, Tiles tl, const KrylovScalars *ko) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ko[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0 + threadIdx.x; i < r1; i += NT) x[i] = fma(sc[i], (double)x32[i], x[i]);
}

// r = b - A x (Ax given) and the outer convergence test.
__global__ void __launch_bounds__(NT) k_ir_resid(const double *__restrict__ b, const double *__restrict__ Ax,
                                                 double *__restrict__ r, Tiles tl, double *partials, unsigned *counter,
                                                 KrylovScalars *ko, const KrylovScalars *ki, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ko[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  double rr = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const double ri = b[i] - Ax[i];
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  double v[1] = {rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ko[sys];
    const double prev = k.rr;
    k.rr = out[0];
    k.res2 = out[0];
    k.iter += 1;
    k.inner_total += ki[sys].iter;
    if (ki[sys].breakdown) k.breakdown = 1;
    // stop when the FP64 residual no longer halves: its rounding floor
    k.stalled = !(out[0] < 0.25 * prev);
    if (out[0] <= k.tol2 || k.iter >= k.maxit || k.stalled || !(out[0] == out[0])) {
      k.done = 1;
      atomicAdd(n_done, 1);
    }
  }
}

// ---- inner FP32 CG preconditioned by the FP32 AMG V-cycle ----

// FP32 difference-form values in the sliced-ELL layout (padding stays 0):
// off-diagonal entries as they are, 0 in the diagonal slot, and the row sum
// sum_j a_ij (FP64, rounded once) in its own array
__global__ void k_dform_vals(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                             const double *__restrict__ val, const int *__restrict__ slice_ptr,
                             float *__restrict__ out, float *__restrict__ rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rowptr[i], e = rowptr[i + 1];
  double rs = 0.0;
  for (int k = b; k < e; ++k) rs += val[k];
  const int base = slice_ptr[i >> 5] + (i & 31);
  for (int k = b; k < e; ++k) out[base + 32 * (k - b)] = col[k] == i ? 0.f : (float)val[k];
  rowsum[i] = (float)rs;
}

// q = A p in difference form and the partial p.q (as k_spmv32)
template <int U>
__global__ void __launch_bounds__(NT) k_spmv32d(const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                                const int *__restrict__ scol, const float *__restrict__ sval,
                                                const float *__restrict__ rowsum, const float *__restrict__ x,
                                                float *__restrict__ y, Tiles tl, double *partials, unsigned *counter,
                                                KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ks[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float dp = 0.f;
  for (int row = r0 + threadIdx.x; row < r1; row += NT) {
    const int len = rowptr[row + 1] - rowptr[row];
    const int base = slice_ptr[row >> 5] + (row & 31);
    const float pi = x[row];
    float s = 0.f;
#pragma unroll(U)
    for (int k = 0; k < len; ++k) {   // the diagonal slot holds 0 and x_i - x_i = 0
      const int idx = base + 32 * k;
      s = fmaf(sval[idx], x[scol[idx]] - pi, s);
    }
    s = fmaf(rowsum[row], pi, s);
    y[row] = s;
    dp = fmaf(pi, s, dp);
  }
  double v[1] = {(double)dp}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.pq = out[0];
    if (!(out[0] > 0.0)) {
      k.breakdown = 1;
      k.alpha = 0.0;
      k.done = 1;
      atomicAdd(n_done, 1);
    } else {
      k.alpha = k.rz / out[0];
    }
  }
}

// r32 = r / ||r|| (per system), x32 = 0; inner scalars and tolerance
__global__ void __launch_bounds__(NT) k_irm_prep(const double *__restrict__ r, float *__restrict__ r32,
                                                 float *__restrict__ x32, Tiles tl, double *partials,
                                                 unsigned *counter, const KrylovScalars *ko, KrylovScalars *ki,
                                                 int *n_done_in, double eta_min, int maxit_in) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const bool outer_done = ko[sys].done;
  const double inv = outer_done ? 0.0 : 1.0 / sqrt(ko[sys].rr);
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rr = 0.f;
  if (!outer_done) {
    for (int i = r0 + threadIdx.x; i < r1; i += NT) {
      const float v = (float)(r[i] * inv);
      r32[i] = v;
      x32[i] = 0.f;
      rr = fmaf(v, v, rr);
    }
  }
  double v[1] = {(double)rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ki[sys];
    const KrylovScalars &o = ko[sys];
    double eta = 0.3 * sqrt(o.tol2 / o.rr);
    eta = eta < eta_min ? eta_min : (eta > 0.1 ? 0.1 : eta);
    k.bb = out[0];
    k.rr = out[0];
    k.tol2 = eta * eta * out[0];
    k.iter = 0;
    k.maxit = maxit_in;
    k.breakdown = 0;
    k.beta = 0.0;
    k.rz = 0.0;
    k.done = (outer_done || !(out[0] > 0.0)) ? 1 : 0;
    if (k.done) atomicAdd(n_done_in, 1);
  }
}

// p32 = z32, rz = r.z (breakdown unless positive)
__global__ void __launch_bounds__(NT) k_irm_rz_start(const float *__restrict__ r, const float *__restrict__ z,
                                                     float *__restrict__ p, Tiles tl, double *partials,
                                                     unsigned *counter, KrylovScalars *ki, int *n_done_in) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ki[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rz = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    const float zi = z[i];
    p[i] = zi;
    rz = fmaf(r[i], zi, rz);
  }
  double v[1] = {(double)rz}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ki[sys];
    k.rz = out[0];
    if (!(out[0] > 0.0)) {
      k.breakdown = 1;
      k.done = 1;
      atomicAdd(n_done_in, 1);
    }
  }
}

// x += alpha p, r -= alpha q, r.r; the last tile counts the iteration and
// tests the inner tolerance
__global__ void __launch_bounds__(NT) k_irm_update(float *__restrict__ x, float *__restrict__ r,
                                                   const float *__restrict__ p, const float *__restrict__ q, Tiles tl,
                                                   double *partials, unsigned *counter, KrylovScalars *ki,
                                                   int *n_done_in, const float *__restrict__ sinv0,
                                                   float *__restrict__ t0, float omega) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ki[sys].done) return;
  const float a = (float)ki[sys].alpha;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rr = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) {
    x[i] = fmaf(a, p[i], x[i]);
    const float ri = fmaf(-a, q[i], r[i]);
    r[i] = ri;
    if (sinv0) t0[i] = omega * sinv0[i] * ri;   // the V-cycle's first sweep from zero
    rr = fmaf(ri, ri, rr);
  }
  double v[1] = {(double)rr}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ki[sys];
    k.rr = out[0];
    k.iter += 1;
    if (out[0] <= k.tol2 || k.iter >= k.maxit || !(out[0] == out[0])) {
      if (!(out[0] == out[0])) k.breakdown = 1;
      k.done = 1;
      atomicAdd(n_done_in, 1);
    }
  }
}

// beta = (r.z)_new / (r.z)_old
__global__ void __launch_bounds__(NT) k_irm_rz(const float *__restrict__ r, const float *__restrict__ z, Tiles tl,
                                               double *partials, unsigned *counter, KrylovScalars *ki,
                                               int *n_done_in) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ki[sys].done) return;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  float rz = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += NT) rz = fmaf(r[i], z[i], rz);
  double v[1] = {(double)rz}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ki[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    if (!(out[0] > 0.0)) {
      k.breakdown = 1;
      k.done = 1;
      atomicAdd(n_done_in, 1);
    }
  }
}

// p = z + beta p
__global__ void __launch_bounds__(NT) k_irm_pdir(float *__restrict__ p, const float *__restrict__ z, Tiles tl,
                                                 const KrylovScalars *ki) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  pdl_wait();
  pdl_trigger();
  if (ki[sys].done) return;
  const float b = (float)ki[sys].beta;
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0 + threadIdx.x; i < r1; i += NT) p[i] = fmaf(b, p[i], z[i]);
}

// x += ||r|| y (the outer residual norm of the step, before it is replaced)
__global__ void __launch_bounds__(NT) k_irm_correct(double *__restrict__ x, const float *__restrict__ y, Tiles tl,
                                                    const KrylovScalars *ko) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ko[sys].done) return;
  const double nr = sqrt(ko[sys].rr);
  const int r0 = tl.row0[t], r1 = tl.row1[t];
  for (int i = r0 + threadIdx.x; i < r1; i += NT) x[i] = fma(nr, (double)y[i], x[i]);
}

}  // namespace

// p = 1 (the product's input for the timing hook)
__global__ void k_fill32(int n, float v, float *__restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// FP32 work vectors and inner scalars of the refinement loop
static void ensure_ir_vectors(System *s) {
  if (s->mx.x32) return;
  const int n = s->n_rows, ns = s->seg.n_sys;
  s->mx.x32 = sys_alloc<float>(s, n);
  s->mx.r32 = sys_alloc<float>(s, n);
  s->mx.p32 = sys_alloc<float>(s, n);
  s->mx.q32 = sys_alloc<float>(s, n);
  s->mx.ks_in = sys_alloc<KrylovScalars>(s, ns);
  s->mx.n_done_in = sys_alloc<int>(s, 1);
}

static void ensure_mixed_buffers(System *s) {
  ensure_ir_vectors(s);
  if (s->mx.sval32) return;
  s->mx.sval32 = sys_alloc<float>(s, (size_t)s->sell_nnz);
  s->mx.sc = sys_alloc<double>(s, s->n_rows);
  s->mx.stale = true;
}

void mixed_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  auto spmv32 = s->sell_u == 2 ? k_spmv32<2> : s->sell_u == 8 ? k_spmv32<8> : k_spmv32<4>;
  cudaStream_t st = s->ctx->stream;
  ensure_mixed_buffers(s);
  Mixed &m = s->mx;
  const int n = s->n_rows, ns = s->seg.n_sys, nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  if (m.stale) {   // FP32 copy of S A S after every numeric phase
    k_dscale<<<grid_for(n, NT), NT, 0, st>>>(n, s->dinv, m.sc);
    note_launches(1);
    sell_values_scaled_f32(s, m.sc, m.sval32);
    m.stale = false;
  }
  VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
  k_ir_init<<<nt, NT, 0, st>>>(s->rhs, s->kx, s->kr, tl, s->partials, s->counter, s->ks, s->n_done, o->rtol,
                               kMaxOuter);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  const int chunk = 16;
  if (!m.graph) {
    cudaGraph_t graph;
    VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    for (int i = 0; i < chunk; ++i) {
      spmv32<<<nt, NT, 0, st>>>(s->rowptr, s->slice_ptr, s->scol, m.sval32, m.p32, m.q32, tl, s->partials,
                                s->counter, m.ks_in, m.n_done_in);
      k_upd32<<<nt, NT, 0, st>>>(m.x32, m.r32, m.p32, m.q32, tl, s->partials, s->counter, m.ks_in, m.n_done_in);
      k_pdir32<<<nt, NT, 0, st>>>(m.p32, m.r32, tl, m.ks_in);
    }
    set_capturing(false);
    VAG_CUDA(cudaStreamEndCapture(st, &graph));
    VAG_CUDA(cudaGraphInstantiate(&m.graph, graph, 0));
    cudaGraphDestroy(graph);
  }
  int outer = 0;
  for (; outer < kMaxOuter + 1; ++outer) {
    VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (*s->n_done_host >= ns) break;
    VAG_CUDA(cudaMemsetAsync(m.n_done_in, 0, sizeof(int), st));
    k_ir_prep<<<nt, NT, 0, st>>>(s->kr, m.sc, m.r32, m.x32, m.p32, tl, s->partials, s->counter, s->ks, m.ks_in,
                                 m.n_done_in, kEta, o->maxit);
    note_launches(1);
    for (int c = 0; c < (o->maxit + chunk - 1) / chunk + 1; ++c) {
      VAG_CUDA(cudaMemcpyAsync(s->n_done_host, m.n_done_in, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*s->n_done_host >= ns) break;
      VAG_CUDA(cudaGraphLaunch(m.graph, st));
      note_launches(3ull * chunk);
    }
    k_ir_correct<<<nt, NT, 0, st>>>(s->kx, m.x32, m.sc, tl, s->ks);
    note_launches(1);
    spmv_f64(s, s->kx, s->kq);
    k_ir_resid<<<nt, NT, 0, st>>>(s->rhs, s->kq, s->kr, tl, s->partials, s->counter, s->ks, m.ks_in, s->n_done);
    note_launches(1);
    VAG_CHECK_LAUNCH();
  }
  finish_solve(s, info, /*mixed=*/true);
}

void mixed_amg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
  tune_sell(s);
  ensure_ir_vectors(s);
  Mixed &m = s->mx;
  if (!m.z32) m.z32 = sys_alloc<float>(s, s->n_rows);
  const int ns = s->seg.n_sys, nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  amg_setup(s, /*f32=*/true, o->precision == VAG_MIXED_F16, o->precond == VAG_PC_AMG_RS);
  if (!m.dval32) {
    m.dval32 = sys_alloc<float>(s, (size_t)std::max<int64_t>(s->sell_nnz, 1));
    m.rowsum32 = sys_alloc<float>(s, (size_t)s->n_rows);
    m.dstale = true;
  }
  if (m.dstale) {   // after every numeric phase
    VAG_CUDA(cudaMemsetAsync(m.dval32, 0, sizeof(float) * (size_t)s->sell_nnz, st));
    k_dform_vals<<<grid_for(s->n_rows, NT), NT, 0, st>>>(s->n_rows, s->rowptr, s->col, s->val, s->slice_ptr,
                                                          m.dval32, m.rowsum32);
    note_launches(1);
    VAG_CHECK_LAUNCH();
    m.dstale = false;
  }
  trace_mark(st, "AMG setup (FP32 hierarchy), difference-form FP32 values");
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float setup_ms = 0.f;
  cudaEventElapsedTime(&setup_ms, s->ev0, s->ev1);
  const float *a32 = m.dval32;   // FP32 difference-form values of A, sliced ELL
  auto spmv32 = s->sell_u == 2 ? k_spmv32d<2> : s->sell_u == 8 ? k_spmv32d<8> : k_spmv32d<4>;
  // one inner iteration: q = A p (p.q, alpha), x/r update, z = V(r), r.z, p
  // the V-cycle's first sweep is formed by the update and its last sweep
  // forms r.z (the same arithmetic as the separate kernels)
  float *t0 = nullptr;
  float omega = 0.f;
  const float *sinv0 = amg_first_sweep_scale_f32(s, t0, omega);
  auto iteration = [&]() {
    launch_pdl(spmv32, nt, NT, 0, st, (const int *)s->rowptr, (const int *)s->slice_ptr, (const int *)s->scol, a32,
               (const float *)m.rowsum32, (const float *)m.p32, m.q32, tl, s->partials, s->counter, m.ks_in,
               m.n_done_in);
    launch_pdl(k_irm_update, nt, NT, 0, st, m.x32, m.r32, (const float *)m.p32, (const float *)m.q32, tl, s->partials,
               s->counter, m.ks_in, m.n_done_in, sinv0, t0, omega);
    const bool rz_done = sinv0 ? amg_apply_f32_cg(s, m.r32, m.z32, st, m.ks_in, m.n_done_in)
                               : (amg_apply_f32(s, m.r32, m.z32, st), false);
    if (!rz_done) {
      launch_pdl(k_irm_rz, nt, NT, 0, st, (const float *)m.r32, (const float *)m.z32, tl, s->partials, s->counter,
                 m.ks_in, m.n_done_in);
      note_launches(1);
    }
    launch_pdl(k_irm_pdir, nt, NT, 0, st, m.p32, (const float *)m.z32, tl, (const KrylovScalars *)m.ks_in);
    note_launches(3);
  };
  VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
  k_ir_init<<<nt, NT, 0, st>>>(s->rhs, s->kx, s->kr, tl, s->partials, s->counter, s->ks, s->n_done, o->rtol,
                               kMaxOuter);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  // the hierarchy is rebuilt every solve, so is the graph of inner iterations
  const int chunk = 8;
  if (m.graph_amg) {
    cudaGraphExecDestroy(m.graph_amg);
    m.graph_amg = nullptr;
  }
  {
    cudaGraph_t graph;
    VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    for (int i = 0; i < chunk; ++i) iteration();
    set_capturing(false);
    VAG_CUDA(cudaStreamEndCapture(st, &graph));
    cudaGraphGetNodes(graph, nullptr, &m.graph_amg_nodes);
    VAG_CUDA(cudaGraphInstantiate(&m.graph_amg, graph, 0));
    cudaGraphDestroy(graph);
    trace_mark(st, "graph capture + instantiate");
  }
  const double eta_min = o->inner_rtol > 0.0 ? o->inner_rtol : kEtaAmg;
  for (int outer = 0; outer < kMaxOuter + 1; ++outer) {
    VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (*s->n_done_host >= ns) break;
    VAG_CUDA(cudaMemsetAsync(m.n_done_in, 0, sizeof(int), st));
    k_irm_prep<<<nt, NT, 0, st>>>(s->kr, m.r32, m.x32, tl, s->partials, s->counter, s->ks, m.ks_in, m.n_done_in,
                                  eta_min, o->maxit);
    note_launches(1);
    amg_apply_f32(s, m.r32, m.z32, st);
    launch_pdl(k_irm_rz_start, nt, NT, 0, st, (const float *)m.r32, (const float *)m.z32, m.p32, tl, s->partials,
               s->counter, m.ks_in, m.n_done_in);
    note_launches(1);
    VAG_CHECK_LAUNCH();
    for (int c = 0; c < (o->maxit + chunk - 1) / chunk + 1; ++c) {
      VAG_CUDA(cudaMemcpyAsync(s->n_done_host, m.n_done_in, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*s->n_done_host >= ns) break;
      VAG_CUDA(cudaGraphLaunch(m.graph_amg, st));
      note_launches(m.graph_amg_nodes);
    }
    k_irm_correct<<<nt, NT, 0, st>>>(s->kx, m.x32, tl, s->ks);
    note_launches(1);
    spmv_f64(s, s->kx, s->kq);
    k_ir_resid<<<nt, NT, 0, st>>>(s->rhs, s->kq, s->kr, tl, s->partials, s->counter, s->ks, m.ks_in, s->n_done);
    note_launches(1);
    VAG_CHECK_LAUNCH();
    trace_mark(st, "refinement step");
  }
  finish_solve(s, info, /*mixed=*/true);
  info->ms_setup = setup_ms;
  info->ms_solve -= setup_ms;
}

// Mean duration of the inner product q = A p with its p.q reduction, as the
// inner CG of mixed_amg_solve launches it (p = 1, every system active).
double time_spmv32(System *s, int reps) {
  if (!s->mx.dval32 || s->mx.dstale || !s->mx.z32)
    fail(VAG_EINVAL, "no FP32 inner solve: solve with VAG_MIXED and VAG_PC_AMG first");
  cudaStream_t st = s->ctx->stream;
  Mixed &m = s->mx;
  const int n = s->n_rows, ns = s->seg.n_sys, nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  auto spmv32 = s->sell_u == 2 ? k_spmv32d<2> : s->sell_u == 8 ? k_spmv32d<8> : k_spmv32d<4>;
  k_fill32<<<grid_for(n, NT), NT, 0, st>>>(n, 1.0f, m.p32);
  note_launches(1);
  VAG_CUDA(cudaMemsetAsync(m.ks_in, 0, sizeof(KrylovScalars) * ns, st));   // done = 0 everywhere
  auto launch = [&]() {
    launch_pdl(spmv32, nt, NT, 0, st, (const int *)s->rowptr, (const int *)s->slice_ptr, (const int *)s->scol,
               (const float *)m.dval32, (const float *)m.rowsum32, (const float *)m.p32, m.q32, tl, s->partials,
               s->counter, m.ks_in, m.n_done_in);
    note_launches(1);
  };
  launch();   // warm-up
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  for (int r = 0; r < reps; ++r) launch();
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  return (double)ms / reps;
}

}  // namespace vag
