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
#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int NT = 256;
constexpr double kEta = 1e-6;      // inner relative tolerance (within FP32 reach on S A S)
constexpr int kMaxOuter = 40;

Tiles tiles_of(const System *s) {
  return Tiles{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0};
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

}  // namespace

static void ensure_mixed_buffers(System *s) {
  if (s->mx.sval32) return;
  const int n = s->n_rows, ns = s->seg.n_sys;
  s->mx.sval32 = sys_alloc<float>(s, (size_t)s->sell_nnz);
  s->mx.x32 = sys_alloc<float>(s, n);
  s->mx.r32 = sys_alloc<float>(s, n);
  s->mx.p32 = sys_alloc<float>(s, n);
  s->mx.q32 = sys_alloc<float>(s, n);
  s->mx.sc = sys_alloc<double>(s, n);
  s->mx.ks_in = sys_alloc<KrylovScalars>(s, ns);
  s->mx.n_done_in = sys_alloc<int>(s, 1);
  s->mx.stale = true;
}

void mixed_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  ensure_krylov_buffers(s);
  tune_sell(s);
  auto spmv32 = s->sell_u == 2 ? k_spmv32<2> : s->sell_u == 8 ? k_spmv32<8> : k_spmv32<4>;
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
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

}  // namespace vag
