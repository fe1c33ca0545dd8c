// Krylov solve of the cell-eliminated system (Sec. 4.2, Eq. eqschur).
//
// The system is the Galerkin form restricted to the non-Dirichlet unknowns,
// hence symmetric positive definite: conjugate gradients with a Jacobi
// preconditioner.  Per iteration three kernels:
//   k_spmv<G>   q = A p (G lanes per CSR row) fused with the partial p.q,
//               the last block computes alpha = r.z / p.q;
//   k_update    x += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r,
//               the last block computes beta and the convergence flag;
//   k_pdir      p = z + beta p.
// Reductions are deterministic (fixed grid, fixed summation order).  The
// iteration is captured in a CUDA graph of `chunk` iterations; once the
// device flag `done` is set every kernel returns at entry, so the host polls
// the flag only between graph launches.
#include "vag_internal.cuh"
#include "vag_reduce.cuh"
#include "vag_hex.cuh"

namespace vag {
namespace {

constexpr int NT = 256;

template <int G>
__global__ void __launch_bounds__(NT) k_spmv(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                             const double *__restrict__ val, const double *__restrict__ x,
                                             double *__restrict__ y, double *partials, unsigned *counter,
                                             KrylovScalars *ks, int with_dot) {
  if (with_dot && ks->done) return;
  const int lane = threadIdx.x & (G - 1);
  const int warp_global = (blockIdx.x * NT + threadIdx.x) >> 5;
  const int warps_total = (gridDim.x * NT) >> 5;
  constexpr int RPW = 32 / G;   // rows per warp per sweep
  const int sub = (threadIdx.x & 31) / G;
  double dp = 0.0;
  for (int base = warp_global * RPW; base < n; base += warps_total * RPW) {
    const int row = base + sub;
    double s = 0.0;
    if (row < n) {
      const int b = rowptr[row], e = rowptr[row + 1];
      for (int k = b + lane; k < e; k += G) s = fma(val[k], __ldg(&x[col[k]]), s);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && lane == 0) {
      y[row] = s;
      dp = fma(x[row], s, dp);
    }
  }
  if (!with_dot) return;
  double v[1] = {dp}, out[1];
  if (grid_sum<NT, 1>(v, partials, counter, out) && threadIdx.x == 0) {
    const double pq = out[0];
    ks->pq = pq;
    if (!(pq > 0.0)) {
      ks->breakdown = 1;
      ks->done = 1;
      ks->alpha = 0.0;
    } else {
      ks->alpha = ks->rz / pq;
    }
  }
}

__global__ void __launch_bounds__(NT) k_init(int n, const double *__restrict__ b, const double *__restrict__ dinv,
                                             double *__restrict__ x, double *__restrict__ r, double *__restrict__ p,
                                             double *partials, unsigned *counter, KrylovScalars *ks, double rtol,
                                             int maxit) {
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    const double bi = b[i];
    const double zi = dinv[i] * bi;
    x[i] = 0.0;
    r[i] = bi;
    p[i] = zi;
    rz = fma(bi, zi, rz);
    rr = fma(bi, bi, rr);
  }
  double v[2] = {rz, rr}, out[2];
  if (grid_sum<NT, 2>(v, partials, counter, out) && threadIdx.x == 0) {
    ks->rz = out[0];
    ks->rr = out[1];
    ks->bb = out[1];
    ks->tol2 = rtol * rtol * out[1];
    ks->iter = 0;
    ks->maxit = maxit;
    ks->breakdown = 0;
    ks->done = (out[1] <= ks->tol2) ? 1 : 0;
    ks->beta = 0.0;
  }
}

__global__ void __launch_bounds__(NT) k_update(int n, double *__restrict__ x, double *__restrict__ r,
                                               const double *__restrict__ p, const double *__restrict__ q,
                                               const double *__restrict__ dinv, double *partials,
                                               unsigned *counter, KrylovScalars *ks) {
  if (ks->done) return;
  const double alpha = ks->alpha;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rz = fma(ri, dinv[i] * ri, rz);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {rz, rr}, out[2];
  if (grid_sum<NT, 2>(v, partials, counter, out) && threadIdx.x == 0) {
    const double rzn = out[0];
    ks->beta = rzn / ks->rz;
    ks->rz = rzn;
    ks->rr = out[1];
    ks->iter += 1;
    if (out[1] <= ks->tol2 || ks->iter >= ks->maxit) ks->done = 1;
    if (!(out[1] == out[1])) { ks->breakdown = 1; ks->done = 1; }
  }
}

__global__ void __launch_bounds__(NT) k_pdir(int n, double *__restrict__ p, const double *__restrict__ r,
                                             const double *__restrict__ dinv, const KrylovScalars *ks) {
  if (ks->done) return;
  const double beta = ks->beta;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) p[i] = fma(beta, p[i], dinv[i] * r[i]);
}

__global__ void __launch_bounds__(NT) k_resid2(int n, const double *__restrict__ b, const double *__restrict__ Ax,
                                               double *partials, unsigned *counter, KrylovScalars *ks) {
  double s = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    const double d = b[i] - Ax[i];
    s = fma(d, d, s);
  }
  double v[1] = {s}, out[1];
  if (grid_sum<NT, 1>(v, partials, counter, out) && threadIdx.x == 0) ks->res2 = out[0];
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

}  // namespace

int spmv_group(const System *s) {
  const double avg = s->n_rows ? (double)s->nnz / s->n_rows : 1.0;
  return avg <= 10.0 ? 4 : (avg <= 40.0 ? 8 : 16);
}

int red_grid(int64_t n) {
  const int64_t want = (n + NT - 1) / NT;
  int64_t g = std::min<int64_t>((int64_t)num_sms() * 4, want);
  if (g < 1) g = 1;
  if (g > kMaxRedBlocks) g = kMaxRedBlocks;
  return (int)g;
}

static void launch_spmv(System *s, const double *x, double *y, int with_dot, cudaStream_t st) {
  const int G = spmv_group(s);
  const int rows_per_block = NT / G;
  int64_t want = (s->n_rows + rows_per_block - 1) / rows_per_block;
  int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)num_sms() * 8);
  if (grid > kMaxRedBlocks) grid = kMaxRedBlocks;
  switch (G) {
    case 4:
      k_spmv<4><<<grid, NT, 0, st>>>(s->n_rows, s->rowptr, s->col, s->val, x, y, s->partials, s->counter, s->ks, with_dot);
      break;
    case 8:
      k_spmv<8><<<grid, NT, 0, st>>>(s->n_rows, s->rowptr, s->col, s->val, x, y, s->partials, s->counter, s->ks, with_dot);
      break;
    default:
      k_spmv<16><<<grid, NT, 0, st>>>(s->n_rows, s->rowptr, s->col, s->val, x, y, s->partials, s->counter, s->ks, with_dot);
  }
}

static void ensure_krylov_buffers(System *s) {
  if (s->kx) return;
  s->kx = sys_alloc<double>(s, s->n_rows);
  s->kr = sys_alloc<double>(s, s->n_rows);
  s->kp = sys_alloc<double>(s, s->n_rows);
  s->kq = sys_alloc<double>(s, s->n_rows);
  s->partials = sys_alloc<double>(s, 4 * (size_t)kMaxRedBlocks);
  s->counter = sys_alloc<unsigned>(s, 4);
  s->ks = sys_alloc<KrylovScalars>(s, 1);
  s->u = sys_alloc<double>(s, (size_t)s->n_cv);
  VAG_CUDA(cudaMemsetAsync(s->counter, 0, 4 * sizeof(unsigned), s->ctx->stream));
  VAG_CUDA(cudaMemsetAsync(s->u, 0, sizeof(double) * s->n_cv, s->ctx->stream));
  if (!s->ks_host) VAG_CUDA(cudaMallocHost(&s->ks_host, sizeof(KrylovScalars)));
}

void spmv_f64(System *s, const double *x, double *y) {
  ensure_krylov_buffers(s);
  launch_spmv(s, x, y, 0, s->ctx->stream);
  VAG_CHECK_LAUNCH();
}

static void pcg_iteration(System *s, cudaStream_t st) {
  const int g = red_grid(s->n_rows);
  launch_spmv(s, s->kp, s->kq, 1, st);
  k_update<<<g, NT, 0, st>>>(s->n_rows, s->kx, s->kr, s->kp, s->kq, s->dinv, s->partials, s->counter, s->ks);
  k_pdir<<<g, NT, 0, st>>>(s->n_rows, s->kp, s->kr, s->dinv, s->ks);
}

void pcg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
  const int n = s->n_rows;
  const int g = red_grid(n);
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  k_init<<<g, NT, 0, st>>>(n, s->rhs, s->dinv, s->kx, s->kr, s->kp, s->partials, s->counter, s->ks, o->rtol,
                           o->maxit);
  VAG_CHECK_LAUNCH();
  // graph of `chunk` iterations, captured once per system
  const int chunk = 16;
  if (!s->pcg_graph || s->pcg_graph_chunk != chunk) {
    if (s->pcg_graph) cudaGraphExecDestroy(s->pcg_graph);
    cudaGraph_t graph;
    VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) pcg_iteration(s, st);
    VAG_CUDA(cudaStreamEndCapture(st, &graph));
    VAG_CUDA(cudaGraphInstantiate(&s->pcg_graph, graph, 0));
    cudaGraphDestroy(graph);
    s->pcg_graph_chunk = chunk;
  }
  const int max_chunks = (o->maxit + chunk - 1) / chunk;
  for (int c = 0; c < max_chunks + 1; ++c) {
    VAG_CUDA(cudaGraphLaunch(s->pcg_graph, st));
    VAG_CUDA(cudaMemcpyAsync(s->ks_host, s->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (s->ks_host->done) break;
  }
  // true residual and the full solution vector
  launch_spmv(s, s->kx, s->kq, 0, st);
  k_resid2<<<g, NT, 0, st>>>(n, s->rhs, s->kq, s->partials, s->counter, s->ks);
  k_scatter_rows<<<grid_for(n, NT), NT, 0, st>>>(n, s->dof_of_row, s->kx, s->u);
  k_scatter_dir<<<grid_for(s->nd, NT), NT, 0, st>>>(s->nd, s->dir_nodes, s->dir_vals, s->u);
  VAG_CHECK_LAUNCH();
  recover_cells_and_fluxes(s);
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaMemcpyAsync(s->ks_host, s->ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  const KrylovScalars &k = *s->ks_host;
  info->iterations = k.iter;
  info->outer = 1;
  info->rel_residual = k.bb > 0 ? sqrt(k.res2 / k.bb) : 0.0;
  info->ms_setup = 0.0;
  info->ms_solve = ms;
  if (k.breakdown) info->status = VAG_EBREAKDOWN;
  else if (k.rr > k.tol2) info->status = VAG_ENOTCONVERGED;
  else info->status = VAG_OK;
  s->solved = true;
}

}  // namespace vag
