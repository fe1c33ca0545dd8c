// Restarted GMRES(m) on the cell-eliminated system (Sec. 4.2, Eq. eqschur):
// the Krylov method of the paper's solver experiments (Sec. 5.3) beside
// BiCGStab, right-preconditioned (Jacobi, Chebyshev-Jacobi or the AMG
// V-cycle), m = kRestart.  Arnoldi with classical Gram-Schmidt applied twice
// (Giraud, Langou, Rozloznik 2005: two passes give an orthogonal basis to
// working precision), the Hessenberg columns reduced by Givens rotations as
// they come (Saad & Schultz 1986), so |g_{j+1}| is the residual norm of the
// current iterate; at the end of a cycle x += M V_k y with R y = g.  Every
// cycle starts from the true residual r = b - A x; a system stops when that
// residual meets the tolerance, when the iteration cap is reached, or when a
// whole cycle no longer lowers it (the rounding floor).
//
// Batches: per-system tiles, Hessenberg data and flags; the dot products of a
// tile are summed in a fixed order and the tiles of a system in tile order,
// so a system is bitwise the same alone or in a batch.  Systems done return
// at entry.  Each cycle runs as CUDA graphs of kChunk Arnoldi steps, the
// host polling the count of systems done between graphs.
#include <cmath>
#include <cstdio>
#include <vector>

#include "vag_gmres_ls.h"
#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int NT = 256;
constexpr int kRestart = 30;           // m
constexpr int kMaxK = 32;              // >= m + 1 (dot products of one pass)
constexpr int kChunk = 5;              // Arnoldi steps per CUDA graph
constexpr double kStall = 0.9999;      // a cycle must lower ||r|| below kStall x its start

// Per-system GMRES state (device).
struct GmState {
  double h1[kMaxK], h2[kMaxK];         // the two Gram-Schmidt passes of the current column
  double R[kRestart][kRestart];        // R[j][i]: column j of the rotated Hessenberg matrix
  double cs[kRestart], sn[kRestart];   // Givens rotations
  double g[kRestart + 1];              // rotated right-hand side
  double y[kRestart];                  // cycle's coefficients
  double hn;                           // norm of the new Arnoldi vector
  double beta, beta_prev;              // ||r|| at this and the previous cycle start
  int k;                               // Arnoldi steps made in this cycle
  int final;                           // no further cycle
};

Tiles tiles_of(const System *s) {
  return Tiles{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0, s->seg.sys_grp0,
               s->seg.n_tiles, s->seg.n_sys};
}

// Sum over the 32 lanes of a warp (all lanes get the total).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// h[q] = V_q . w for q <= j: one pass of Gram-Schmidt.  Per tile, the 8
// warps' sums are added in warp order; the last tile of a system adds its
// system's tile sums in a fixed order (8 lanes per value, tiles dealt
// round-robin by their index inside the system, lanes combined by a fixed
// butterfly).
__global__ void __launch_bounds__(NT) k_gm_dots(const double *__restrict__ V, size_t ldv, int j,
                                                const double *__restrict__ w, Tiles tl, double *gpart,
                                                unsigned *counter, const KrylovScalars *ks, GmState *gs, int pass) {
  __shared__ double red[NT / 32][kMaxK];
  __shared__ bool last;
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;   // uniform in the block: one system per tile
  const int nk = j + 1;
  const int i = tl.row0[t] + threadIdx.x;
  const bool valid = i < tl.row1[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double wi = valid ? w[i] : 0.0;
  for (int q = 0; q < nk; ++q) {
    const double p = warp_sum(valid ? V[(size_t)q * ldv + i] * wi : 0.0);
    if (lane == 0) red[warp][q] = p;
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    double a = 0.0;
#pragma unroll
    for (int u = 0; u < NT / 32; ++u) a += red[u][threadIdx.x];
    gpart[(size_t)kMaxK * t + threadIdx.x] = a;
    __threadfence();
  }
  __syncthreads();
  const int t0 = tl.sys_tile0[sys], t1 = tl.sys_tile0[sys + 1];
  if (threadIdx.x == 0) last = atomicAdd(&counter[sys], 1u) == (unsigned)(t1 - t0 - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int q = threadIdx.x >> 3, l8 = threadIdx.x & 7;
  double a = 0.0;
  if (q < nk)
    for (int b = t0 + l8; b < t1; b += 8) a += __ldcg(&gpart[(size_t)kMaxK * b + q]);
  a += __shfl_xor_sync(0xffffffffu, a, 4);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  if (q < nk && l8 == 0) (pass == 1 ? gs[sys].h1 : gs[sys].h2)[q] = a;
  if (threadIdx.x == 0) counter[sys] = 0u;
}

// w -= sum_q h[q] V_q (q = 0..j, in order).  Pass 2 also forms ||w||, and
// the last tile of the system the new Hessenberg column h1 + h2, ||w||: it
// applies the previous rotations, makes the new one, updates g and tests
// convergence on |g_{j+1}|.
__global__ void __launch_bounds__(NT) k_gm_update(const double *__restrict__ V, size_t ldv, int j, double *w, Tiles tl,
                                                  double *partials, unsigned *counter, KrylovScalars *ks, GmState *gs,
                                                  int *n_done, int pass) {
  __shared__ double hs[kMaxK];
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const int nk = j + 1;
  const double *h = pass == 1 ? gs[sys].h1 : gs[sys].h2;
  if (threadIdx.x < nk) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const int i = tl.row0[t] + threadIdx.x;
  double ww = 0.0;
  if (i < tl.row1[t]) {
    double wi = w[i];
    for (int q = 0; q < nk; ++q) wi = fma(-hs[q], V[(size_t)q * ldv + i], wi);
    w[i] = wi;
    ww = wi * wi;
  }
  if (pass == 1) return;
  double v[1] = {ww}, out[1];
  if (seg_sum<NT, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    GmState &G = gs[sys];
    KrylovScalars &k = ks[sys];
    const double hn = sqrt(out[0]);
    double c[kRestart + 1];
    for (int q = 0; q <= j; ++q) c[q] = G.h1[q] + G.h2[q];
    c[j + 1] = hn;
    bool fin = false;
    if (!gm_rotate_column(j, c, G.cs, G.sn, G.g)) {
      k.breakdown = 1;
      G.k = j;
      fin = true;
    } else {
      for (int q = 0; q <= j; ++q) G.R[j][q] = c[q];
      G.hn = hn;
      G.k = j + 1;
      k.iter += 1;
      const double e2 = G.g[j + 1] * G.g[j + 1];
      fin = e2 <= k.tol2 || k.iter >= k.maxit || hn == 0.0;   // hn = 0: the space holds the solution
    }
    if (fin) {
      k.done = 1;
      atomicAdd(n_done, 1);
    }
  }
}

// V_{j+1} = w / ||w||
__global__ void __launch_bounds__(NT) k_gm_next(double *__restrict__ V, size_t ldv, int j, const double *__restrict__ w,
                                                Tiles tl, const KrylovScalars *ks, const GmState *gs) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double inv = 1.0 / gs[sys].hn;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) V[(size_t)(j + 1) * ldv + i] = w[i] * inv;
}

// z = D^-1 v (with ks: for systems not done)
__global__ void __launch_bounds__(NT) k_gm_jacobi(const double *__restrict__ v, const double *__restrict__ dinv,
                                                  double *__restrict__ z, Tiles tl, const KrylovScalars *ks) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks && ks[sys].done) return;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) z[i] = dinv[i] * v[i];
}

// End of a cycle, one thread per system: R y = g by back substitution over
// the k steps made (k = 0: nothing to add).
__global__ void k_gm_solve(int ns, GmState *gs) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= ns) return;
  GmState &G = gs[sys];
  gm_back_substitute(G.k, &G.R[0][0], kRestart, G.g, G.y);
}

// u = sum_{q < k} y_q V_q (zero for systems that made no step)
__global__ void __launch_bounds__(NT) k_gm_combine(const double *__restrict__ V, size_t ldv,
                                                   double *__restrict__ u, Tiles tl, const GmState *gs) {
  __shared__ double ys[kRestart];
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int k = gs[sys].k;
  if (threadIdx.x < k) ys[threadIdx.x] = gs[sys].y[threadIdx.x];
  __syncthreads();
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    double a = 0.0;
    for (int q = 0; q < k; ++q) a = fma(ys[q], V[(size_t)q * ldv + i], a);
    u[i] = a;
  }
}

// x += z for systems that made a step this cycle
__global__ void __launch_bounds__(NT) k_gm_xupdate(double *__restrict__ x, const double *__restrict__ z, Tiles tl,
                                                   const GmState *gs) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (gs[sys].k == 0) return;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) x[i] += z[i];
}

// Cycle start: r = b - A x into V_0 (unscaled) and ||r||.  The last tile of
// a system decides: final systems stay done; the tolerance met, the cap
// reached or a cycle without progress make the system final; otherwise it
// starts a cycle (g = ||r|| e_1).
__global__ void __launch_bounds__(NT) k_gm_restart(const double *__restrict__ b, const double *__restrict__ Ax,
                                                   double *__restrict__ V0, Tiles tl, double *partials,
                                                   unsigned *counter, KrylovScalars *ks, GmState *gs, int *n_done,
                                                   int first, double rtol, int maxit) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  double rr = 0.0, bb = 0.0;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) {
    const double ri = b[i] - Ax[i];
    V0[i] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  double v[2] = {rr, bb}, out[2];
  if (seg_sum<NT, 2>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    GmState &G = gs[sys];
    KrylovScalars &k = ks[sys];
    if (first) {
      k.bb = out[1];
      k.tol2 = rtol * rtol * out[1];
      k.iter = 0;
      k.maxit = maxit;
      k.breakdown = 0;
      k.stalled = 0;
      k.inner_total = 0;
      G.final = 0;
      G.beta_prev = INFINITY;
    }
    const double beta = sqrt(out[0]);
    k.rr = out[0];
    k.res2 = out[0];
    G.k = 0;
    if (!G.final) {
      if (out[0] <= k.tol2 || k.iter >= k.maxit || k.breakdown) {
        G.final = 1;
      } else if (!(beta < kStall * G.beta_prev)) {
        G.final = 1;
        k.stalled = 1;
      }
    }
    if (G.final) {
      k.done = 1;
      atomicAdd(n_done, 1);
    } else {
      k.done = 0;
      G.beta = beta;
      G.beta_prev = beta;
      G.g[0] = beta;
    }
  }
}

// V_0 = r / ||r|| for systems starting a cycle
__global__ void __launch_bounds__(NT) k_gm_scale0(double *__restrict__ V0, Tiles tl, const KrylovScalars *ks,
                                                  const GmState *gs) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  if (ks[sys].done) return;
  const double inv = 1.0 / gs[sys].beta;
  for (int i = tl.row0[t] + threadIdx.x; i < tl.row1[t]; i += NT) V0[i] *= inv;
}

}  // namespace

void gmres_solve(System *s, const vag_solve_opts *o, vag_solve_info *info) {
  cudaStream_t st = s->ctx->stream;
  ensure_krylov_buffers(s);
  tune_sell(s);
  const bool amg = o->precond == VAG_PC_AMG || o->precond == VAG_PC_AMG_RS;
  const bool cheb = o->precond == VAG_PC_CHEBYSHEV;
  const int ns = s->seg.n_sys;
  const int nt = s->seg.n_tiles;
  const Tiles tl = tiles_of(s);
  const size_t ldv = (size_t)std::max(s->n_rows, 1);
  if (!s->gm_V) {
    s->gm_V = sys_alloc<double>(s, ldv * (kRestart + 1));
    s->gm_w = sys_alloc<double>(s, ldv);
    s->gm_part = sys_alloc<double>(s, (size_t)kMaxK * std::max(nt, 1));
    s->gm_state = sys_alloc<unsigned char>(s, sizeof(GmState) * (size_t)ns);
  }
  if (!s->kz) s->kz = sys_alloc<double>(s, s->n_rows);
  double *V = s->gm_V, *w = s->gm_w, *z = s->kz;
  GmState *gs = reinterpret_cast<GmState *>(s->gm_state);
  float setup_ms = 0.f;
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  if (amg || cheb) {
    if (amg) amg_setup(s, o->precision != VAG_FP64, o->precision == VAG_MIXED_F16, o->precond == VAG_PC_AMG_RS);
    else cheb_setup(s);
    VAG_CUDA(cudaEventRecord(s->ev1, st));
    VAG_CUDA(cudaEventSynchronize(s->ev1));
    cudaEventElapsedTime(&setup_ms, s->ev0, s->ev1);
  }
  // z = M v; in_iter: systems already done are skipped where the
  // preconditioner allows it (the AMG V-cycle runs for every system)
  auto precond = [&](const double *in, double *out, bool in_iter) {
    if (amg) {
      amg_apply(s, in, out, st);
    } else if (cheb) {
      cheb_apply(s, in, out, st, in_iter, false, false);
    } else {
      k_gm_jacobi<<<nt, NT, 0, st>>>(in, s->dinv, out, tl, in_iter ? s->ks : nullptr);
      note_launches(1);
    }
  };
  auto restart = [&](int first) {
    VAG_CUDA(cudaMemsetAsync(s->n_done, 0, sizeof(int), st));
    launch_spmv_plain(s, s->kx, s->kq, st);
    k_gm_restart<<<nt, NT, 0, st>>>(s->rhs, s->kq, V, tl, s->partials, s->counter, s->ks, gs, s->n_done, first,
                                    o->rtol, o->maxit);
    k_gm_scale0<<<nt, NT, 0, st>>>(V, tl, s->ks, gs);
    note_launches(2);
    VAG_CHECK_LAUNCH();
  };
  auto step = [&](int j) {
    precond(V + (size_t)j * ldv, z, true);
    launch_spmv_plain(s, z, w, st);
    for (int pass = 1; pass <= 2; ++pass) {
      k_gm_dots<<<nt, NT, 0, st>>>(V, ldv, j, w, tl, s->gm_part, s->counter, s->ks, gs, pass);
      k_gm_update<<<nt, NT, 0, st>>>(V, ldv, j, w, tl, s->partials, s->counter, s->ks, gs, s->n_done, pass);
    }
    k_gm_next<<<nt, NT, 0, st>>>(V, ldv, j, w, tl, s->ks, gs);
    note_launches(5);
  };
  // the Arnoldi steps of a cycle, kChunk to a graph (rebuilt every solve:
  // the preconditioner's buffers are new each time)
  const int nchunks = (kRestart + kChunk - 1) / kChunk;
  std::vector<cudaGraphExec_t> chunks(nchunks, nullptr);
  std::vector<size_t> chunk_nodes(nchunks, 0);
  for (int c = 0; c < nchunks; ++c) {
    cudaGraph_t graph;
    VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    for (int j = c * kChunk; j < std::min(kRestart, (c + 1) * kChunk); ++j) step(j);
    set_capturing(false);
    VAG_CUDA(cudaStreamEndCapture(st, &graph));
    cudaGraphGetNodes(graph, nullptr, &chunk_nodes[c]);
    VAG_CUDA(cudaGraphInstantiate(&chunks[c], graph, 0));
    cudaGraphDestroy(graph);
  }
  VAG_CUDA(cudaMemsetAsync(s->kx, 0, sizeof(double) * s->n_rows, st));
  restart(1);
  const int max_cycles = o->maxit + 2;   // an active system makes at least one step per cycle
  for (int cyc = 0; cyc < max_cycles; ++cyc) {
    VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (*s->n_done_host >= ns) break;
    for (int c = 0; c < nchunks; ++c) {
      VAG_CUDA(cudaGraphLaunch(chunks[c], st));
      note_launches(chunk_nodes[c]);
      VAG_CUDA(cudaMemcpyAsync(s->n_done_host, s->n_done, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*s->n_done_host >= ns) break;
    }
    // x += M V_k y for every system that made steps in this cycle
    k_gm_solve<<<(ns + 127) / 128, 128, 0, st>>>(ns, gs);
    k_gm_combine<<<nt, NT, 0, st>>>(V, ldv, w, tl, gs);
    note_launches(2);
    precond(w, z, false);
    k_gm_xupdate<<<nt, NT, 0, st>>>(s->kx, z, tl, gs);
    note_launches(1);
    restart(0);
  }
  for (auto &g : chunks)
    if (g) cudaGraphExecDestroy(g);
  // the true residual decides the status
  true_residual2(s, st);
  finish_solve(s, info, false);
  info->ms_setup = setup_ms;
  info->ms_solve -= setup_ms;
}

}  // namespace vag
