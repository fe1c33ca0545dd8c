// Cell recovery, Darcy fluxes and the explicit upwind transport of Sec. 3.2.
//
//  k_recover     Eq. (eqschurcell): u_K = -(sum_nu M_K,nu u_nu) / M_KK.
//  k_cell_flux   Eq. (VAGFluxMatrix): F_{K,nu} = sum_nu' a_{K,nu}^{nu'} (u_K - u_nu').
//  k_ff_flux     Eq. (VAGFluxFracture): F_{sigma,s} = sum_s' a_{sigma,s}^{s'} (u_sigma - u_s').
//  k_porous      porous volumes phi_K, phi_sigma, phi_s of Sec. 3.2.1.
//  k_map_count / k_map_fill
//                one explicit Euler step with the upwind fluxes of
//                Eq. (darcyfluxH) is the linear map
//                  c^{n+1}_mu = d_mu c^n_mu + sum_{nu upstream of mu} w_{mu,nu} c^n_nu,
//                  d_mu = 1 - dt/phi_mu * (outflow of mu),  w >= 0,
//                because every edge with F != 0 has one upstream end: its
//                flux enters the downstream control volume with the upstream
//                concentration and leaves the upstream one with it.  The map
//                is built once per (fluxes, dt) from the inflow edges;
//                Dirichlet rows keep c = cbar (d = 1, no inflow).
//  k_sigma_sort  the map's row order: inside each window of kSigma control
//                volumes, rows by decreasing inflow count (stable), so that
//                the 32 rows of a warp have nearly the same number of edges;
//                the map is stored as sliced ELL over that order.
//  k_map_count / k_pick_dt
//                Eq. (eq_CFL): per system the min over non-Dirichlet CVs of
//                phi / outflow (taken while counting the inflow edges), and
//                the step cfl x that bound.
//  k_step        c' = d c + W c (one thread per row slot, one warp per slice).
//
// Wells (Sec. 5.5): perforation p exchanges the rate Fw[p] =
// WI (u_sigma - p_w) - q between its fracture face and the well.  The well
// side is one extra state entry n_cv + p held at the injected concentration
// (a fixed row like a Dirichlet node), so a production rate is outflow of
// the face and an injection rate an inflow edge from that entry; k_step is
// unchanged.  The extra entries live only in the library's buffers.
#include "vag_internal.cuh"
#include "vag_reduce.cuh"
#include "vag_topo.h"

namespace vag {
namespace {

constexpr int TB = 256;

__device__ __forceinline__ double mcK(const double *Mc, int nc, int i, int j, int K) {
  return Mc[(size_t)topo::pidx(i, j) * nc + K];
}
__device__ __forceinline__ double mfcK(const double *Mfc, int n_fc, int lf, int k, int fi) {
  return Mfc[(size_t)(lf * 6 + k) * n_fc + fi];
}

__global__ void k_recover(int nc, int nv, const int *__restrict__ cn, const int *__restrict__ cell_ff,
                          const int *__restrict__ fc_index, int n_fc, const double *__restrict__ Mc,
                          const double *__restrict__ Mfc, double *__restrict__ u, int nf) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int nb = cn[8 * (size_t)K + b];
    if (nb >= 0) s = fma(mcK(Mc, nc, 0, 1 + b, K), u[nb], s);
  }
  const int fi = fc_index[K];
  if (fi >= 0) {
    for (int lf = 0; lf < 6; ++lf) {
      const int f = cell_ff[6 * (size_t)K + lf];
      if (f >= 0) s = fma(mfcK(Mfc, n_fc, lf, 1, fi), u[nv + f], s);
    }
  }
  u[(size_t)nv + nf + K] = -s / mcK(Mc, nc, 0, 0, K);
}

// GEN: cells of any shape (shape[K]); otherwise hexahedra only.
template <bool GEN>
__global__ void k_cell_flux(int nc, int nv, int nf, const int8_t *__restrict__ shape, const int *__restrict__ cn,
                            const int *__restrict__ cell_ff, const int *__restrict__ fc_index, int n_fc,
                            const double *__restrict__ Mc, const double *__restrict__ Mfc,
                            const double *__restrict__ u, double *__restrict__ Fcn, double *__restrict__ Fcf) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  const int sh = GEN ? shape[K] : topo::HEX;
  const double uK = u[(size_t)nv + nf + K];
  double du[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int nb = cn[8 * (size_t)K + b];
    du[b] = (!GEN || nb >= 0) ? uK - u[nb] : 0.0;
  }
  const int fi = fc_index[K];
  double dus[6];
  int ffid[6];
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    ffid[lf] = fi >= 0 ? cell_ff[6 * (size_t)K + lf] : -1;
    dus[lf] = ffid[lf] >= 0 ? uK - u[nv + ffid[lf]] : 0.0;
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double F = 0.0;
#pragma unroll
    for (int b = 0; b < 8; ++b) F = fma(mcK(Mc, nc, 1 + a, 1 + b, K), du[b], F);
    if (fi >= 0) {
#pragma unroll
      for (int lf = 0; lf < 6; ++lf) {
        const int t = topo::pos_on_face(sh, lf, a);
        if (t >= 0 && ffid[lf] >= 0) F = fma(mfcK(Mfc, n_fc, lf, 2 + t, fi), dus[lf], F);
      }
    }
    Fcn[8 * (size_t)K + a] = F;
  }
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    double F = 0.0;
    if (ffid[lf] >= 0) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int b = topo::face(sh, lf, t);
        if (b >= 0) F = fma(mfcK(Mfc, n_fc, lf, 2 + t, fi), du[b], F);
      }
      F = fma(mfcK(Mfc, n_fc, lf, 0, fi), dus[lf], F);
    }
    Fcf[6 * (size_t)K + lf] = F;
  }
}

__global__ void k_ff_flux(int nf, int nv, const int *__restrict__ ffn, const double *__restrict__ Mff,
                          const double *__restrict__ u, double *__restrict__ Fff) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const double us = u[nv + f];
  double du[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int nb = ffn[4 * (size_t)f + t];   // -1: a triangle's unused slot
    du[t] = nb >= 0 ? us - u[nb] : 0.0;
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    double F = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) F = fma(Mff[(size_t)((1 + t) * 5 + 1 + v) * nf + f], du[v], F);
    Fff[4 * (size_t)f + t] = F;
  }
}

// Fw[p] = WI (u_sigma - p_w) - q: the rate leaving the perforated face into
// the well.
__global__ void k_well_flux(int n_perf, int nv, const int *__restrict__ ff, const double *__restrict__ wi,
                            const double *__restrict__ pw, const double *__restrict__ q,
                            const double *__restrict__ u, double *__restrict__ Fw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_perf) return;
  Fw[p] = fma(wi[p], u[nv + ff[p]] - pw[p], -q[p]);
}

struct TView {
  int nv, nf, nc;
  const int8_t *shape;   // nullptr: every cell is a hexahedron
  const int *cn, *ffn, *cell_ff, *ff_cells, *ff_lface, *node_dir, *node_isfrac;
  const int *ff_perf;    // [nf] perforation of each fracture face or -1 (nullptr: no wells)
  const double *Fw;      // [n_perf]
  const int *n2c_ptr, *n2c, *n2f_ptr, *n2f;
  const double *cvol, *ffarea, *df, *phi_m, *phi_f;
  const double *Fcn, *Fcf, *Fff;
  double omega;
};

__global__ void k_porous(TView t, double *__restrict__ phi, int *status) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = t.nv + t.nf + t.nc;
  if (mu >= n) return;
  double p = 0.0;
  if (mu < t.nv) {
    const int s = mu;
    if (t.node_dir[s] >= 0) { phi[mu] = 0.0; return; }
    // alpha = omega / |V_sigma| (fracture nodes) or omega / |V_K| (others)
    if (t.node_isfrac[s]) {
      for (int e = t.n2f_ptr[s]; e < t.n2f_ptr[s + 1]; ++e) {
        const int f = t.n2f[e] >> 2;
        const int q = t.ffn[4 * (size_t)f + 3] < 0 ? 3 : 4;
        p += (t.omega / q) * t.df[f] * t.ffarea[f] * t.phi_f[f];
      }
    } else {
      for (int e = t.n2c_ptr[s]; e < t.n2c_ptr[s + 1]; ++e) {
        const int K = t.n2c[e] >> 3;
        const int nK = topo::n_nodes(t.shape ? t.shape[K] : topo::HEX);
        p += (t.omega / nK) * t.cvol[K] * t.phi_m[K];
      }
    }
  } else if (mu < t.nv + t.nf) {
    const int f = mu - t.nv;
    int cnt = 0, q = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int s = t.ffn[4 * (size_t)f + k];
      if (s < 0) continue;
      ++q;
      cnt += t.node_dir[s] < 0;
    }
    p = (1.0 - (t.omega / q) * cnt) * t.df[f] * t.ffarea[f] * t.phi_f[f];
  } else {
    const int K = mu - t.nv - t.nf;
    const int nK = topo::n_nodes(t.shape ? t.shape[K] : topo::HEX);
    int cnt = 0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int s = t.cn[8 * (size_t)K + l];
      if (s < 0) continue;
      cnt += (t.node_dir[s] < 0) && !t.node_isfrac[s];
    }
    p = (1.0 - (t.omega / nK) * cnt) * t.cvol[K] * t.phi_m[K];
  }
  if (!(p > 0.0)) atomicOr(status, ST_NONPOSITIVE);
  phi[mu] = p;
}

// Visit the edges of control volume mu: fn(F_in_view, neighbour) where
// F_in_view > 0 means the flux enters mu from the neighbour (the neighbour is
// upstream) and F_in_view < 0 means it leaves mu.
template <class Fn>
__device__ __forceinline__ void for_edges(const TView &t, int mu, Fn &&fn) {
  if (mu < t.nv) {
    const int s = mu;
    for (int e = t.n2c_ptr[s]; e < t.n2c_ptr[s + 1]; ++e) {   // F_{K,s} > 0: K -> s
      const int K = t.n2c[e] >> 3, a = t.n2c[e] & 7;
      fn(t.Fcn[8 * (size_t)K + a], t.nv + t.nf + K);
    }
    for (int e = t.n2f_ptr[s]; e < t.n2f_ptr[s + 1]; ++e) {   // F_{sigma,s} > 0: sigma -> s
      const int f = t.n2f[e] >> 2, q = t.n2f[e] & 3;
      fn(t.Fff[4 * (size_t)f + q], t.nv + f);
    }
  } else if (mu < t.nv + t.nf) {
    const int f = mu - t.nv;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s = t.ffn[4 * (size_t)f + q];
      if (s >= 0) fn(-t.Fff[4 * (size_t)f + q], s);
    }
    for (int c = 0; c < 2; ++c) {                                // F_{K,sigma} > 0: K -> sigma
      const int K = t.ff_cells[2 * f + c];
      if (K < 0) continue;
      fn(t.Fcf[6 * (size_t)K + t.ff_lface[2 * f + c]], t.nv + t.nf + K);
    }
    if (t.ff_perf) {                                             // Fw > 0: sigma -> well
      const int p = t.ff_perf[f];
      if (p >= 0) fn(-t.Fw[p], t.nv + t.nf + t.nc + p);
    }
  } else {
    const int K = mu - t.nv - t.nf;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int s = t.cn[8 * (size_t)K + a];
      if (s >= 0) fn(-t.Fcn[8 * (size_t)K + a], s);
    }
#pragma unroll
    for (int lf = 0; lf < 6; ++lf) {
      const int f = t.cell_ff[6 * (size_t)K + lf];
      if (f >= 0) fn(-t.Fcf[6 * (size_t)K + lf], t.nv + f);
    }
  }
}

// rows held fixed: Dirichlet nodes and the wells' entries past the n_cv
// control volumes
__device__ __forceinline__ bool is_dir(const TView &t, int mu) {
  return (mu < t.nv && t.node_dir[mu] >= 0) || mu >= t.nv + t.nf + t.nc;
}

// Per CV: number of inflow edges and the CFL ratio phi / outflow; the ratio
// is min-reduced per system with atomicMin on the bit pattern of a positive
// double (order-independent, hence deterministic).  A warp whose control
// volumes all belong to one system reduces first and makes one atomic.
__global__ void __launch_bounds__(TB) k_map_count(TView t, int n, const double *__restrict__ phi,
                                                  const int *__restrict__ cv_sys, int *__restrict__ cnt,
                                                  unsigned long long *dt_bits) {
  const int mu = blockIdx.x * TB + threadIdx.x;
  unsigned long long bits = ~0ull;   // no bound
  int sys = -1;
  if (mu < n) {
    if (is_dir(t, mu)) {
      cnt[mu] = 0;
    } else {
      int c = 0;
      double out = 0.0;
      for_edges(t, mu, [&](double Fin, int) {
        if (Fin > 0.0) ++c;
        else out -= Fin;
      });
      cnt[mu] = c;
      sys = cv_sys[mu];
      if (out > 0.0) bits = (unsigned long long)__double_as_longlong(phi[mu] / out);
    }
  }
  const int s0 = __shfl_sync(0xffffffffu, sys, 0);
  if (__all_sync(0xffffffffu, sys == s0 || sys < 0) && s0 >= 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits = min(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    if ((threadIdx.x & 31) == 0 && bits != ~0ull) atomicMin(&dt_bits[s0], bits);
  } else if (sys >= 0 && bits != ~0ull) {
    atomicMin(&dt_bits[sys], bits);
  }
}

// Per system: dts[2g] = CFL bound (bits -> double), dts[2g+1] = the step
// (cfl * bound, or the given dt; 0 when no control volume has outflow).
__global__ void k_pick_dt(int n_sys, const unsigned long long *__restrict__ dt_bits, double *dts, double cfl,
                          double dt) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_sys) return;
  double m = __longlong_as_double((long long)dt_bits[g]);
  if (m > 1e300) m = INFINITY;   // no control volume of this system has outflow
  dts[2 * g] = m;
  double h = cfl > 0 ? cfl * m : dt;
  if (!(h < INFINITY)) h = 0.0;
  dts[2 * g + 1] = h;
}

// Row mu in slot inv[mu]: inflow entry j at tsp[s] + 32 j + r (slice s, lane
// r), its column the upstream volume's slot (the steps run on the state in
// slot order); the slice's remaining entries of the row are padding (the
// row's own slot, weight 0), which leaves every product chain unchanged.
__global__ void k_map_fill(TView t, int n, const double *__restrict__ phi, const int *__restrict__ cv_sys,
                           const int *__restrict__ inv, const int *__restrict__ sp, const double *__restrict__ dts,
                           double *__restrict__ diag, int *__restrict__ col, double *__restrict__ w) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= n) return;
  const int slot = inv[mu];
  const int k0 = sp[slot >> 5] + (slot & 31), width = (sp[(slot >> 5) + 1] - sp[slot >> 5]) >> 5;
  int j = 0;
  if (is_dir(t, mu)) {
    diag[slot] = 1.0;
  } else {
    const double h = dts[2 * cv_sys[mu] + 1] / phi[mu];
    double out = 0.0;
    for_edges(t, mu, [&](double Fin, int nb) {
      if (Fin > 0.0) {
        col[k0 + 32 * j] = inv[nb];
        w[k0 + 32 * j] = h * Fin;
        ++j;
      } else {
        out -= Fin;
      }
    });
    diag[slot] = 1.0 - h * out;
  }
  for (; j < width; ++j) {
    col[k0 + 32 * j] = slot;
    w[k0 + 32 * j] = 0.0;
  }
}

// One block per window of kSigma rows: perm (slot -> row) and inv (row ->
// slot) with the rows of the window ordered by decreasing inflow count
// (counts of 31 and more share the first bucket), equal counts by row index;
// slice_len[s] = 32 x the widest row of slice s.  Deterministic: ranks come
// from warp matches and prefix sums, not from atomics.
constexpr int kSigma = 1024;
__global__ void __launch_bounds__(kSigma) k_sigma_sort(int n, const int *__restrict__ cnt, int *__restrict__ perm,
                                                       int *__restrict__ inv, int *__restrict__ slice_len) {
  constexpr int NW = kSigma / 32;
  __shared__ int wc[NW][32];   // rows per (warp, bucket), then the warp's offset in the bucket
  __shared__ int start[32];    // first position of each bucket in the window
  __shared__ int srow[kSigma];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w0 = blockIdx.x * kSigma, i = w0 + threadIdx.x;
  const bool valid = i < n;
  const int c = valid ? cnt[i] : 0;
  const int b = valid ? 31 - min(c, 31) : 32;   // bucket 0 = the longest rows
  wc[warp][lane] = 0;
  __syncthreads();
  const unsigned same = __match_any_sync(0xffffffffu, b);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (valid && rank == 0) wc[warp][b] = __popc(same);
  __syncthreads();
  if (warp == 0) {
    int run = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      const int x = wc[q][lane];
      wc[q][lane] = run;
      run += x;
    }
    int incl = run;   // bucket totals -> exclusive scan over buckets
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    start[lane] = incl - run;
  }
  __syncthreads();
  if (valid) {
    const int pos = start[b] + wc[warp][b] + rank;
    perm[w0 + pos] = i;
    inv[i] = w0 + pos;
    srow[pos] = c;
  }
  __syncthreads();
  const int slot = w0 + threadIdx.x;
  int m = slot < n ? srow[threadIdx.x] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && slot < n) slice_len[slot >> 5] = 32 * m;
}

// system of every control volume of the union ([nodes | ffaces | cells])
__global__ void k_cv_sys(int nv, int nf, int nc, int n_sys, const int *__restrict__ node_start,
                         const int *__restrict__ ff_start, const int *__restrict__ cell_start, int *cv_sys) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= nv + nf + nc) return;
  const int *st;
  int i;
  if (mu < nv) { st = node_start; i = mu; }
  else if (mu < nv + nf) { st = ff_start; i = mu - nv; }
  else { st = cell_start; i = mu - nv - nf; }
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (st[mid] <= i) lo = mid; else hi = mid - 1;
  }
  cv_sys[mu] = lo;
}

// One thread per row slot, one warp per slice, on the state in slot order
// (c[i] is the concentration of volume tperm[i]): the slice's entries and
// the rows' own values are read lane-contiguous (coalesced), and every lane
// walks the slice's width, so a warp's fma instructions are as many as its
// widest row (rows of a slice have nearly equal counts, see k_sigma_sort).
// Launched with programmatic dependent launch: the map (written once per
// solve) is read before the dependency wait, the previous step's c after it.
// The map streams through once a step (evict-first loads), so the cache keeps
// the concentrations that the gathers reuse.
constexpr int kStepPF = 4;
constexpr int kStepTB = 128;   // 128 / 256 / 512 threads: 54.8 / 55.3 / 58.7 us at 128^3
__global__ void __launch_bounds__(kStepTB) k_step(int n, const int *__restrict__ sp, const int *__restrict__ col,
                                                  const double *__restrict__ w, const double *__restrict__ diag,
                                                  const double *__restrict__ c, double *__restrict__ cn) {
  const int i = blockIdx.x * kStepTB + threadIdx.x;
  if ((i >> 5) >= (n + 31) >> 5) return;   // whole warps
  const int r = i & 31;
  const int k0 = __ldcs(sp + (i >> 5)), width = (__ldcs(sp + (i >> 5) + 1) - k0) >> 5;
  const bool valid = i < n;
  const double d = valid ? __ldcs(diag + i) : 0.0;
  int pc[kStepPF];
  double pw[kStepPF];
#pragma unroll
  for (int u = 0; u < kStepPF; ++u) {
    pc[u] = valid && u < width ? __ldcs(col + k0 + 32 * u + r) : 0;
    pw[u] = valid && u < width ? __ldcs(w + k0 + 32 * u + r) : 0.0;
  }
  pdl_wait();
  pdl_trigger();
  if (!valid) return;
  double v = d * c[i];
#pragma unroll
  for (int u = 0; u < kStepPF; ++u)
    if (u < width) v = fma(pw[u], c[pc[u]], v);
  for (int u = kStepPF; u < width; ++u) v = fma(__ldcs(w + k0 + 32 * u + r), c[__ldcs(col + k0 + 32 * u + r)], v);
  cn[i] = v;
}

// state in control-volume order <-> slot order
__global__ void k_to_slots(int n, const int *__restrict__ perm, const double *__restrict__ c_cv,
                           double *__restrict__ c_slot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c_slot[i] = c_cv[perm[i]];
}
__global__ void k_from_slots(int n, const int *__restrict__ perm, const double *__restrict__ c_slot,
                             double *__restrict__ c_cv, int n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int mu = perm[i];
  if (mu < n_out) c_cv[mu] = c_slot[i];
}

__global__ void k_set_dir(int nd, const int *__restrict__ dn, const double *__restrict__ cbar, double *__restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nd) c[dn[i]] = cbar[i];
}

}  // namespace

// Mean duration of one explicit step on the current upwind map.
double time_transport_step(System *s, int reps) {
  if (!s->tsp || !s->cbuf || !s->tdiag) fail(VAG_EINVAL, "no upwind map: run vag_transport first");
  cudaStream_t st = s->ctx->stream;
  const int n = s->n_cv + s->n_perf;
  const int gs = grid_for(32 * ((n + 31) / 32), kStepTB);
  double *a = s->cbuf, *b = s->cbuf + n;
  auto step = [&](const double *c, double *cn) {
    launch_pdl(k_step, gs, kStepTB, 0, st, n, (const int *)s->tsp, (const int *)s->tcol, (const double *)s->tval,
               (const double *)s->tdiag, c, cn);
    note_launches(1);
  };
  step(a, b);   // warm-up
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  for (int r = 0; r < reps; ++r) {
    if (r & 1) step(b, a);
    else step(a, b);
  }
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  return (double)ms / reps;
}

void recover_cells_and_fluxes(System *s) {
  cudaStream_t st = s->ctx->stream;
  if (!s->Fcn) {
    s->Fcn = sys_alloc<double>(s, 8 * (size_t)s->nc);
    s->Fcf = sys_alloc<double>(s, 6 * (size_t)s->nc);
    s->Fff = sys_alloc<double>(s, 4 * (size_t)(s->nf > 0 ? s->nf : 1));
  }
  k_recover<<<grid_for(s->nc, TB), TB, 0, st>>>(s->nc, s->nv, s->cell_nodes, s->cell_ff, s->fc_index, s->n_fc,
                                                s->Mc, s->Mfc, s->u, s->nf); note_launches(1);
  if (s->cell_shape)
    k_cell_flux<true><<<grid_for(s->nc, 128), 128, 0, st>>>(s->nc, s->nv, s->nf, s->cell_shape, s->cell_nodes,
                                                            s->cell_ff, s->fc_index, s->n_fc, s->Mc, s->Mfc, s->u,
                                                            s->Fcn, s->Fcf);
  else
    k_cell_flux<false><<<grid_for(s->nc, 128), 128, 0, st>>>(s->nc, s->nv, s->nf, nullptr, s->cell_nodes,
                                                             s->cell_ff, s->fc_index, s->n_fc, s->Mc, s->Mfc, s->u,
                                                             s->Fcn, s->Fcf);
  note_launches(1);
  if (s->nf) {
    k_ff_flux<<<grid_for(s->nf, TB), TB, 0, st>>>(s->nf, s->nv, s->ff_nodes, s->Mff, s->u, s->Fff);
    note_launches(1);
  }
  if (s->n_perf) {
    k_well_flux<<<grid_for(s->n_perf, TB), TB, 0, st>>>(s->n_perf, s->nv, s->well_ff, s->well_wi, s->well_pw,
                                                         s->well_q, s->u, s->Fw);
    note_launches(1);
  }
  VAG_CHECK_LAUNCH();
  s->have_flux = true;
}

namespace {
// Stream-ordered scratch allocations, released on every exit path.
struct StreamScratch {
  cudaStream_t st;
  std::vector<void *> p;
  template <class T>
  T *get(size_t count) {
    void *q = nullptr;
    VAG_CUDA(cudaMallocAsync(&q, sizeof(T) * std::max<size_t>(count, 1), st));
    p.push_back(q);
    return static_cast<T *>(q);
  }
  ~StreamScratch() {
    for (void *q : p) cudaFreeAsync(q, st);
  }
};
}  // namespace

// phi_m [nc], phi_f [nf], cbar [nd] already on the device.
void transport_run(System *s, const vag_transport_opts *o, double *c_dev, vag_transport_info *info,
                   const double *phi_m, const double *phi_f, const double *cbar) {
  cudaStream_t st = s->ctx->stream;
  const int n = s->n_cv;
  const int nt = n + s->n_perf;   // rows of the step: control volumes, then the wells' entries
  const int ns = s->seg.n_sys;
  if (!s->phi) {
    s->phi = sys_alloc<double>(s, n);
    s->dts = sys_alloc<double>(s, 2 * (size_t)ns);
    s->seg.cv_sys = sys_alloc<int>(s, n);
    k_cv_sys<<<grid_for(n, TB), TB, 0, st>>>(s->nv, s->nf, s->nc, ns, s->seg.d_node_start, s->seg.d_ff_start,
                                             s->seg.d_cell_start, s->seg.cv_sys);
    note_launches(1);
  }
  const int n_slices = (nt + 31) / 32;
  if (nt > s->t_rows) {
    s->tdiag = sys_alloc<double>(s, nt);
    s->tperm = sys_alloc<int>(s, nt);
    s->tsp = sys_alloc<int>(s, (size_t)n_slices + 1);
    s->cbuf = sys_alloc<double>(s, 2 * (size_t)nt);
    s->t_rows = nt;
  }
  TView t{s->nv, s->nf, s->nc, s->cell_shape, s->cell_nodes, s->ff_nodes, s->cell_ff, s->ff_cells, s->ff_lface,
          s->node_dir, s->node_isfrac, s->n_perf ? s->ff_perf : nullptr, s->Fw, s->n2c_ptr, s->n2c, s->n2f_ptr,
          s->n2f, s->cvol, s->ffarea, s->df, phi_m, phi_f, s->Fcn, s->Fcf, s->Fff, o->omega};
  VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  k_porous<<<grid_for(n, TB), TB, 0, st>>>(t, s->phi, s->status);
  note_launches(1);
  StreamScratch scratch{st, {}};
  int *cnt = scratch.get<int>((size_t)nt + 1);
  int *inv = scratch.get<int>((size_t)nt + 1);
  int *slice_len = scratch.get<int>((size_t)n_slices + 1);
  unsigned long long *dt_bits = scratch.get<unsigned long long>(ns);
  VAG_CUDA(cudaMemsetAsync(dt_bits, 0x7f, sizeof(unsigned long long) * ns, st));   // > every finite ratio
  k_map_count<<<grid_for(nt, TB), TB, 0, st>>>(t, nt, s->phi, s->seg.cv_sys, cnt, dt_bits);
  note_launches(1);
  k_pick_dt<<<grid_for(ns, TB), TB, 0, st>>>(ns, dt_bits, s->dts, o->cfl, o->dt);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  const int64_t nnz_t = scan_exclusive(cnt, inv, nt, st);   // inflow entries (inv as scratch)
  if (read_status(s) & ST_NONPOSITIVE) fail(VAG_EINVAL, "a control volume has a non-positive porous volume");
  k_sigma_sort<<<(nt + kSigma - 1) / kSigma, kSigma, 0, st>>>(nt, cnt, s->tperm, inv, slice_len);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  const int64_t n_stored = scan_exclusive(slice_len, s->tsp, n_slices, st);
  if (n_stored < nnz_t) fail(VAG_EINVAL, "the transport map exceeds 2^31 stored entries");
  if (n_stored > s->t_cap) {
    // grow the entry arrays (kept across calls)
    s->tcol = sys_alloc<int>(s, (size_t)std::max<int64_t>(n_stored, 1));
    s->tval = sys_alloc<double>(s, (size_t)std::max<int64_t>(n_stored, 1));
    s->t_cap = n_stored;
  }
  s->nnz_t = nnz_t;
  k_map_fill<<<grid_for(nt, TB), TB, 0, st>>>(t, nt, s->phi, s->seg.cv_sys, inv, s->tsp, s->dts, s->tdiag, s->tcol,
                                              s->tval);
  note_launches(1);
  // c^0 with the Dirichlet values and the injected concentrations
  // (assembled in control-volume order in the second half of cbuf, then
  // gathered into slot order in the first)
  double *c0 = s->cbuf, *c1 = s->cbuf + nt;
  VAG_CUDA(cudaMemcpyAsync(c1, c_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (s->n_perf)
    VAG_CUDA(cudaMemcpyAsync(c1 + n, s->well_cin, sizeof(double) * s->n_perf, cudaMemcpyDeviceToDevice, st));
  k_set_dir<<<grid_for(s->nd, TB), TB, 0, st>>>(s->nd, s->dir_nodes, cbar, c1);
  k_to_slots<<<grid_for(nt, TB), TB, 0, st>>>(nt, s->tperm, c1, c0);
  note_launches(2);
  VAG_CHECK_LAUNCH();
  trace_mark(st, "porous volumes + CFL + upwind map");
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  const int gs = grid_for(32 * n_slices, kStepTB);
  // steps in CUDA graphs of kStepChunk launches (an even count: the chunk
  // starts and ends in the same buffer), the remainder launched directly
  constexpr int kStepChunk = 20;
  const int chunks = o->n_steps / kStepChunk;
  if (chunks > 0) {
    if (!s->step_graph || s->step_graph_cap != s->t_cap || s->step_graph_rows != nt) {
      if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
      s->step_graph = nullptr;
      cudaGraph_t graph;
      VAG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      set_capturing(true);
      double *a = s->cbuf, *b = s->cbuf + nt;
      for (int k = 0; k < kStepChunk; ++k) {
        launch_pdl(k_step, gs, kStepTB, 0, st, nt, (const int *)s->tsp, (const int *)s->tcol, (const double *)s->tval,
                   (const double *)s->tdiag, (const double *)a, b);
        std::swap(a, b);
      }
      set_capturing(false);
      VAG_CUDA(cudaStreamEndCapture(st, &graph));
      VAG_CUDA(cudaGraphInstantiate(&s->step_graph, graph, 0));
      cudaGraphDestroy(graph);
      s->step_graph_cap = s->t_cap;
      s->step_graph_rows = nt;
    }
    for (int c = 0; c < chunks; ++c) {
      VAG_CUDA(cudaGraphLaunch(s->step_graph, st));
      note_launches(kStepChunk);
    }
  }
  for (int k = chunks * kStepChunk; k < o->n_steps; ++k) {
    launch_pdl(k_step, gs, kStepTB, 0, st, nt, (const int *)s->tsp, (const int *)s->tcol, (const double *)s->tval,
               (const double *)s->tdiag, (const double *)c0, c1);
    note_launches(1);
    std::swap(c0, c1);
  }
  VAG_CHECK_LAUNCH();
  trace_mark(st, "explicit steps");
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  k_from_slots<<<grid_for(nt, TB), TB, 0, st>>>(nt, s->tperm, c0, c_dev, n);
  note_launches(1);
  s->dts_host.resize(2 * (size_t)ns);
  VAG_CUDA(cudaMemcpyAsync(s->dts_host.data(), s->dts, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, s->ev0, s->ev1);
  // a batch reports its smallest bound and step; vag_transport_get_dts gives each
  double dmax = s->dts_host[0], dt = s->dts_host[1];
  for (int g = 1; g < ns; ++g) {
    dmax = std::min(dmax, s->dts_host[2 * g]);
    dt = std::min(dt, s->dts_host[2 * g + 1]);
  }
  info->dt_max = dmax;
  info->dt = dt;
  info->steps = o->n_steps;
  info->ms = ms;
}

}  // namespace vag
