// Numeric phase of vag_assemble (FP64):
//  k_cell_local  one thread per cell: the local VAG matrix
//                a_{K,nu}^{nu'} = int_K Lambda_m/mu grad eta_nu . grad eta_nu'
//                of Eq. (VAGFluxMatrix), integrated exactly on the
//                tetrahedra T_{K,sigma,e} = conv(x_K, x_sigma, e) (Sec. 3.1):
//                24 for a hexahedron, 18 for a prism, 16 for a pyramid, 12
//                for a tetrahedron (vag_topo.h).  The face-centre vertex of
//                a non-fracture face is the interpolation I_sigma (beta =
//                1/|V_sigma| on the face nodes); on a fracture face it is the
//                unknown v_sigma.
//  k_ff_local    one thread per fracture face: a_{sigma,s}^{s'} of
//                Eq. (VAGFluxFracture) on the triangles (x_sigma, e).
//  k_gather_rows one thread per Krylov row: the Schur complement of
//                Eq. (eqschur), A = A_[vf][vf] - A_[vf]c A_cc^{-1} A_c[vf],
//                summed over the row's cells and fracture faces in a fixed
//                order (deterministic, no atomics); Dirichlet columns go to
//                the right-hand side.
//  k_wells       one thread per well perforation: the Peaceman term of
//                Sec. 5.5, q_sigma = WI_sigma (p_sigma - p_w) - q_sigma^inj,
//                on the fracture-face row (diagonal and right-hand side).
#include "vag_internal.cuh"
#include "vag_topo.h"

namespace vag {
namespace {

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 ldv(const double *__restrict__ xyz, int n) {
  return {xyz[3 * (size_t)n], xyz[3 * (size_t)n + 1], xyz[3 * (size_t)n + 2]};
}

// packed index in a 6x6 symmetric matrix over (K, sigma, t0, t1, t2, t3)
__host__ __device__ constexpr int p6(int i, int j) {
  return i <= j ? i * 6 - (i * (i - 1)) / 2 + (j - i) : j * 6 - (j * (j - 1)) / 2 + (i - j);
}
// L v for the symmetric tensor L = (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ V3 lmul(const double (&L)[6], V3 v) {
  return {L[0] * v.x + L[3] * v.y + L[4] * v.z, L[3] * v.x + L[1] * v.y + L[5] * v.z,
          L[4] * v.x + L[5] * v.y + L[2] * v.z};
}
__device__ __forceinline__ V3 neg(V3 a) { return {-a.x, -a.y, -a.z}; }

// The local matrix of one cell of shape SH: M over (K, node slots 0..7)
// packed, Mfc over (sigma sigma, sigma K, sigma n_t) for each fracture face.
//
// Each face's tetrahedra T_{K,sigma,e} = (x_K, x_sigma, q_e, q_e+1) add their
// P1 stiffness to F (packed 6x6 over (K, sigma, q0..q3)).  For a tetrahedron
// (p0..p3) with e_k = p_k - p0, the area vectors n1 = e2 x e3, n2 = e3 x e1,
// n3 = e1 x e2 and n0 = -(n1 + n2 + n3) give grad l_k = n_k / det
// (det = e1 . n1) and S_ij = |T| grad l_i . L grad l_j = n_i . L n_j / (6 |det|).
// Here e1 = x_sigma - x_K for the whole face and, with d_t = q_t - x_K,
// n1 = d_e x d_e+1, n2 = -(e1 x d_e+1), n3 = e1 x d_e: the corner vectors
// c_t = e1 x d_t and L c_t are formed once and shared by the two tetrahedra
// at corner t.  The gradients of a tetrahedron's barycentric coordinates sum
// to zero, so every row of S, and of the face's sum F, sums to zero: only the
// entries among (sigma, q0..q3) are integrated, and the x_K row follows as
// F_K,j = -sum_i F_i,j, F_K,K = -sum_j F_K,j.
template <int SH>
__device__ __forceinline__ void cell_local(int K, int nc, const int *__restrict__ cn, const double *__restrict__ xyz,
                                           const double (&L)[6], const int *__restrict__ cell_ff, int fi, int n_fc,
                                           double *__restrict__ Mc, double *__restrict__ Mfc,
                                           double *__restrict__ cvol, int *status) {
  constexpr int NN = topo::n_nodes(SH), NF = topo::n_faces(SH);
  int nd[NN];
#pragma unroll
  for (int l = 0; l < NN; ++l) nd[l] = cn[8 * (size_t)K + l];
  V3 xK = {0, 0, 0};
#pragma unroll
  for (int l = 0; l < NN; ++l) xK = xK + ldv(xyz, nd[l]);
  xK = {xK.x / NN, xK.y / NN, xK.z / NN};

  double M[topo::kPacked];
#pragma unroll
  for (int k = 0; k < topo::kPacked; ++k) M[k] = 0.0;
  double vol = 0.0;
  double minvol = 1e300;

#pragma unroll
  for (int lf = 0; lf < NF; ++lf) {
    constexpr int Q4 = 4;
    const int Q = topo::face_size(SH, lf);     // 3 or 4, known at compile time
    const double w = 1.0 / Q;                  // beta_{sigma,s} of I_sigma
    V3 q[Q4];
#pragma unroll
    for (int t = 0; t < Q4; ++t) q[t] = t < Q ? ldv(xyz, nd[topo::face(SH, lf, t)]) : V3{0, 0, 0};
    V3 xs = q[0] + q[1] + q[2];
    if (Q == 4) xs = xs + q[3];
    xs = {xs.x / Q, xs.y / Q, xs.z / Q};
    double F[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) F[k] = 0.0;
    const V3 ev = xs - xK;
    V3 d[Q4], c[Q4], Lc[Q4];
#pragma unroll
    for (int t = 0; t < Q4; ++t) {
      if (t >= Q) break;
      d[t] = q[t] - xK;
      c[t] = cross(ev, d[t]);
      Lc[t] = lmul(L, c[t]);
    }
    // 6 |T| = |e1 . (d_e x d_e+1)| = |c_e . d_e+1| for each tetrahedron of the
    // face, and all their reciprocals from one division (prefix products)
    double a6[Q4], rinv[Q4];
#pragma unroll
    for (int e = 0; e < Q4; ++e) {
      if (e >= Q) break;
      const double ad = fabs(dot(c[e], d[e + 1 == Q ? 0 : e + 1]));
      const double tv = ad * (1.0 / 6.0);
      vol += tv;
      minvol = fmin(minvol, tv);
      a6[e] = 6.0 * ad;
    }
    {
      double pre[Q4];
      pre[0] = a6[0];
#pragma unroll
      for (int e = 1; e < Q4; ++e)
        if (e < Q) pre[e] = pre[e - 1] * a6[e];
      double r = 1.0 / pre[Q - 1];
#pragma unroll
      for (int e = Q4 - 1; e >= 1; --e) {
        if (e >= Q) continue;
        rinv[e] = r * pre[e - 1];
        r *= a6[e];
      }
      rinv[0] = r;
    }
#pragma unroll
    for (int e = 0; e < Q4; ++e) {
      if (e >= Q) break;
      const int e1 = e + 1 == Q ? 0 : e + 1;
      V3 n[3], Ln[3];   // area vectors of (sigma, q_e, q_e+1)
      n[0] = cross(d[e], d[e1]);
      Ln[0] = lmul(L, n[0]);
      n[1] = neg(c[e1]);
      Ln[1] = neg(Lc[e1]);
      n[2] = c[e];
      Ln[2] = Lc[e];
      const double inv = rinv[e];
      const int map[3] = {1, 2 + e, 2 + e1};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) F[p6(map[i], map[j])] = fma(dot(n[i], Ln[j]), inv, F[p6(map[i], map[j])]);
    }
    // the x_K row from the zero row sums
#pragma unroll
    for (int j = 1; j < 2 + Q4; ++j) {
      if (j >= 2 + Q) break;
      double sj = 0.0;
#pragma unroll
      for (int i = 1; i < 2 + Q4; ++i)
        if (i < 2 + Q) sj += F[p6(i, j)];
      F[p6(0, j)] = -sj;
    }
    {
      double sk = 0.0;
#pragma unroll
      for (int j = 1; j < 2 + Q4; ++j)
        if (j < 2 + Q) sk += F[p6(0, j)];
      F[p6(0, 0)] = -sk;
    }
    const bool isff = cell_ff[6 * (size_t)K + lf] >= 0;
    M[topo::pidx(0, 0)] += F[p6(0, 0)];
    if (!isff) {
      // x_sigma = I_sigma: the sigma row/column is spread with weight 1/Q
#pragma unroll
      for (int t = 0; t < Q4; ++t) {
        if (t >= Q) break;
        const int a = 1 + topo::face(SH, lf, t);
        M[topo::pidx(0, a)] += F[p6(0, 2 + t)] + w * F[p6(0, 1)];
#pragma unroll
        for (int u = t; u < Q4; ++u) {
          if (u >= Q) break;
          const int b = 1 + topo::face(SH, lf, u);
          M[topo::pidx(a, b)] += F[p6(2 + t, 2 + u)] + w * (F[p6(1, 2 + u)] + F[p6(1, 2 + t)]) +
                                 (w * w) * F[p6(1, 1)];
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < Q4; ++t) {
        if (t >= Q) break;
        const int a = 1 + topo::face(SH, lf, t);
        M[topo::pidx(0, a)] += F[p6(0, 2 + t)];
#pragma unroll
        for (int u = t; u < Q4; ++u) {
          if (u >= Q) break;
          const int b = 1 + topo::face(SH, lf, u);
          M[topo::pidx(a, b)] += F[p6(2 + t, 2 + u)];
        }
      }
      if (fi >= 0) {
        Mfc[(size_t)(lf * 6 + 0) * n_fc + fi] = F[p6(1, 1)];
        Mfc[(size_t)(lf * 6 + 1) * n_fc + fi] = F[p6(0, 1)];
#pragma unroll
        for (int t = 0; t < Q4; ++t) Mfc[(size_t)(lf * 6 + 2 + t) * n_fc + fi] = t < Q ? F[p6(1, 2 + t)] : 0.0;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < topo::kPacked; ++k) Mc[(size_t)k * nc + K] = M[k];
  cvol[K] = vol;
  if (!(minvol > 0.0)) atomicOr(status, ST_BAD_GEOMETRY);
}

// One thread per cell of shape SH: cell cells[i] (or cell i when the list is
// NULL, a mesh of that shape alone).  Every cell of a shape runs this one
// kernel whatever else the mesh or batch holds, so its arithmetic, and the
// system's, do not depend on the other cells.
template <int SH>
__global__ void __launch_bounds__(128) k_cell_local(int n, const int *__restrict__ cells, int nc,
                                                    const int *__restrict__ cn, const double *__restrict__ xyz,
                                                    const double *__restrict__ lam, double inv_mu,
                                                    const int *__restrict__ cell_ff, const int *__restrict__ fc_index,
                                                    int n_fc, double *__restrict__ Mc, double *__restrict__ Mfc,
                                                    double *__restrict__ cvol, int *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int K = cells ? cells[i] : i;
  double L[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) L[k] = lam[6 * (size_t)K + k] * inv_mu;
  cell_local<SH>(K, nc, cn, xyz, L, cell_ff, fc_index[K], n_fc, Mc, Mfc, cvol, status);
}

// Fracture-face matrix on (sigma, n0..n3) from the P1 tangential stiffness of
// the triangles (x_sigma, n_e, n_{e+1}) of a quadrilateral or triangular
// face (node slot 3 = -1; its row and column stay zero): with the edge vectors E_i opposite
// vertex i (E0 + E1 + E2 = 0), S_ij = coef (E_i . E_j) / (4 |T|).
__global__ void k_ff_local(int nf, const int *__restrict__ ffn, const double *__restrict__ xyz,
                           const double *__restrict__ lamf, const double *__restrict__ df, double inv_mu,
                           double *__restrict__ Mff, double *__restrict__ area, int *status) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int Q = ffn[4 * (size_t)f + 3] < 0 ? 3 : 4;   // triangle or quadrilateral
  V3 q[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) q[t] = t < Q ? ldv(xyz, ffn[4 * (size_t)f + t]) : V3{0, 0, 0};
  const V3 xs = Q == 4 ? V3{0.25 * (q[0].x + q[1].x + q[2].x + q[3].x), 0.25 * (q[0].y + q[1].y + q[2].y + q[3].y),
                            0.25 * (q[0].z + q[1].z + q[2].z + q[3].z)}
                       : V3{(q[0].x + q[1].x + q[2].x) / 3.0, (q[0].y + q[1].y + q[2].y) / 3.0,
                            (q[0].z + q[1].z + q[2].z) / 3.0};
  const double coef = df[f] * lamf[f] * inv_mu;
  double M[25];
#pragma unroll
  for (int k = 0; k < 25; ++k) M[k] = 0.0;
  double ar = 0.0, minar = 1e300;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e >= Q) break;
    const int e1 = e + 1 == Q ? 0 : e + 1;
    const V3 a = q[e], b = q[e1];
    const V3 E[3] = {b - a, xs - b, a - xs};
    const V3 nrm = cross(a - xs, b - xs);
    const double A = 0.5 * sqrt(dot(nrm, nrm));
    ar += A;
    minar = fmin(minar, A);
    const double c = coef / (4.0 * A);
    const int map[3] = {0, 1 + e, 1 + e1};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M[map[i] * 5 + map[j]] += c * dot(E[i], E[j]);
  }
#pragma unroll
  for (int k = 0; k < 25; ++k) Mff[(size_t)k * nf + f] = M[k];
  area[f] = ar;
  if (!(minar > 0.0)) atomicOr(status, ST_BAD_GEOMETRY);
}

struct GatherView {
  int nv, nc, nf, n_fc;
  const int8_t *shape;   // per-cell shape, or nullptr when every cell is a hexahedron
  const int *cn, *ffn, *node_dir, *cell_ff, *ff_cells, *ff_lface, *fc_index;
  const int *n2c_ptr, *n2c, *n2f_ptr, *n2f, *row_of_dof, *dof_of_row;
  const int *rowptr, *col, *diag_pos;
  const double *Mc, *Mfc, *Mff, *dir_vals;
  double *val, *rhs, *dinv;
};

struct RowAcc {
  const GatherView &g;
  int beg, end;
  double b;
  int *status;
  __device__ RowAcc(const GatherView &gv, int bg, int en, int *st) : g(gv), beg(bg), end(en), b(0.0), status(st) {}
  __device__ void add(int dof, double v) {
    if (dof < g.nv) {
      const int d = g.node_dir[dof];
      if (d >= 0) { b -= v * g.dir_vals[d]; return; }
    }
    const int c = g.row_of_dof[dof];
    int lo = beg, hi = end;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (g.col[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (c < 0 || lo >= end || g.col[lo] != c) { atomicOr(status, ST_NO_SLOT); return; }
    g.val[lo] += v;
  }
};

__device__ __forceinline__ double mc(const GatherView &g, int i, int j, int K) {
  return g.Mc[(size_t)topo::pidx(i, j) * g.nc + K];
}
__device__ __forceinline__ double mfc(const GatherView &g, int lf, int k, int fi) {
  return g.Mfc[(size_t)(lf * 6 + k) * g.n_fc + fi];
}

// GEN: cells of any shape (g.shape) and triangular fracture faces (node
// slot 3 = -1); otherwise every cell is a hexahedron.
template <bool GEN>
__global__ void k_gather_rows(GatherView g, int n_rows, int *status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int beg = g.rowptr[r], end = g.rowptr[r + 1];
  for (int k = beg; k < end; ++k) g.val[k] = 0.0;
  RowAcc acc(g, beg, end, status);
  const int dof = g.dof_of_row[r];
  if (dof < g.nv) {
    // node row s: Schur rows of the cells around s, then fracture rows
    for (int e = g.n2c_ptr[dof]; e < g.n2c_ptr[dof + 1]; ++e) {
      const int K = g.n2c[e] >> 3, a = g.n2c[e] & 7;
      const int sh = GEN ? g.shape[K] : topo::HEX;
      const double fac = mc(g, 0, 1 + a, K) / mc(g, 0, 0, K);     // M_aK / M_KK
      for (int bn = 0; bn < 8; ++bn) {
        const int nb = g.cn[8 * (size_t)K + bn];
        if (GEN && nb < 0) continue;
        acc.add(nb, mc(g, 1 + a, 1 + bn, K) - fac * mc(g, 0, 1 + bn, K));
      }
      const int fi = g.fc_index[K];
      if (fi >= 0) {
        for (int lf = 0; lf < 6; ++lf) {
          const int f = g.cell_ff[6 * (size_t)K + lf];
          if (f < 0) continue;
          const int t = topo::pos_on_face(sh, lf, a);
          const double Mas = t >= 0 ? mfc(g, lf, 2 + t, fi) : 0.0;
          acc.add(g.nv + f, Mas - fac * mfc(g, lf, 1, fi));
        }
      }
    }
    for (int e = g.n2f_ptr[dof]; e < g.n2f_ptr[dof + 1]; ++e) {
      const int f = g.n2f[e] >> 2, t = g.n2f[e] & 3;
      acc.add(g.nv + f, g.Mff[(size_t)((1 + t) * 5) * g.nf + f]);
      for (int u = 0; u < 4; ++u) {
        const int nb = g.ffn[4 * (size_t)f + u];
        if (GEN && nb < 0) continue;
        acc.add(nb, g.Mff[(size_t)((1 + t) * 5 + 1 + u) * g.nf + f]);
      }
    }
  } else {
    const int f = dof - g.nv;
    for (int c = 0; c < 2; ++c) {
      const int K = g.ff_cells[2 * f + c];
      if (K < 0) continue;
      const int lf = g.ff_lface[2 * f + c];
      const int fi = g.fc_index[K];
      const int sh = GEN ? g.shape[K] : topo::HEX;
      const double fac = mfc(g, lf, 1, fi) / mc(g, 0, 0, K);      // M_sigmaK / M_KK
      for (int bn = 0; bn < 8; ++bn) {
        const int nb = g.cn[8 * (size_t)K + bn];
        if (GEN && nb < 0) continue;
        const int t = topo::pos_on_face(sh, lf, bn);
        const double Msb = t >= 0 ? mfc(g, lf, 2 + t, fi) : 0.0;
        acc.add(nb, Msb - fac * mc(g, 0, 1 + bn, K));
      }
      for (int lf2 = 0; lf2 < 6; ++lf2) {
        const int f2 = g.cell_ff[6 * (size_t)K + lf2];
        if (f2 < 0) continue;
        const double Mss = lf2 == lf ? mfc(g, lf, 0, fi) : 0.0;
        acc.add(g.nv + f2, Mss - fac * mfc(g, lf2, 1, fi));
      }
    }
    acc.add(g.nv + f, g.Mff[(size_t)0 * g.nf + f]);
    for (int u = 0; u < 4; ++u) {
      const int nb = g.ffn[4 * (size_t)f + u];
      if (GEN && nb < 0) continue;
      acc.add(nb, g.Mff[(size_t)(1 + u) * g.nf + f]);
    }
  }
  g.rhs[r] = acc.b;
  const double d = g.val[g.diag_pos[r]];   // the symbolic phase guarantees a diagonal slot
  if (!(d > 0.0)) atomicOr(status, ST_NONPOSITIVE);
  g.dinv[r] = 1.0 / d;
}

// Perforation p of fracture face ff[p] adds WI[p] to the face's diagonal and
// WI[p] p_w[p] + q[p] to its right-hand side (the faces are distinct).
__global__ void k_wells(int n_perf, int nv, const int *__restrict__ ff, const double *__restrict__ wi,
                        const double *__restrict__ pw, const double *__restrict__ q, const int *__restrict__ row_of_dof,
                        const int *__restrict__ diag_pos, double *__restrict__ val, double *__restrict__ rhs,
                        double *__restrict__ dinv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_perf) return;
  const int r = row_of_dof[nv + ff[p]];
  const int k = diag_pos[r];
  const double d = val[k] + wi[p];
  val[k] = d;
  rhs[r] += fma(wi[p], pw[p], q[p]);
  dinv[r] = 1.0 / d;
}

// The local matrices of every cell: one launch for a mesh of hexahedra, one
// launch per shape over its cell list otherwise.
void launch_cell_local(System *s, double inv_mu) {
  cudaStream_t st = s->ctx->stream;
  if (!s->cell_shape) {
    k_cell_local<topo::HEX><<<grid_for(s->nc, 128), 128, 0, st>>>(s->nc, nullptr, s->nc, s->cell_nodes, s->xyz,
                                                                   s->lam, inv_mu, s->cell_ff, s->fc_index, s->n_fc,
                                                                   s->Mc, s->Mfc, s->cvol, s->status);
    note_launches(1);
    return;
  }
  decltype(&k_cell_local<topo::HEX>) kern[topo::N_SHAPES] = {k_cell_local<topo::HEX>, k_cell_local<topo::TET>,
                                                             k_cell_local<topo::PRISM>, k_cell_local<topo::PYRAMID>};
  for (int sh = 0; sh < topo::N_SHAPES; ++sh) {
    const int n = s->shape_start[sh + 1] - s->shape_start[sh];
    if (!n) continue;
    kern[sh]<<<grid_for(n, 128), 128, 0, st>>>(n, s->shape_cells + s->shape_start[sh], s->nc, s->cell_nodes,
                                               s->xyz, s->lam, inv_mu, s->cell_ff, s->fc_index, s->n_fc, s->Mc,
                                               s->Mfc, s->cvol, s->status);
    note_launches(1);
  }
}

}  // namespace

double time_cell_local(System *s, int reps) {
  if (!s->Mc) fail(VAG_EINVAL, "no local matrices: assemble first");
  cudaStream_t st = s->ctx->stream;
  const double inv_mu = 1.0 / s->mu;
  launch_cell_local(s, inv_mu);   // warm-up
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  for (int r = 0; r < reps; ++r) launch_cell_local(s, inv_mu);
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  return (double)ms / reps;
}

void numeric_phase(System *s) {
  cudaStream_t st = s->ctx->stream;
  if (!s->Mc) {
    s->Mc = sys_alloc<double>(s, (size_t)topo::kPacked * s->nc);
    s->Mfc = sys_alloc<double>(s, (size_t)36 * (s->n_fc > 0 ? s->n_fc : 1));
    s->Mff = sys_alloc<double>(s, (size_t)25 * (s->nf > 0 ? s->nf : 1));
    s->cvol = sys_alloc<double>(s, s->nc);
    s->ffarea = sys_alloc<double>(s, s->nf > 0 ? s->nf : 1);
    s->val = sys_alloc<double>(s, (size_t)s->nnz);
    s->rhs = sys_alloc<double>(s, s->n_rows);
    s->dinv = sys_alloc<double>(s, s->n_rows);
  }
  VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  const double inv_mu = 1.0 / s->mu;
  launch_cell_local(s, inv_mu);
  VAG_CHECK_LAUNCH();
  if (s->nf) {
    k_ff_local<<<grid_for(s->nf, 128), 128, 0, st>>>(s->nf, s->ff_nodes, s->xyz, s->lamf, s->df, inv_mu, s->Mff,
                                                      s->ffarea, s->status); note_launches(1);
    VAG_CHECK_LAUNCH();
  }
  GatherView g{s->nv, s->nc, s->nf, s->n_fc, s->cell_shape, s->cell_nodes, s->ff_nodes, s->node_dir, s->cell_ff,
               s->ff_cells, s->ff_lface, s->fc_index, s->n2c_ptr, s->n2c, s->n2f_ptr, s->n2f,
               s->row_of_dof, s->dof_of_row, s->rowptr, s->col, s->diag_pos, s->Mc, s->Mfc, s->Mff,
               s->dir_vals, s->val, s->rhs, s->dinv};
  if (s->cell_shape || s->tri_ff)
    k_gather_rows<true><<<grid_for(s->n_rows, 128), 128, 0, st>>>(g, s->n_rows, s->status);
  else
    k_gather_rows<false><<<grid_for(s->n_rows, 128), 128, 0, st>>>(g, s->n_rows, s->status);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  if (s->n_perf) {
    k_wells<<<grid_for(s->n_perf, 128), 128, 0, st>>>(s->n_perf, s->nv, s->well_ff, s->well_wi, s->well_pw,
                                                       s->well_q, s->row_of_dof, s->diag_pos, s->val, s->rhs,
                                                       s->dinv);
    note_launches(1);
    VAG_CHECK_LAUNCH();
  }
  if (s->sval) sell_values(s);
  s->mx.stale = true;
  s->mx.dstale = true;
  const int stv = read_status(s);
  if (stv & ST_BAD_GEOMETRY) fail(VAG_EMESH, "degenerate sub-tetrahedron or fracture triangle");
  if (stv & ST_NONPOSITIVE) fail(VAG_EINVAL, "non-positive diagonal in the eliminated system");
  if (stv & ST_NO_SLOT) fail(VAG_EMESH, "internal: a Schur contribution has no CSR slot");
}

}  // namespace vag
