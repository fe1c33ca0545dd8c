// Symbolic phase of vag_assemble (once per mesh, integer work only):
//  - Dirichlet map and fracture-node flags,
//  - fracture faces matched to cell faces through a device hash table
//    (F_Gamma,K and the cells K in M_sigma of Sec. 3.1),
//  - node -> cell and node -> fracture-face adjacency (M_s and F_Gamma,s),
//  - the Krylov unknowns (V \ V_D) u F_Gamma and the CSR pattern of the
//    cell-eliminated system of Eq. (eqschur).
#include <algorithm>

#include "vag_internal.cuh"
#include "vag_sizes.h"
#include "vag_topo.h"

namespace vag {
namespace {

constexpr int TB = 256;

__device__ __forceinline__ void flag(int *status, int bit) { atomicOr(status, bit); }

__device__ __forceinline__ void sort4(int &a, int &b, int &c, int &d) {
  int t;
#define SW(x, y) if (x > y) { t = x; x = y; y = t; }
  SW(a, b) SW(c, d) SW(a, c) SW(b, d) SW(b, c)
#undef SW
}

__device__ __forceinline__ uint32_t hash4(int a, int b, int c, int d) {
  uint64_t h = 0x9E3779B97F4A7C15ull;
  h ^= (uint32_t)a; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
  h ^= (uint32_t)b; h *= 0x94D049BB133111EBull; h ^= h >> 31;
  h ^= (uint32_t)c; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
  h ^= (uint32_t)d; h *= 0x94D049BB133111EBull; h ^= h >> 32;
  return (uint32_t)h;
}

__global__ void k_mark_dirichlet(int nd, const int *__restrict__ dir_nodes, int nv, int *node_dir,
                                 int *status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  int s = dir_nodes[i];
  if (s < 0 || s >= nv) { flag(status, ST_BAD_INDEX); return; }
  int old = atomicCAS(&node_dir[s], -1, i);
  if (old != -1) flag(status, ST_DUP_DIRICHLET);
}

// Node slot l of cell K holds a node id when l < n_nodes(shape) and -1
// otherwise.
__global__ void k_check_cells(int nc, const int8_t *__restrict__ shape, const int *__restrict__ cn, int nv,
                              int *n2c_cnt, int *status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nc * 8) return;
  const int K = (int)(i >> 3), l = (int)(i & 7);
  const int sh = shape ? shape[K] : topo::HEX;
  int s = cn[i];
  if (sh < 0 || sh >= topo::N_SHAPES) { flag(status, ST_BAD_INDEX); return; }
  if (l >= topo::n_nodes(sh)) {
    if (s != -1) flag(status, ST_BAD_INDEX);
    return;
  }
  if (s < 0 || s >= nv) { flag(status, ST_BAD_INDEX); return; }
  atomicAdd(&n2c_cnt[s], 1);
}

__global__ void k_ff_prep(int nf, const int *__restrict__ ffn, int nv, bool tri_ok, int *ffs, int *node_isfrac,
                          int *n2f_cnt, int *status) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int a = ffn[4 * f], b = ffn[4 * f + 1], c = ffn[4 * f + 2], d = ffn[4 * f + 3];
  // a quadrilateral, or a triangle with d = -1 (general meshes only)
  const bool tri = d == -1 && tri_ok;
  if (a < 0 || a >= nv || b < 0 || b >= nv || c < 0 || c >= nv || (!tri && (d < 0 || d >= nv))) {
    flag(status, ST_BAD_INDEX);
    a = b = c = d = -1;
  } else {
    node_isfrac[a] = 1; node_isfrac[b] = 1; node_isfrac[c] = 1;
    atomicAdd(&n2f_cnt[a], 1); atomicAdd(&n2f_cnt[b], 1); atomicAdd(&n2f_cnt[c], 1);
    if (!tri) { node_isfrac[d] = 1; atomicAdd(&n2f_cnt[d], 1); }
  }
  sort4(a, b, c, d);
  ffs[4 * f] = a; ffs[4 * f + 1] = b; ffs[4 * f + 2] = c; ffs[4 * f + 3] = d;
}

__global__ void k_ff_insert(int nf, const int *__restrict__ ffs, int *table, uint32_t mask, int *status) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int a = ffs[4 * f], b = ffs[4 * f + 1], c = ffs[4 * f + 2], d = ffs[4 * f + 3];
  if (b < 0) return;   // rejected face (a = -1 is a triangle's padding after sorting)
  uint32_t h = hash4(a, b, c, d) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int old = atomicCAS(&table[h], -1, f);
    if (old == -1) return;
    if (ffs[4 * old] == a && ffs[4 * old + 1] == b && ffs[4 * old + 2] == c && ffs[4 * old + 3] == d) {
      flag(status, ST_DUP_FFACE);
      return;
    }
    h = (h + 1) & mask;
  }
  flag(status, ST_HASH_FULL);
}

__global__ void k_cell_face_lookup(int nc, const int8_t *__restrict__ shape, const int *__restrict__ cn,
                                   const int *__restrict__ ffs, const int *__restrict__ table, uint32_t mask, int nf,
                                   int *cell_ff, int *ff_cnt, int *ff_cells, int *ff_lface, int *status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nc * 6) return;
  int K = (int)(i / 6), lf = (int)(i % 6);
  const int sh = shape ? shape[K] : topo::HEX;
  int res = -1;
  if (nf > 0 && lf < topo::n_faces(sh)) {
    const int t3 = topo::face(sh, lf, 3);
    int a = cn[8 * K + topo::face(sh, lf, 0)], b = cn[8 * K + topo::face(sh, lf, 1)];
    int c = cn[8 * K + topo::face(sh, lf, 2)], d = t3 >= 0 ? cn[8 * K + t3] : -1;
    sort4(a, b, c, d);
    uint32_t h = hash4(a, b, c, d) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      int f = table[h];
      if (f < 0) break;
      if (ffs[4 * f] == a && ffs[4 * f + 1] == b && ffs[4 * f + 2] == c && ffs[4 * f + 3] == d) {
        res = f;
        break;
      }
      h = (h + 1) & mask;
    }
    if (res >= 0) {
      int slot = atomicAdd(&ff_cnt[res], 1);
      if (slot < 2) {
        ff_cells[2 * res + slot] = K;
        ff_lface[2 * res + slot] = lf;
      } else {
        flag(status, ST_FACE_3CELLS);
      }
    }
  }
  cell_ff[i] = res;
}

__global__ void k_ff_finish(int nf, const int *__restrict__ ff_cnt, int *ff_cells, int *ff_lface,
                            int *status) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int n = ff_cnt[f];
  if (n == 0) { flag(status, ST_FFACE_NOT_FACE); ff_cells[2 * f] = -1; ff_cells[2 * f + 1] = -1; return; }
  if (n == 1) { ff_cells[2 * f + 1] = -1; ff_lface[2 * f + 1] = -1; return; }
  if (ff_cells[2 * f] > ff_cells[2 * f + 1]) {
    int t = ff_cells[2 * f]; ff_cells[2 * f] = ff_cells[2 * f + 1]; ff_cells[2 * f + 1] = t;
    t = ff_lface[2 * f]; ff_lface[2 * f] = ff_lface[2 * f + 1]; ff_lface[2 * f + 1] = t;
  }
}

__global__ void k_shape_flag(int nc, const int8_t *__restrict__ shape, int sh, int *flagv) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K < nc) flagv[K] = shape[K] == sh;
}

// cells of shape sh at out[scan[K]] (scan: exclusive scan of the flags)
__global__ void k_shape_fill(int nc, const int8_t *__restrict__ shape, int sh, const int *__restrict__ scan,
                             int *out) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K < nc && shape[K] == sh) out[scan[K]] = K;
}

__global__ void k_fc_flag(int nc, const int *__restrict__ cell_ff, int *flagv) {
  int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  int any = 0;
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) any |= (cell_ff[6 * K + lf] >= 0);
  flagv[K] = any;
}

__global__ void k_fc_index(int nc, const int *__restrict__ flagv, const int *__restrict__ scan, int *fc_index) {
  int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  fc_index[K] = flagv[K] ? scan[K] : -1;
}

__global__ void k_fill_adj(int64_t n_items, int per, const int *__restrict__ nodes_of,
                           const int *__restrict__ ptr, int *cursor, int *adj) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  int s = nodes_of[i];
  if (s < 0) return;
  int pos = atomicAdd(&cursor[s], 1);
  adj[ptr[s] + pos] = (int)i;   // = owner * per + local
  (void)per;
}

__global__ void k_sort_segments(int n, const int *__restrict__ ptr, int *adj) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int b = ptr[s], e = ptr[s + 1];
  for (int i = b + 1; i < e; ++i) {
    int v = adj[i];
    int j = i - 1;
    while (j >= b && adj[j] > v) { adj[j + 1] = adj[j]; --j; }
    adj[j + 1] = v;
  }
}

__global__ void k_node_flags(int nv, const int *__restrict__ node_dir, int *flagv) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nv) return;
  flagv[d] = node_dir[d] < 0;
}

// system of entity i given the segment starts (n_sys+1 entries, increasing)
__device__ __forceinline__ int seg_of(int i, const int *__restrict__ start, int n_sys) {
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Krylov rows, system by system: the non-Dirichlet nodes of system g in
// increasing id, then the fracture faces of g.  With node_rank the exclusive
// scan of the non-Dirichlet flags, node s of g gets row node_rank[s] +
// ff_start[g] and fracture face f of g gets node_rank[node_start[g+1]] + f.
__global__ void k_row_maps(int nv, int nf, int n_sys, const int *__restrict__ node_start,
                           const int *__restrict__ ff_start, const int *__restrict__ flagv,
                           const int *__restrict__ node_rank, int *row_of_dof, int *dof_of_row) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nv + nf) return;
  int row = -1;
  if (d < nv) {
    if (flagv[d]) row = node_rank[d] + ff_start[seg_of(d, node_start, n_sys)];
  } else {
    const int f = d - nv;
    row = node_rank[node_start[seg_of(f, ff_start, n_sys) + 1]] + f;
  }
  row_of_dof[d] = row;
  if (row >= 0) dof_of_row[row] = d;
}

__global__ void k_row_starts(int n_sys, const int *__restrict__ node_start, const int *__restrict__ ff_start,
                             const int *__restrict__ node_rank, int *row_start) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > n_sys) return;
  row_start[g] = node_rank[node_start[g]] + ff_start[g];
}

struct PatView {
  int nv, nf;
  const int *cn, *ffn, *node_dir, *cell_ff, *ff_cells, *n2c_ptr, *n2c, *n2f_ptr, *n2f, *row_of_dof;
};

// Sorted set of at most kMaxRowWidth DOF ids kept in thread-local storage.
struct RowSet {
  int v[kMaxRowWidth];
  int n = 0;
  bool overflow = false;
  __device__ void insert(int x) {
    int lo = 0, hi = n;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    if (lo < n && v[lo] == x) return;
    if (n == kMaxRowWidth) { overflow = true; return; }
    for (int j = n; j > lo; --j) v[j] = v[j - 1];
    v[lo] = x;
    ++n;
  }
};

__device__ void row_add_cell(const PatView &p, RowSet &rs, int K) {
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    int s = p.cn[8 * K + l];
    if (s >= 0 && p.node_dir[s] < 0) rs.insert(s);
  }
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    int f = p.cell_ff[6 * K + lf];
    if (f >= 0) rs.insert(p.nv + f);
  }
}

__device__ void row_add_ff(const PatView &p, RowSet &rs, int f) {
  rs.insert(p.nv + f);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int s = p.ffn[4 * f + t];
    if (s >= 0 && p.node_dir[s] < 0) rs.insert(s);
  }
}

__device__ void row_collect(const PatView &p, int dof, RowSet &rs) {
  if (dof < p.nv) {
    for (int e = p.n2c_ptr[dof]; e < p.n2c_ptr[dof + 1]; ++e) row_add_cell(p, rs, p.n2c[e] >> 3);
    for (int e = p.n2f_ptr[dof]; e < p.n2f_ptr[dof + 1]; ++e) row_add_ff(p, rs, p.n2f[e] >> 2);
  } else {
    int f = dof - p.nv;
    for (int c = 0; c < 2; ++c) {
      int K = p.ff_cells[2 * f + c];
      if (K >= 0) row_add_cell(p, rs, K);
    }
    row_add_ff(p, rs, f);
  }
}

__global__ void k_row_count(PatView p, int n_rows, const int *__restrict__ dof_of_row, int *cnt, int *status) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  RowSet rs;
  const int dof = dof_of_row[r];
  row_collect(p, dof, rs);
  if (rs.overflow) flag(status, ST_ROW_OVERFLOW);
  bool has_diag = false;
  for (int j = 0; j < rs.n; ++j) has_diag |= (rs.v[j] == dof);
  if (!has_diag) flag(status, ST_ISOLATED);
  cnt[r] = rs.n;
}

__global__ void k_row_fill(PatView p, int n_rows, const int *__restrict__ dof_of_row,
                           const int *__restrict__ rowptr, int *col, int *diag_pos) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  RowSet rs;
  int dof = dof_of_row[r];
  row_collect(p, dof, rs);
  int b = rowptr[r];
  int n = min(rs.n, rowptr[r + 1] - b);
  for (int j = 0; j < n; ++j) {
    int c = p.row_of_dof[rs.v[j]];
    col[b + j] = c;
    if (c == r) diag_pos[r] = b + j;
  }
}

}  // namespace

void symbolic_phase(System *s) {
  cudaStream_t st = s->ctx->stream;
  const int nv = s->nv, nc = s->nc, nf = s->nf, nd = s->nd;

  s->node_dir = sys_alloc<int>(s, nv);
  s->node_isfrac = sys_alloc<int>(s, nv);
  s->cell_ff = sys_alloc<int>(s, 6 * (size_t)nc);
  s->ff_cells = sys_alloc<int>(s, 2 * (size_t)nf);
  s->ff_lface = sys_alloc<int>(s, 2 * (size_t)nf);
  s->fc_index = sys_alloc<int>(s, nc);
  s->n2c_ptr = sys_alloc<int>(s, nv + 1);
  s->n2c = sys_alloc<int>(s, 8 * (size_t)nc);
  s->n2f_ptr = sys_alloc<int>(s, nv + 1);
  s->n2f = sys_alloc<int>(s, 4 * (size_t)nf);
  s->row_of_dof = sys_alloc<int>(s, nv + nf);

  // scratch (stream-ordered, released at the end of the phase)
  const size_t ncnt = (size_t)nv + 1;
  int *n2c_cnt, *n2f_cnt, *cursor, *ffs, *table, *ff_cnt, *flagv, *scanv;
  uint32_t H = 2;
  while (H < 2u * (uint32_t)(nf > 0 ? nf : 1)) H <<= 1;
  const size_t nflag = std::max<size_t>({(size_t)nc, (size_t)nv + nf, 1}) + 1;
  VAG_CUDA(cudaMallocAsync(&n2c_cnt, sizeof(int) * ncnt, st));
  VAG_CUDA(cudaMallocAsync(&n2f_cnt, sizeof(int) * ncnt, st));
  VAG_CUDA(cudaMallocAsync(&cursor, sizeof(int) * ncnt, st));
  VAG_CUDA(cudaMallocAsync(&ffs, sizeof(int) * 4 * (size_t)(nf > 0 ? nf : 1), st));
  VAG_CUDA(cudaMallocAsync(&table, sizeof(int) * H, st));
  VAG_CUDA(cudaMallocAsync(&ff_cnt, sizeof(int) * (size_t)(nf > 0 ? nf : 1), st));
  VAG_CUDA(cudaMallocAsync(&flagv, sizeof(int) * nflag, st));
  VAG_CUDA(cudaMallocAsync(&scanv, sizeof(int) * nflag, st));

  VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
  VAG_CUDA(cudaMemsetAsync(s->node_dir, 0xff, sizeof(int) * nv, st));
  VAG_CUDA(cudaMemsetAsync(s->node_isfrac, 0, sizeof(int) * nv, st));
  VAG_CUDA(cudaMemsetAsync(n2c_cnt, 0, sizeof(int) * ncnt, st));
  VAG_CUDA(cudaMemsetAsync(n2f_cnt, 0, sizeof(int) * ncnt, st));
  VAG_CUDA(cudaMemsetAsync(table, 0xff, sizeof(int) * H, st));
  VAG_CUDA(cudaMemsetAsync(ff_cnt, 0, sizeof(int) * (size_t)(nf > 0 ? nf : 1), st));

  k_mark_dirichlet<<<grid_for(nd, TB), TB, 0, st>>>(nd, s->dir_nodes, nv, s->node_dir, s->status); note_launches(1);
  k_check_cells<<<grid_for((int64_t)nc * 8, TB), TB, 0, st>>>(nc, s->cell_shape, s->cell_nodes, nv, n2c_cnt,
                                                               s->status); note_launches(1);
  if (nf) {
    k_ff_prep<<<grid_for(nf, TB), TB, 0, st>>>(nf, s->ff_nodes, nv, s->tri_ff, ffs, s->node_isfrac, n2f_cnt,
                                               s->status); note_launches(1);
    k_ff_insert<<<grid_for(nf, TB), TB, 0, st>>>(nf, ffs, table, H - 1, s->status); note_launches(1);
  }
  VAG_CHECK_LAUNCH();
  // bad indices make every later kernel unsafe: stop here
  int st0 = read_status(s);
  if (st0 & ST_BAD_INDEX) fail(VAG_EINVAL, "mesh or Dirichlet index out of range");
  if (st0 & ST_DUP_DIRICHLET) fail(VAG_EINVAL, "a Dirichlet node is listed twice");
  if (st0 & ST_DUP_FFACE) fail(VAG_EMESH, "a fracture face is listed twice");
  if (st0 & ST_HASH_FULL) fail(VAG_EMESH, "fracture-face table overflow");

  k_cell_face_lookup<<<grid_for((int64_t)nc * 6, TB), TB, 0, st>>>(
      nc, s->cell_shape, s->cell_nodes, ffs, table, H - 1, nf, s->cell_ff, ff_cnt, s->ff_cells, s->ff_lface,
      s->status); note_launches(1);
  if (nf) {
    k_ff_finish<<<grid_for(nf, TB), TB, 0, st>>>(nf, ff_cnt, s->ff_cells, s->ff_lface, s->status);
    note_launches(1);
  }
  VAG_CHECK_LAUNCH();

  // cells grouped by shape (general meshes with some non-hexahedral cell)
  if (s->cell_shape) {
    s->shape_cells = sys_alloc<int>(s, nc);
    s->shape_start[0] = 0;
    for (int sh = 0; sh < topo::N_SHAPES; ++sh) {
      k_shape_flag<<<grid_for(nc, TB), TB, 0, st>>>(nc, s->cell_shape, sh, flagv);
      const int cnt = scan_exclusive(flagv, scanv, nc, st);
      k_shape_fill<<<grid_for(nc, TB), TB, 0, st>>>(nc, s->cell_shape, sh, scanv,
                                                    s->shape_cells + s->shape_start[sh]);
      note_launches(2);
      s->shape_start[sh + 1] = s->shape_start[sh] + cnt;
    }
    VAG_CHECK_LAUNCH();
    if (s->shape_start[topo::N_SHAPES] != nc) fail(VAG_EMESH, "a cell has no known shape");
  }

  // fracture cells
  k_fc_flag<<<grid_for(nc, TB), TB, 0, st>>>(nc, s->cell_ff, flagv); note_launches(1);
  s->n_fc = scan_exclusive(flagv, scanv, nc, st);
  k_fc_index<<<grid_for(nc, TB), TB, 0, st>>>(nc, flagv, scanv, s->fc_index); note_launches(1);

  // node -> cell adjacency, sorted by cell id
  scan_exclusive(n2c_cnt, s->n2c_ptr, nv, st, false);
  VAG_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * ncnt, st));
  k_fill_adj<<<grid_for((int64_t)nc * 8, TB), TB, 0, st>>>((int64_t)nc * 8, 8, s->cell_nodes, s->n2c_ptr,
                                                          cursor, s->n2c); note_launches(1);
  k_sort_segments<<<grid_for(nv, TB), TB, 0, st>>>(nv, s->n2c_ptr, s->n2c); note_launches(1);
  // node -> fracture-face adjacency
  scan_exclusive(n2f_cnt, s->n2f_ptr, nv, st, false);
  if (nf) {
    VAG_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * ncnt, st));
    k_fill_adj<<<grid_for((int64_t)nf * 4, TB), TB, 0, st>>>((int64_t)nf * 4, 4, s->ff_nodes, s->n2f_ptr,
                                                            cursor, s->n2f); note_launches(1);
    k_sort_segments<<<grid_for(nv, TB), TB, 0, st>>>(nv, s->n2f_ptr, s->n2f); note_launches(1);
  }
  VAG_CHECK_LAUNCH();

  // Krylov unknowns, contiguous per system of the batch
  k_node_flags<<<grid_for(nv, TB), TB, 0, st>>>(nv, s->node_dir, flagv);
  note_launches(1);
  const int n_row_nodes = scan_exclusive(flagv, scanv, nv, st);
  s->n_rows = n_row_nodes + nf;
  s->n_row_nodes = n_row_nodes;
  s->dof_of_row = sys_alloc<int>(s, s->n_rows);
  Segments &g = s->seg;
  k_row_maps<<<grid_for(nv + nf, TB), TB, 0, st>>>(nv, nf, g.n_sys, g.d_node_start, g.d_ff_start, flagv, scanv,
                                                   s->row_of_dof, s->dof_of_row);
  note_launches(1);
  k_row_starts<<<grid_for(g.n_sys + 1, TB), TB, 0, st>>>(g.n_sys, g.d_node_start, g.d_ff_start, scanv,
                                                         g.d_row_start);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  g.row_start.assign(g.n_sys + 1, 0);
  VAG_CUDA(cudaMemcpyAsync(g.row_start.data(), g.d_row_start, sizeof(int) * (g.n_sys + 1), cudaMemcpyDeviceToHost,
                           st));

  int st1 = read_status(s);
  if (st1 & ST_FFACE_NOT_FACE) fail(VAG_EMESH, "a fracture face is not a face of any cell");
  if (st1 & ST_FACE_3CELLS) fail(VAG_EMESH, "a fracture face is shared by more than two cells");

  // CSR pattern of the eliminated system
  PatView pv{nv, nf, s->cell_nodes, s->ff_nodes, s->node_dir, s->cell_ff, s->ff_cells,
             s->n2c_ptr, s->n2c, s->n2f_ptr, s->n2f, s->row_of_dof};
  s->rowptr = sys_alloc<int>(s, (size_t)s->n_rows + 1);
  s->diag_pos = sys_alloc<int>(s, s->n_rows);
  int *cnt;
  VAG_CUDA(cudaMallocAsync(&cnt, sizeof(int) * ((size_t)s->n_rows + 1), st));
  k_row_count<<<grid_for(s->n_rows, 128), 128, 0, st>>>(pv, s->n_rows, s->dof_of_row, cnt, s->status); note_launches(1);
  VAG_CHECK_LAUNCH();
  if ((int64_t)s->n_rows * kMaxRowWidth > INT32_MAX) {
    // Row pointers, sliced-ELL offsets and column indices are int32: a system
    // this large may hold more stored entries than they address, so count
    // them exactly (64-bit, on the host) before the 32-bit scan.
    std::vector<int> h((size_t)s->n_rows);
    VAG_CUDA(cudaMemcpyAsync(h.data(), cnt, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (!fits_int32_indices(h.data(), h.size()))
      fail(VAG_EINVAL, "the eliminated system holds more than 2^31 - 1 stored entries (int32 indices)");
  }
  s->nnz = scan_exclusive(cnt, s->rowptr, s->n_rows, st);
  const int st2 = read_status(s);
  if (st2 & ST_ROW_OVERFLOW) fail(VAG_EMESH, "an eliminated row couples too many unknowns");
  if (st2 & ST_ISOLATED) fail(VAG_EMESH, "a node belongs to no cell");
  s->col = sys_alloc<int>(s, (size_t)s->nnz);
  k_row_fill<<<grid_for(s->n_rows, 128), 128, 0, st>>>(pv, s->n_rows, s->dof_of_row, s->rowptr, s->col,
                                                      s->diag_pos); note_launches(1);
  VAG_CHECK_LAUNCH();

  VAG_CUDA(cudaFreeAsync(cnt, st));
  VAG_CUDA(cudaFreeAsync(n2c_cnt, st));
  VAG_CUDA(cudaFreeAsync(n2f_cnt, st));
  VAG_CUDA(cudaFreeAsync(cursor, st));
  VAG_CUDA(cudaFreeAsync(ffs, st));
  VAG_CUDA(cudaFreeAsync(table, st));
  VAG_CUDA(cudaFreeAsync(ff_cnt, st));
  VAG_CUDA(cudaFreeAsync(flagv, st));
  VAG_CUDA(cudaFreeAsync(scanv, st));
  VAG_CUDA(cudaStreamSynchronize(st));
}

}  // namespace vag
