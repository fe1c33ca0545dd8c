// Aggregation algebraic multigrid preconditioner for the eliminated VAG
// system (the paper's §5 compares Trilinos aggregation AMG and Hypre's
// classical AMG as GMRES/BiCGStab preconditioners; this is the library's own
// aggregation AMG, used inside CG).
//
// Setup, level by level, all on the device:
//  strength   j is a strong neighbour of i if |a_ij| >= theta sqrt(a_ii a_jj);
//  MIS(2)     roots: undecided nodes whose key is the largest within two
//             strong hops (keys hash the system-local row index, so a system's
//             hierarchy does not depend on the rest of a batch); nodes within
//             two hops of a root drop out; repeat until no node is undecided;
//  aggregates a root and its strong neighbours, then every remaining node
//             joins the aggregate of its strongest aggregated neighbour; nodes
//             without a strong neighbour stay out of the coarse space;
//  Galerkin   A_c = P^T A P for the piecewise-constant P, one thread per
//             coarse row summing its members' rows in row order;
//  terminal   a system whose level has at most kDenseMax rows leaves the
//             hierarchy there: its block is inverted densely (Gauss-Jordan,
//             SPD) and applied exactly in the cycle.  The depth of a system's
//             hierarchy therefore depends on that system alone.
// Apply: a V(2,2) cycle with damped Jacobi (omega = 2/3) before and after the
// coarse correction; it is a fixed symmetric linear operator, as CG needs.
#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int TB = 256;
constexpr double kTheta = 0.08;
constexpr double kOmega = 2.0 / 3.0;
constexpr int kDenseMax = 48;       // two 48x48 FP64 blocks fit the static shared limit
constexpr int kMaxLevels = 16;
constexpr int kCoarseWidth = 160;   // unique columns of one coarse row (< 256)

constexpr unsigned long long KEY_IN = ~0ull;
constexpr unsigned long long KEY_OUT = 0ull;

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x | 1u;
}

__device__ __forceinline__ int sys_of_row(int i, const int *__restrict__ start, int n_sys) {
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// strength mask per CSR entry, isolated flag per row, diagonal inverse
__global__ void k_strength(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ dinv,
                           const uint8_t *__restrict__ skip, uint8_t *strong, int8_t *state) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (skip[i]) {   // terminal system: no aggregation at all
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) strong[k] = 0;
    state[i] = -2;
    return;
  }
  const double di = 1.0 / dinv[i];
  int cnt = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = col[k];
    const double dj = 1.0 / dinv[j];
    const bool s = (j != i) && fabs(val[k]) >= kTheta * sqrt(fabs(di * dj));
    strong[k] = s;
    cnt += s;
  }
  state[i] = cnt ? 0 : -2;   // 0 undecided, 1 root, -1 out, -2 isolated
}

__global__ void k_skip_rows(int n, const int *__restrict__ sys_start, int n_sys, const uint8_t *__restrict__ term,
                            uint8_t *skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) skip[i] = term[sys_of_row(i, sys_start, n_sys)];
}

__device__ __forceinline__ unsigned long long node_key(int i, int8_t st, const int *__restrict__ sys_start, int n_sys) {
  if (st == 1) return KEY_IN;
  if (st != 0) return KEY_OUT;
  const int loc = i - sys_start[sys_of_row(i, sys_start, n_sys)];
  return ((unsigned long long)hash32((uint32_t)loc) << 32) | (uint32_t)i;
}

__global__ void k_mis_max1(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                           const int *__restrict__ sys_start, int n_sys, unsigned long long *m1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = node_key(i, state[i], sys_start, n_sys);
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
    if (strong[k]) {
      const int j = col[k];
      const unsigned long long kj = node_key(j, state[j], sys_start, n_sys);
      m = kj > m ? kj : m;
    }
  m1[i] = m;
}

__global__ void k_mis_max2_decide(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                  const uint8_t *__restrict__ strong, int8_t *state,
                                  const unsigned long long *__restrict__ m1, const int *__restrict__ sys_start,
                                  int n_sys, int8_t *next, int *undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int8_t st = state[i];
  int8_t ns = st;
  if (st == 0) {
    unsigned long long m = m1[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (strong[k]) {
        const unsigned long long v = m1[col[k]];
        m = v > m ? v : m;
      }
    if (m == node_key(i, st, sys_start, n_sys)) ns = 1;
    else if (m == KEY_IN) ns = -1;
    else atomicAdd(undecided, 1);
  }
  next[i] = ns;
}

__global__ void k_root_flags(int n, const int8_t *__restrict__ state, int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == 1;
}

// pass 1: roots get their id; nodes next to a root (strongly) join it
__global__ void k_agg_pass1(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                            const int *__restrict__ rscan, int *agg1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = -1;
  if (state[i] == 1) {
    a = rscan[i];
  } else if (state[i] != -2) {
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (strong[k] && state[col[k]] == 1) { a = rscan[col[k]]; break; }
  }
  agg1[i] = a;
}

// pass 2: remaining nodes join their strongest aggregated neighbour
__global__ void k_agg_pass2(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ dinv,
                            const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                            const int *__restrict__ agg1, int *agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0 && state[i] != -2) {
    double best = -1.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (!strong[k]) continue;
      const int j = col[k];
      if (agg1[j] < 0) continue;
      const double w = fabs(val[k]) * sqrt(dinv[j]);
      if (w > best) { best = w; a = agg1[j]; }
    }
  }
  agg[i] = a;
}

__global__ void k_member_count(int n, const int *__restrict__ agg, int *cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void k_member_fill(int n, const int *__restrict__ agg, const int *__restrict__ mptr, int *cursor,
                              int *mem) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  const int a = agg[i];
  mem[mptr[a] + atomicAdd(&cursor[a], 1)] = i;
}

__global__ void k_sort_members(int nc, const int *__restrict__ mptr, int *mem) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  for (int p = mptr[I] + 1; p < mptr[I + 1]; ++p) {
    const int v = mem[p];
    int q = p - 1;
    while (q >= mptr[I] && mem[q] > v) { mem[q + 1] = mem[q]; --q; }
    mem[q + 1] = v;
  }
}

// One coarse row of A_c = P^T A P: the entries of the members' rows (members
// in row order, entries in CSR order) are summed per coarse column in a
// thread-local open-addressing table; columns are emitted in order of first
// appearance, so the sums and their order are deterministic.
constexpr int kHash = 256;
__global__ void __launch_bounds__(64) k_coarse_build(int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                                                     const int *__restrict__ rowptr, const int *__restrict__ col,
                                                     const double *__restrict__ val, const int *__restrict__ agg,
                                                     int *tcol, double *tval, int *cnt, double *cdinv, int *status) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int keys[kHash];
  double sums[kHash];
  unsigned char slot_of[kCoarseWidth];
  for (int h = 0; h < kHash; ++h) keys[h] = -1;
  int n = 0;
  bool overflow = false;
  for (int p = mptr[I]; p < mptr[I + 1]; ++p) {
    const int i = mem[p];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int J = agg[col[k]];
      if (J < 0) continue;
      unsigned h = ((unsigned)J * 2654435761u) & (kHash - 1);
      while (keys[h] != -1 && keys[h] != J) h = (h + 1) & (kHash - 1);
      if (keys[h] == J) {
        sums[h] += val[k];
      } else if (n < kCoarseWidth) {
        keys[h] = J;
        sums[h] = val[k];
        slot_of[n++] = (unsigned char)h;
      } else {
        overflow = true;
      }
    }
  }
  if (overflow) atomicOr(status, ST_ROW_OVERFLOW);
  double d = 0.0;
  const size_t base = (size_t)I * kCoarseWidth;
  for (int q = 0; q < n; ++q) {
    const int h = slot_of[q];
    tcol[base + q] = keys[h];
    tval[base + q] = sums[h];
    if (keys[h] == I) d = sums[h];
  }
  cnt[I] = n;
  if (!(d > 0.0)) atomicOr(status, ST_NONPOSITIVE);
  cdinv[I] = 1.0 / d;
}

__global__ void k_coarse_compact(int nc, const int *__restrict__ tcol, const double *__restrict__ tval,
                                 const int *__restrict__ rowptr, int *col, double *val) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const size_t base = (size_t)I * kCoarseWidth;
  for (int q = 0; q < rowptr[I + 1] - rowptr[I]; ++q) {
    col[rowptr[I] + q] = tcol[base + q];
    val[rowptr[I] + q] = tval[base + q];
  }
}

__global__ void k_coarse_starts(int n_sys, const int *__restrict__ sys_start, const int *__restrict__ rscan,
                                int *csys_start) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g <= n_sys) csys_start[g] = rscan[sys_start[g]];
}

// Dense inverse of each system's coarsest block (Gauss-Jordan without
// pivoting: the block is SPD), one thread block per system.
__global__ void k_dense_inverse(const int *__restrict__ sys_start, const int *__restrict__ rowptr,
                                const int *__restrict__ col, const double *__restrict__ val,
                                const long long *__restrict__ off, double *inv, int *status) {
  __shared__ double A[kDenseMax * kDenseMax];
  __shared__ double B[kDenseMax * kDenseMax];
  const int g = blockIdx.x;
  const int r0 = sys_start[g], m = sys_start[g + 1] - r0;
  if (m == 0 || off[g + 1] - off[g] != (long long)m * m) return;   // not terminal here
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    A[e] = 0.0;
    B[e] = (e / m == e % m) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    for (int k = rowptr[r0 + i]; k < rowptr[r0 + i + 1]; ++k) A[i * m + (col[k] - r0)] = val[k];
  __syncthreads();
  for (int p = 0; p < m; ++p) {
    const double piv = A[p * m + p];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) atomicOr(status, ST_NONPOSITIVE);
      return;   // uniform across the block: every thread read the same pivot
    }
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      A[p * m + j] /= piv;
      B[p * m + j] /= piv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e / m, j = e % m;
      if (i == p) continue;
      const double f = A[i * m + p];
      if (j != p) A[i * m + j] -= f * A[p * m + j];
      B[i * m + j] -= f * B[p * m + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      if (i != p) A[i * m + p] = 0.0;
    __syncthreads();
  }
  double *out = inv + off[g];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) out[e] = B[e];
}

// ------------------------------------------------------------- V-cycle ----
// Templated on the value type: T = double (FP64 hierarchy) or float (FP32
// copy of the hierarchy, for the mixed-precision path).

template <class T>
__global__ void k_jac_first(int n, const T *__restrict__ b, const T *__restrict__ dinv, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)kOmega * dinv[i] * b[i];
}

// x_out = x_in + omega D^-1 (b - A x_in), CSR, one thread per row
template <class T>
__global__ void k_jac_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                          const T *__restrict__ val, const T *__restrict__ dinv, const T *__restrict__ b,
                          const T *__restrict__ xin, T *__restrict__ xout, const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || skip[i]) return;
  T s = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], xin[col[k]], s);
  xout[i] = fma((T)kOmega * dinv[i], b[i] - s, xin[i]);
}

// same sweep in the sliced-ELL layout (finest level)
template <class T>
__global__ void k_jac_sell(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                           const int *__restrict__ scol, const T *__restrict__ sval, const T *__restrict__ dinv,
                           const T *__restrict__ b, const T *__restrict__ xin, T *__restrict__ xout,
                           const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || skip[i]) return;
  const int len = rowptr[i + 1] - rowptr[i];
  const int base = slice_ptr[i >> 5] + (i & 31);
  T s = 0;
#pragma unroll 4
  for (int k = 0; k < len; ++k) {
    const int idx = base + 32 * k;
    s = fma(sval[idx], __ldg(&xin[scol[idx]]), s);
  }
  xout[i] = fma((T)kOmega * dinv[i], b[i] - s, xin[i]);
}

// r = b - A x, one thread per row (CSR / sliced ELL)
template <class T>
__global__ void k_resid_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const T *__restrict__ val, const T *__restrict__ b, const T *__restrict__ x,
                            T *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], x[col[k]], s);
  r[i] = b[i] - s;
}

template <class T>
__global__ void k_resid_sell(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                             const int *__restrict__ scol, const T *__restrict__ sval, const T *__restrict__ b,
                             const T *__restrict__ x, T *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int len = rowptr[i + 1] - rowptr[i];
  const int base = slice_ptr[i >> 5] + (i & 31);
  T s = 0;
#pragma unroll 4
  for (int k = 0; k < len; ++k) {
    const int idx = base + 32 * k;
    s = fma(sval[idx], __ldg(&x[scol[idx]]), s);
  }
  r[i] = b[i] - s;
}

// b_c[I] = sum of r over the members of aggregate I (row order)
template <class T>
__global__ void k_restrict(int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                           const T *__restrict__ r, T *__restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  T acc = 0;
  for (int p = mptr[I]; p < mptr[I + 1]; ++p) acc += r[mem[p]];
  bc[I] = acc;
}

template <class T>
__global__ void k_prolong(int n, const int *__restrict__ agg, const T *__restrict__ xc, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) x[i] += xc[agg[i]];
}

// x = inv_g b per system block (one thread block per system)
template <class T>
__global__ void k_dense_apply(const int *__restrict__ sys_start, const long long *__restrict__ off,
                              const T *__restrict__ inv, const T *__restrict__ b, T *x) {
  const int g = blockIdx.x;
  const int r0 = sys_start[g], m = sys_start[g + 1] - r0;
  if (m == 0 || off[g + 1] - off[g] != (long long)m * m) return;   // not terminal here
  const T *M = inv + off[g];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T s = 0;
    for (int j = 0; j < m; ++j) s = fma(M[i * m + j], b[r0 + j], s);
    x[r0 + i] = s;
  }
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_f64(int n, const float *__restrict__ a, double *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

static void free_later(std::vector<void *> &v, void *p) { v.push_back(p); }

// Build the hierarchy for the current matrix values (called before every
// AMG solve: the numeric phase may have changed them).
void amg_setup(System *s, bool f32) {
  cudaStream_t st = s->ctx->stream;
  Amg &A = s->amg;
  const int ns = s->seg.n_sys;
  // the device memory of a previous hierarchy is reused only if the
  // structure matches; simplest: free the old one (its allocations are
  // tracked separately from the system's)
  for (void *p : A.allocs) ctx_free(s->ctx, p);
  A.allocs.clear();
  A.levels.clear();
  s->ctx->in_use -= A.bytes;
  A.bytes = 0;
  auto alloc = [&](size_t bytes) -> void * {
    bytes = (bytes + 255) & ~size_t(255);
    if (!bytes) bytes = 256;
    if (s->ctx->budget && s->ctx->in_use + bytes > s->ctx->budget) fail(VAG_EBUDGET, "AMG hierarchy exceeds the budget");
    void *p = ctx_alloc(s->ctx, bytes);
    A.allocs.push_back(p);
    A.bytes += bytes;
    s->ctx->in_use += bytes;
    return p;
  };
  // level 0 is the system matrix itself
  AmgLevel L0;
  L0.n = s->n_rows;
  L0.nnz = s->nnz;
  L0.rowptr = s->rowptr;
  L0.col = s->col;
  L0.val = s->val;
  L0.dinv = s->dinv;
  L0.sys_start = s->seg.row_start;
  L0.d_sys_start = s->seg.d_row_start;
  L0.slice_ptr = s->slice_ptr;
  L0.scol = s->scol;
  L0.sval = s->sval;
  L0.sell_nnz = s->sell_nnz;
  A.levels.push_back(L0);
  int *undecided = static_cast<int *>(alloc(sizeof(int)));
  int *und_host = s->n_done_host;   // pinned int
  std::vector<uint8_t> term(ns);
  std::vector<long long> off(ns + 1);
  for (int lvl = 0;; ++lvl) {
    if (lvl == kMaxLevels) fail(VAG_ECUDA, "AMG: hierarchy deeper than the level cap");
    // systems that end here: at most kDenseMax rows at this level (a system
    // that ended earlier has no rows left)
    {
      AmgLevel &L = A.levels[lvl];
      const int n = L.n;
      bool any = false, all = true;
      off[0] = 0;
      for (int g = 0; g < ns; ++g) {
        const int m = L.sys_start[g + 1] - L.sys_start[g];
        term[g] = m <= kDenseMax;
        any |= term[g] && m > 0;
        all &= term[g];
        off[g + 1] = off[g] + (term[g] && m > 0 ? (long long)m * m : 0);
      }
      L.any_term = any;
      L.all_term = all;
      L.n_inv = off[ns];
      uint8_t *dterm = static_cast<uint8_t *>(alloc(ns));
      VAG_CUDA(cudaMemcpyAsync(dterm, term.data(), ns, cudaMemcpyHostToDevice, st));
      L.skip = static_cast<uint8_t *>(alloc(std::max(n, 1)));
      k_skip_rows<<<grid_for(n, TB), TB, 0, st>>>(n, L.d_sys_start, ns, dterm, L.skip);
      note_launches(1);
      if (any) {
        L.inv = static_cast<double *>(alloc(8 * (size_t)std::max<long long>(off[ns], 1)));
        L.inv_off = static_cast<long long *>(alloc(8 * ((size_t)ns + 1)));
        VAG_CUDA(cudaMemcpyAsync(L.inv_off, off.data(), 8 * (ns + 1), cudaMemcpyHostToDevice, st));
        VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
        k_dense_inverse<<<ns, TB, 0, st>>>(L.d_sys_start, L.rowptr, L.col, L.val, L.inv_off, L.inv, s->status);
        note_launches(1);
        VAG_CHECK_LAUNCH();
        if (read_status(s) & ST_NONPOSITIVE) fail(VAG_EINVAL, "AMG: a terminal block is not positive definite");
      }
      if (all) break;
    }
    AmgLevel &L = A.levels[lvl];
    const int n = L.n;
    uint8_t *strong = static_cast<uint8_t *>(alloc(L.nnz));
    int8_t *state = static_cast<int8_t *>(alloc(n));
    int8_t *next = static_cast<int8_t *>(alloc(n));
    unsigned long long *m1 = static_cast<unsigned long long *>(alloc(8 * (size_t)n));
    k_strength<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, L.val, L.dinv, L.skip, strong, state);
    note_launches(1);
    for (int it = 0; it < 64; ++it) {
      VAG_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int), st));
      k_mis_max1<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, L.d_sys_start, ns, m1);
      k_mis_max2_decide<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, m1, L.d_sys_start, ns,
                                                         next, undecided);
      note_launches(2);
      VAG_CUDA(cudaMemcpyAsync(state, next, n, cudaMemcpyDeviceToDevice, st));
      VAG_CUDA(cudaMemcpyAsync(und_host, undecided, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*und_host == 0) break;
    }
    if (*und_host != 0) fail(VAG_ECUDA, "AMG: MIS(2) did not finish in 64 rounds");
    int *flag = static_cast<int *>(alloc(4 * (size_t)n));
    int *rscan = static_cast<int *>(alloc(4 * ((size_t)n + 1)));
    k_root_flags<<<grid_for(n, TB), TB, 0, st>>>(n, state, flag);
    note_launches(1);
    const int nc = scan_exclusive(flag, rscan, n, st);
    int *agg1 = static_cast<int *>(alloc(4 * (size_t)n));
    L.agg = static_cast<int *>(alloc(4 * (size_t)n));
    k_agg_pass1<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, rscan, agg1);
    k_agg_pass2<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, L.val, L.dinv, strong, state, agg1, L.agg);
    note_launches(2);
    // members of every aggregate, sorted by row
    L.nc = nc;
    int *cnt = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
    int *cursor = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
    L.mptr = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
    VAG_CUDA(cudaMemsetAsync(cnt, 0, 4 * ((size_t)nc + 1), st));
    VAG_CUDA(cudaMemsetAsync(cursor, 0, 4 * ((size_t)nc + 1), st));
    k_member_count<<<grid_for(n, TB), TB, 0, st>>>(n, L.agg, cnt);
    note_launches(1);
    const int nmem = scan_exclusive(cnt, L.mptr, nc, st);
    L.mem = static_cast<int *>(alloc(4 * (size_t)std::max(nmem, 1)));
    k_member_fill<<<grid_for(n, TB), TB, 0, st>>>(n, L.agg, L.mptr, cursor, L.mem);
    k_sort_members<<<grid_for(nc, TB), TB, 0, st>>>(nc, L.mptr, L.mem);
    note_launches(2);
    // Galerkin coarse matrix, then its sliced-ELL copy
    AmgLevel C;
    C.n = nc;
    C.rowptr = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
    C.dinv = static_cast<double *>(alloc(8 * (size_t)std::max(nc, 1)));
    int *tcol;
    double *tval;
    VAG_CUDA(cudaMallocAsync(&tcol, 4 * (size_t)std::max(nc, 1) * kCoarseWidth, st));
    VAG_CUDA(cudaMallocAsync(&tval, 8 * (size_t)std::max(nc, 1) * kCoarseWidth, st));
    VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
    k_coarse_build<<<grid_for(nc, 64), 64, 0, st>>>(nc, L.mptr, L.mem, L.rowptr, L.col, L.val, L.agg, tcol, tval, cnt,
                                                     C.dinv, s->status);
    note_launches(1);
    C.nnz = scan_exclusive(cnt, C.rowptr, nc, st);
    const int cst = read_status(s);
    if (cst & ST_ROW_OVERFLOW) fail(VAG_EMESH, "AMG: a coarse row couples too many aggregates");
    if (cst & ST_NONPOSITIVE) fail(VAG_EINVAL, "AMG: non-positive coarse diagonal");
    C.col = static_cast<int *>(alloc(4 * (size_t)std::max<int64_t>(C.nnz, 1)));
    C.val = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(C.nnz, 1)));
    k_coarse_compact<<<grid_for(nc, TB), TB, 0, st>>>(nc, tcol, tval, C.rowptr, C.col, C.val);
    note_launches(1);
    VAG_CUDA(cudaFreeAsync(tcol, st));
    VAG_CUDA(cudaFreeAsync(tval, st));
    const int64_t snnz = sell_structure(st, nc, C.rowptr, C.col, &C.slice_ptr, &C.scol, alloc);
    C.sval = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(snnz, 1)));
    C.sell_nnz = snnz;
    sell_fill<double>(st, nc, C.rowptr, C.col, C.val, C.slice_ptr, C.sval);
    C.d_sys_start = static_cast<int *>(alloc(4 * ((size_t)ns + 1)));
    k_coarse_starts<<<grid_for(ns + 1, TB), TB, 0, st>>>(ns, L.d_sys_start, rscan, C.d_sys_start);
    note_launches(1);
    C.sys_start.assign(ns + 1, 0);
    VAG_CUDA(cudaMemcpyAsync(C.sys_start.data(), C.d_sys_start, 4 * (ns + 1), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    A.levels.push_back(C);   // invalidates L
  }
  // work vectors per level (x, b, t)
  for (auto &L : A.levels) {
    L.x = static_cast<double *>(alloc(8 * (size_t)std::max(L.n, 1)));
    L.b = static_cast<double *>(alloc(8 * (size_t)std::max(L.n, 1)));
    L.t = static_cast<double *>(alloc(8 * (size_t)std::max(L.n, 1)));
  }
  // FP32 copy of the hierarchy (the mixed-precision path)
  A.f32 = f32;
  if (f32) {
    auto cast = [&](const double *src, int64_t n) -> float * {
      float *d = static_cast<float *>(alloc(4 * (size_t)std::max<int64_t>(n, 1)));
      if (n > 0 && src) {
        k_to_f32<<<grid_for(n, TB), TB, 0, st>>>(n, src, d);
        note_launches(1);
      }
      return d;
    };
    A.sval32 = static_cast<float *>(alloc(4 * (size_t)std::max<int64_t>(s->sell_nnz, 1)));
    sell_values_f32(s, A.sval32);
    for (size_t l = 0; l < A.levels.size(); ++l) {
      AmgLevel &L = A.levels[l];
      if (l == 0) {
        L.sval32 = A.sval32;
      } else {
        L.sval32 = static_cast<float *>(alloc(4 * (size_t)std::max<int64_t>(L.sell_nnz, 1)));
        sell_fill<float>(st, L.n, L.rowptr, L.col, L.val, L.slice_ptr, L.sval32);
      }
      L.dinv32 = cast(L.dinv, L.n);
      L.inv32 = L.any_term ? cast(L.inv, L.n_inv) : nullptr;
      L.x32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.b32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.t32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
    }
  }
  VAG_CHECK_LAUNCH();
  A.built = true;
}

// Level arrays of one precision.
template <class T>
struct LV {
  const T *val, *dinv, *inv, *sval;
  T *x, *b, *t;
};
template <class T>
static LV<T> lv(System *s, AmgLevel &L);
template <>
LV<double> lv<double>(System *, AmgLevel &L) {
  return {L.val, L.dinv, L.inv, L.sval, L.x, L.b, L.t};
}
template <>
LV<float> lv<float>(System *, AmgLevel &L) {
  return {L.val32, L.dinv32, L.inv32, L.sval32, L.x32, L.b32, L.t32};
}

// x = V(b): one V(2,2) cycle from a zero initial guess.  Systems that end at
// this level are solved exactly; the others are smoothed, restricted,
// corrected from the next level and smoothed again.
template <class T>
static void vcycle(System *s, int lvl, const T *b, T *x, cudaStream_t st) {
  Amg &A = s->amg;
  AmgLevel &L = A.levels[lvl];
  const LV<T> v = lv<T>(s, L);
  const int n = L.n;
  const int g = grid_for(n, TB);
  if (L.any_term) {
    k_dense_apply<T><<<s->seg.n_sys, 64, 0, st>>>(L.d_sys_start, L.inv_off, v.inv, b, x);
    note_launches(1);
  }
  if (L.all_term) return;
  AmgLevel &C = A.levels[lvl + 1];
  const LV<T> c = lv<T>(s, C);
  // pre-smoothing: two damped Jacobi sweeps from x = 0
  k_jac_first<T><<<g, TB, 0, st>>>(n, b, v.dinv, v.t);
  k_jac_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, v.dinv, b, v.t, x, L.skip);
  // residual, restricted to the coarse level (t is free again)
  k_resid_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, b, x, v.t);
  k_restrict<T><<<grid_for(C.n, TB), TB, 0, st>>>(C.n, L.mptr, L.mem, v.t, c.b);
  note_launches(4);
  vcycle<T>(s, lvl + 1, c.b, c.x, st);
  k_prolong<T><<<g, TB, 0, st>>>(n, L.agg, c.x, x);
  // post-smoothing: two sweeps
  k_jac_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, v.dinv, b, x, v.t, L.skip);
  k_jac_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, v.dinv, b, v.t, x, L.skip);
  note_launches(3);
}

void amg_apply(System *s, const double *r, double *z, cudaStream_t st) {
  Amg &A = s->amg;
  if (!A.f32) {
    vcycle<double>(s, 0, r, z, st);
    return;
  }
  AmgLevel &L0 = A.levels[0];
  const int n = L0.n;
  k_to_f32<<<grid_for(n, TB), TB, 0, st>>>(n, r, L0.b32);
  vcycle<float>(s, 0, L0.b32, L0.x32, st);
  k_to_f64<<<grid_for(n, TB), TB, 0, st>>>(n, L0.x32, z);
  note_launches(2);
}

void amg_free(System *s) {
  for (void *p : s->amg.allocs) ctx_free(s->ctx, p);
  if (s->ctx) s->ctx->in_use -= s->amg.bytes;
  s->amg.allocs.clear();
  s->amg.bytes = 0;
  s->amg.levels.clear();
  s->amg.built = false;
}

}  // namespace vag
