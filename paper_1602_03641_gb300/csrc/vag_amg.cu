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
// Smoother: l1-Jacobi, x += omega (b - A x) / sum_j |a_ij| (Baker, Falgout,
// Kolev, Yang, "Multigrid smoothers for ultraparallel computing", SIAM J. Sci.
// Comput. 33 (2011)).  diag(sum_j |a_ij|) - A is diagonally dominant, hence
// A <= D_l1 and the sweep is A-norm convergent for any SPD A and omega < 2; on
// zero-row-sum rows with non-positive couplings D_l1 = 2 a_ii, so omega = 4/3
// equals damped Jacobi with 2/3 there.  Plain damped Jacobi diverges on VAG
// rows where lambda_max(D^-1 A) > 3 (jittered, anisotropic cells), and the
// V-cycle then stops being positive definite.
constexpr double kOmega = 4.0 / 3.0;
constexpr int kDenseMax = 48;       // two 48x48 FP64 blocks fit the static shared limit
constexpr int kMaxLevels = 16;
constexpr int kCoarseWidth = 160;   // unique columns of one coarse row (< 256)
constexpr int kTailRows = 1024;     // FP32 levels at most this big per system run in one kernel

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

__global__ void k_l1_inv(int n, const int *__restrict__ rowptr, const double *__restrict__ val,
                         double *__restrict__ sinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) a += fabs(val[k]);
  sinv[i] = 1.0 / a;
}

// sqrt of each diagonal entry, FP32 (the strength test is a heuristic: FP32
// decides it, deterministically)
__global__ void k_sqrt_diag(int n, const double *__restrict__ dinv, float *__restrict__ sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sd[i] = (float)sqrt(1.0 / dinv[i]);
}

// strength mask per CSR entry and isolated flag per row
__global__ void k_strength(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const double *__restrict__ val, const float *__restrict__ sd,
                           const uint8_t *__restrict__ skip, uint8_t *strong, int8_t *state) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (skip[i]) {   // terminal system: no aggregation at all
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) strong[k] = 0;
    state[i] = -2;
    return;
  }
  const float ti = (float)kTheta * sd[i];
  int cnt = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = col[k];
    const bool st = (j != i) && fabsf((float)val[k]) >= ti * sd[j];
    strong[k] = st;
    cnt += st;
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
                            const double *__restrict__ val, const float *__restrict__ sd,
                            const uint8_t *__restrict__ strong, const int8_t *__restrict__ state,
                            const int *__restrict__ agg1, int *agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0 && state[i] != -2) {
    float best = -1.f;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (!strong[k]) continue;
      const int j = col[k];
      if (agg1[j] < 0) continue;
      const float w = fabsf((float)val[k]) / sd[j];
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
__device__ __forceinline__ T row_sell(int i, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                      const int *__restrict__ scol, const T *__restrict__ sval,
                                      const T *__restrict__ x) {
  const int len = rowptr[i + 1] - rowptr[i];
  const int base = slice_ptr[i >> 5] + (i & 31);
  T s = 0;
#pragma unroll 4
  for (int k = 0; k < len; ++k) {
    const int idx = base + 32 * k;
    s = fma(sval[idx], x[scol[idx]], s);
  }
  return s;
}

// Row product of a coarse level: 8 lanes per CSR row, lane l takes entries
// l, l+8, ... and the partial sums meet in a fixed shuffle tree.  All 32 lanes
// of the warp must call it together (rows past the end pass valid = false).
template <class T>
__device__ __forceinline__ T row_csr8(int i, bool valid, int lane, const int *__restrict__ rowptr,
                                      const int *__restrict__ col, const T *__restrict__ val,
                                      const T *__restrict__ x) {
  T s = 0;
  if (valid)
    for (int k = rowptr[i] + lane; k < rowptr[i + 1]; k += 8) s = fma(val[k], x[col[k]], s);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

template <class T>
__device__ __forceinline__ T jac_first_row(T b, T sinv) { return (T)kOmega * sinv * b; }
template <class T>
__device__ __forceinline__ T jac_row(T xin, T sinv, T b, T ax) { return fma((T)kOmega * sinv, b - ax, xin); }

template <class T>
__global__ void k_jac_first(int n, const T *__restrict__ b, const T *__restrict__ sinv, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = jac_first_row(b[i], sinv[i]);
}

// x_out = x_in + omega D^-1 (b - A x_in), CSR, one thread per row
template <class T>
__global__ void k_jac_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                          const T *__restrict__ val, const T *__restrict__ sinv, const T *__restrict__ b,
                          const T *__restrict__ xin, T *__restrict__ xout, const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || skip[i]) return;
  T s = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], xin[col[k]], s);
  xout[i] = jac_row(xin[i], sinv[i], b[i], s);
}

// coarse-level sweep and residual, 8 lanes per row (32 rows per block)
template <class T>
__global__ void __launch_bounds__(256) k_jac_csr8(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                                  const T *__restrict__ val, const T *__restrict__ sinv,
                                                  const T *__restrict__ b, const T *__restrict__ xin,
                                                  T *__restrict__ xout, const uint8_t *__restrict__ skip) {
  const int lane = threadIdx.x & 7;
  const int i = blockIdx.x * 32 + (threadIdx.x >> 3);
  const bool valid = i < n;
  const T s = row_csr8(i, valid, lane, rowptr, col, val, xin);
  if (valid && lane == 0 && !skip[i]) xout[i] = jac_row(xin[i], sinv[i], b[i], s);
}

template <class T>
__global__ void __launch_bounds__(256) k_resid_csr8(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                                    const T *__restrict__ val, const T *__restrict__ b,
                                                    const T *__restrict__ x, T *__restrict__ r) {
  const int lane = threadIdx.x & 7;
  const int i = blockIdx.x * 32 + (threadIdx.x >> 3);
  const bool valid = i < n;
  const T s = row_csr8(i, valid, lane, rowptr, col, val, x);
  if (valid && lane == 0) r[i] = b[i] - s;
}

// same sweep in the sliced-ELL layout
template <class T>
__global__ void k_jac_sell(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                           const int *__restrict__ scol, const T *__restrict__ sval, const T *__restrict__ sinv,
                           const T *__restrict__ b, const T *__restrict__ xin, T *__restrict__ xout,
                           const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || skip[i]) return;
  xout[i] = jac_row(xin[i], sinv[i], b[i], row_sell(i, rowptr, slice_ptr, scol, sval, xin));
}

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
  r[i] = b[i] - row_sell(i, rowptr, slice_ptr, scol, sval, x);
}

// b_c[I] = sum of r over the members of aggregate I (row order)
template <class T>
__device__ __forceinline__ T restrict_row(int I, const int *__restrict__ mptr, const int *__restrict__ mem,
                                          const T *__restrict__ r) {
  T acc = 0;
  for (int p = mptr[I]; p < mptr[I + 1]; ++p) acc += r[mem[p]];
  return acc;
}

template <class T>
__global__ void k_restrict(int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                           const T *__restrict__ r, T *__restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  bc[I] = restrict_row(I, mptr, mem, r);
}

template <class T>
__global__ void k_prolong(int n, const int *__restrict__ agg, const T *__restrict__ xc, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) x[i] += xc[agg[i]];
}

// x = inv_g b per system block (one thread block per system)
template <class T>
__device__ __forceinline__ T dense_row(int i, int m, const T *__restrict__ M, const T *__restrict__ b) {
  T s = 0;
  for (int j = 0; j < m; ++j) s = fma(M[i * m + j], b[j], s);
  return s;
}

template <class T>
__global__ void k_dense_apply(const int *__restrict__ sys_start, const long long *__restrict__ off,
                              const T *__restrict__ inv, const T *__restrict__ b, T *x) {
  const int g = blockIdx.x;
  const int r0 = sys_start[g], m = sys_start[g + 1] - r0;
  if (m == 0 || off[g + 1] - off[g] != (long long)m * m) return;   // not terminal here
  const T *M = inv + off[g];
  for (int i = threadIdx.x; i < m; i += blockDim.x) x[r0 + i] = dense_row(i, m, M, b + r0);
}

// The lower part of the FP32 V-cycle (levels with at most kTailRows rows per
// system) in one kernel: one thread block per system walks its levels down
// and up with a barrier between phases.  Same row arithmetic as the grid
// kernels, so the result is identical to launching them level by level.
constexpr int kTailLevels = 10;
struct TailLevel {
  const int *sys_start, *rowptr, *col, *agg, *mptr, *mem;
  const float *val, *sinv, *inv;
  const long long *inv_off;
  float *x, *b, *t;
};
struct TailDesc {
  TailLevel lv[kTailLevels];
  int nlev;
};

__global__ void __launch_bounds__(1024) k_vcycle_tail32(TailDesc d) {
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 7, grp = threadIdx.x >> 3;   // 128 groups of 8 lanes
  int last = d.nlev - 1;   // deepest level with a coarse correction below it
  // one op per row over [r0, r0+m), 8 lanes per row, uniform loop bound
  auto rows8 = [&](const TailLevel &L, int r0, int m, const float *x, auto &&emit) {
    for (int base = 0; base < m; base += 128) {
      const int i = r0 + base + grp;
      const bool valid = base + grp < m;
      const float s = row_csr8(i, valid, lane, L.rowptr, L.col, L.val, x);
      if (valid && lane == 0) emit(i, s);
    }
  };
  for (int l = 0; l < d.nlev; ++l) {
    const TailLevel &L = d.lv[l];
    const int r0 = L.sys_start[g], m = L.sys_start[g + 1] - r0;
    if (m == 0) { last = l - 1; break; }
    if (L.inv_off && L.inv_off[g + 1] - L.inv_off[g] == (long long)m * m) {   // terminal here
      const float *M = L.inv + L.inv_off[g];
      for (int i = threadIdx.x; i < m; i += blockDim.x) L.x[r0 + i] = dense_row(i, m, M, L.b + r0);
      __syncthreads();
      last = l - 1;
      break;
    }
    for (int i = r0 + threadIdx.x; i < r0 + m; i += blockDim.x) L.t[i] = jac_first_row(L.b[i], L.sinv[i]);
    __syncthreads();
    rows8(L, r0, m, L.t, [&](int i, float s) { L.x[i] = jac_row(L.t[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
    rows8(L, r0, m, L.x, [&](int i, float s) { L.t[i] = L.b[i] - s; });
    __syncthreads();
    if (l + 1 < d.nlev) {
      const TailLevel &C = d.lv[l + 1];
      for (int I = C.sys_start[g] + threadIdx.x; I < C.sys_start[g + 1]; I += blockDim.x)
        C.b[I] = restrict_row(I, L.mptr, L.mem, L.t);
    }
    __syncthreads();
  }
  for (int l = last; l >= 0; --l) {
    const TailLevel &L = d.lv[l];
    const int r0 = L.sys_start[g], m = L.sys_start[g + 1] - r0;
    if (l + 1 < d.nlev) {
      const float *xc = d.lv[l + 1].x;
      for (int i = r0 + threadIdx.x; i < r0 + m; i += blockDim.x)
        if (L.agg[i] >= 0) L.x[i] += xc[L.agg[i]];
    }
    __syncthreads();
    rows8(L, r0, m, L.x, [&](int i, float s) { L.t[i] = jac_row(L.x[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
    rows8(L, r0, m, L.t, [&](int i, float s) { L.x[i] = jac_row(L.t[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
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
    float *sd = static_cast<float *>(alloc(4 * (size_t)std::max(n, 1)));
    k_sqrt_diag<<<grid_for(n, TB), TB, 0, st>>>(n, L.dinv, sd);
    k_strength<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, L.val, sd, L.skip, strong, state);
    note_launches(2);
    // MIS(2) rounds, three between polls (a round after the last decision
    // changes nothing)
    for (int it = 0; it < 64; it += 3) {
      for (int r = 0; r < 3; ++r) {
        VAG_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int), st));
        k_mis_max1<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, L.d_sys_start, ns, m1);
        k_mis_max2_decide<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, m1, L.d_sys_start,
                                                           ns, next, undecided);
        note_launches(2);
        VAG_CUDA(cudaMemcpyAsync(state, next, n, cudaMemcpyDeviceToDevice, st));
      }
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
    k_agg_pass2<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, L.val, sd, strong, state, agg1, L.agg);
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
  // work vectors per level (x, b, t) and the l1 smoother scaling
  for (auto &L : A.levels) {
    L.sinv = static_cast<double *>(alloc(8 * (size_t)std::max(L.n, 1)));
    if (L.n > 0) {
      k_l1_inv<<<grid_for(L.n, TB), TB, 0, st>>>(L.n, L.rowptr, L.val, L.sinv);
      note_launches(1);
    }
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
        L.val32 = cast(L.val, L.nnz);
      }
      L.sinv32 = cast(L.sinv, L.n);
      L.inv32 = L.any_term ? cast(L.inv, L.n_inv) : nullptr;
      L.x32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.b32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.t32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
    }
  }
  // first level where every system has at most kTailRows rows: from there
  // the FP32 V-cycle runs in one kernel
  A.tail_start = -1;
  if (f32) {
    for (size_t l = 1; l < A.levels.size(); ++l) {
      int mx = 0;
      for (int g = 0; g < ns; ++g) mx = std::max(mx, A.levels[l].sys_start[g + 1] - A.levels[l].sys_start[g]);
      if (mx <= kTailRows && (int)(A.levels.size() - l) <= kTailLevels) {
        A.tail_start = (int)l;
        break;
      }
    }
  }
  VAG_CHECK_LAUNCH();
  A.built = true;
}

// Level arrays of one precision.
template <class T>
struct LV {
  const T *val, *sinv, *inv, *sval;
  T *x, *b, *t;
};
template <class T>
static LV<T> lv(System *s, AmgLevel &L);
template <>
LV<double> lv<double>(System *, AmgLevel &L) {
  return {L.val, L.sinv, L.inv, L.sval, L.x, L.b, L.t};
}
template <>
LV<float> lv<float>(System *, AmgLevel &L) {
  return {L.val32, L.sinv32, L.inv32, L.sval32, L.x32, L.b32, L.t32};
}   // val32 on coarse levels, sval32 on level 0

// x = V(b): one V(2,2) cycle from a zero initial guess.  Systems that end at
// this level are solved exactly; the others are smoothed, restricted,
// corrected from the next level and smoothed again.
static void tail32(System *s, int lvl, cudaStream_t st) {
  Amg &A = s->amg;
  TailDesc d{};
  d.nlev = (int)A.levels.size() - lvl;
  if (d.nlev > kTailLevels) fail(VAG_ECUDA, "AMG: too many levels below the tail start");
  for (int k = 0; k < d.nlev; ++k) {
    AmgLevel &L = A.levels[lvl + k];
    d.lv[k] = TailLevel{L.d_sys_start, L.rowptr, L.col, L.agg, L.mptr, L.mem, L.val32, L.sinv32,
                        L.inv32, L.any_term ? L.inv_off : nullptr, L.x32, L.b32, L.t32};
  }
  k_vcycle_tail32<<<s->seg.n_sys, 1024, 0, st>>>(d);
  note_launches(1);
}

template <class T>
static void vcycle(System *s, int lvl, const T *b, T *x, cudaStream_t st) {
  Amg &A = s->amg;
  AmgLevel &L = A.levels[lvl];
  if (sizeof(T) == 4 && lvl > 0 && lvl == A.tail_start) {   // b, x are this level's b32, x32
    tail32(s, lvl, st);
    return;
  }
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
  // level 0: sliced ELL, one thread per row; coarser levels: CSR, 8 lanes per row
  const int g8 = grid_for(n, 32);
  auto sweep = [&](const T *xin, T *xout) {
    if (lvl == 0)
      k_jac_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, v.sinv, b, xin, xout, L.skip);
    else
      k_jac_csr8<T><<<g8, 256, 0, st>>>(n, L.rowptr, L.col, v.val, v.sinv, b, xin, xout, L.skip);
  };
  // pre-smoothing: two damped Jacobi sweeps from x = 0
  k_jac_first<T><<<g, TB, 0, st>>>(n, b, v.sinv, v.t);
  sweep(v.t, x);
  // residual, restricted to the coarse level (t is free again)
  if (lvl == 0)
    k_resid_sell<T><<<g, TB, 0, st>>>(n, L.rowptr, L.slice_ptr, L.scol, v.sval, b, x, v.t);
  else
    k_resid_csr8<T><<<g8, 256, 0, st>>>(n, L.rowptr, L.col, v.val, b, x, v.t);
  k_restrict<T><<<grid_for(C.n, TB), TB, 0, st>>>(C.n, L.mptr, L.mem, v.t, c.b);
  note_launches(4);
  vcycle<T>(s, lvl + 1, c.b, c.x, st);
  k_prolong<T><<<g, TB, 0, st>>>(n, L.agg, c.x, x);
  // post-smoothing: two sweeps
  sweep(x, v.t);
  sweep(v.t, x);
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
