// Aggregation algebraic multigrid preconditioner for the eliminated VAG
// system (the paper's §5 compares Trilinos aggregation AMG and Hypre's
// classical AMG as GMRES/BiCGStab preconditioners; this is the library's own
// aggregation AMG, used inside CG or BiCGStab).
//
// Setup, level by level, all on the device:
//  strength   j is a strong neighbour of i if |a_ij| >= theta sqrt(a_ii a_jj)
//             (theta per level and system, see kTheta);
//  MIS(2)     roots: undecided nodes whose key is the largest within two
//             strong hops (keys hash the system-local row index, so a system's
//             hierarchy does not depend on the rest of a batch); nodes within
//             two hops of a root drop out; repeat until no node is undecided;
//  aggregates a root and its strong neighbours, then every remaining node
//             joins the aggregate of its strongest aggregated neighbour; nodes
//             without a strong neighbour stay out of the coarse space;
//  Galerkin   A_c = P^T A P for the piecewise-constant P, one warp per
//             coarse row summing its members' rows in row order (entries of a
//             coarse column added in that order; columns sorted);
//  terminal   a system whose level has at most kDenseMax rows leaves the
//             hierarchy there: its block is inverted densely (Gauss-Jordan,
//             SPD) and applied exactly in the cycle.  The depth of a system's
//             hierarchy therefore depends on that system alone.
// Apply: a V-cycle with l1-Jacobi sweeps before and after the coarse
// correction, one each on the finest level and two each on the coarse levels
// (V(1,1) / V(2,2)); as many sweeps after as before on every level, so it is
// a fixed symmetric linear operator, as CG needs.  FP64, or
// on an FP32 copy of the hierarchy (VAG_MIXED; VAG_MIXED_F16 also keeps the
// finest level in FP16 after symmetric diagonal scaling).
#include <climits>
#include <cstdio>

#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace vag {
namespace {

constexpr int TB = 256;
// Strength threshold: 0.08; 0.02 on a coarse level (not the finest) where the
// system has at most kSmallLevel rows, where coarsening faster costs few iterations and every
// level saved is four latency-bound launches per V-cycle (measured: 64^3,
// 73 -> 70 iterations and one level less; applied to large levels too, the
// 128^3 DFN needed 10-20 % more iterations).  Per system, so a system's
// hierarchy does not depend on its batch.
constexpr double kTheta = 0.08;
constexpr double kThetaCoarse = 0.02;
constexpr int kSmallLevel = 50000;
// Smoother: l1-Jacobi, x += omega (b - A x) / sum_j |a_ij| (Baker, Falgout,
// Kolev, Yang, "Multigrid smoothers for ultraparallel computing", SIAM J. Sci.
// Comput. 33 (2011)).  diag(sum_j |a_ij|) - A is diagonally dominant, hence
// A <= D_l1 and the sweep is A-norm convergent for any SPD A and omega < 2; on
// zero-row-sum rows with non-positive couplings D_l1 = 2 a_ii, so omega = 4/3
// equals damped Jacobi with 2/3 there.  Plain damped Jacobi diverges on VAG
// rows where lambda_max(D^-1 A) > 3 (jittered, anisotropic cells), and the
// V-cycle then stops being positive definite.
constexpr double kOmega = 4.0 / 3.0;
// A system whose level has at most kDenseMax rows is solved there with a dense
// inverse (an inversion of at most about 0.2 ms on one SM at setup, against
// four latency-bound launches per V-cycle for every level it saves)
constexpr int kDenseMax = 96;
constexpr size_t kDenseSmem = 2 * sizeof(double) * kDenseMax * kDenseMax;   // [A | B] in dynamic shared memory
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
                           const uint8_t *__restrict__ skip, uint8_t *strong, int8_t *state,
                           const int *__restrict__ sys_start, int n_sys, int coarse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (skip[i]) {   // terminal system: no aggregation at all
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) strong[k] = 0;
    state[i] = -2;
    return;
  }
  const int g = sys_of_row(i, sys_start, n_sys);
  const float theta = (float)(coarse && sys_start[g + 1] - sys_start[g] <= kSmallLevel ? kThetaCoarse : kTheta);
  const float ti = theta * sd[i];
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
                           const int *__restrict__ sys_start, int n_sys, unsigned long long *m1, int *undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *undecided = 0;   // counted by this round's k_mis_max2_decide
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

// One coarse row of A_c = P^T A P per warp.  The entries of the members'
// rows (members in row order, entries in CSR order: the sequence p) are read
// 32 at a time; each entry finds its coarse column's slot in the warp's
// shared-memory hash table, lanes that hit the same slot are grouped
// (__match_any_sync) and the lowest of them adds their values to the slot in
// lane order.  Every coarse entry is therefore the sum of its contributions
// in sequence order, whatever the scheduling; the row is emitted sorted by
// coarse column.
constexpr int kHash = 256;
constexpr int kBuildWarps = 8;
__global__ void __launch_bounds__(32 * kBuildWarps) k_coarse_build(int nc, const int *__restrict__ mptr,
                                                                   const int *__restrict__ mem,
                                                                   const int *__restrict__ rowptr,
                                                                   const int *__restrict__ col,
                                                                   const double *__restrict__ val,
                                                                   const int *__restrict__ agg, int *tcol,
                                                                   double *tval, int *cnt, double *cdinv,
                                                                   int *status) {
  __shared__ int keys[kBuildWarps][kHash];
  __shared__ double sums[kBuildWarps][kHash];
  __shared__ double vals[kBuildWarps][32];
  __shared__ int nuniq[kBuildWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x * kBuildWarps + w;
  if (I >= nc) return;   // whole warps leave together
  int *K = keys[w];
  double *S = sums[w];
  for (int h = lane; h < kHash; h += 32) {
    K[h] = -1;
    S[h] = 0.0;
  }
  if (lane == 0) nuniq[w] = 0;
  __syncwarp();
  bool overflow = false;
  for (int p = mptr[I]; p < mptr[I + 1]; ++p) {
    const int i = mem[p];
    const int kb = rowptr[i], ke = rowptr[i + 1];
    for (int c = kb; c < ke; c += 32) {
      const int k = c + lane;
      const int J = k < ke ? agg[col[k]] : -1;
      const double v = k < ke ? val[k] : 0.0;
      int slot = -1;
      if (J >= 0) {
        unsigned h = ((unsigned)J * 2654435761u) & (kHash - 1);
        for (int probe = 0; probe < kHash; ++probe, h = (h + 1) & (kHash - 1)) {
          const int cur = ((volatile int *)K)[h];
          if (cur == J) { slot = (int)h; break; }
          if (cur == -1) {
            const int old = atomicCAS(&K[h], -1, J);
            if (old == -1) { atomicAdd(&nuniq[w], 1); slot = (int)h; break; }
            if (old == J) { slot = (int)h; break; }
          }
        }
        if (slot < 0) overflow = true;
      }
      vals[w][lane] = v;
      __syncwarp();
      const unsigned grp = __match_any_sync(0xffffffffu, slot >= 0 ? slot : -1 - lane);
      if (slot >= 0 && lane == __ffs(grp) - 1) {
        double acc = S[slot];
        for (unsigned m = grp; m; m &= m - 1) acc += vals[w][__ffs(m) - 1];
        S[slot] = acc;
      }
      __syncwarp();
    }
  }
  const int nu = nuniq[w];
  if (__any_sync(0xffffffffu, overflow) || nu > kCoarseWidth) {
    if (lane == 0) {
      atomicOr(status, ST_ROW_OVERFLOW);
      cnt[I] = 0;
    }
    return;
  }
  // the distinct columns in ascending order: compact the (column, sum) pairs
  // to the front of the table in place (a pair only moves left, past pairs
  // already read), pad to a power of two and sort them (bitonic, by column)
  int pos = 0;
  for (int h0 = 0; h0 < kHash; h0 += 32) {
    const int key = K[h0 + lane];
    const double sum = S[h0 + lane];
    const unsigned b = __ballot_sync(0xffffffffu, key >= 0);
    __syncwarp();
    if (key >= 0) {
      const int q = pos + __popc(b & ((1u << lane) - 1u));
      K[q] = key;
      S[q] = sum;
    }
    pos += __popc(b);
    __syncwarp();
  }
  int n2 = 32;
  while (n2 < nu) n2 <<= 1;
  for (int q = nu + lane; q < n2; q += 32) K[q] = INT_MAX;
  __syncwarp();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = lane; q < n2; q += 32) {
        const int o = q ^ stride;
        if (o > q) {
          const bool up = (q & size) == 0;
          const int a = K[q], b = K[o];
          if ((a > b) == up) {
            K[q] = b; K[o] = a;
            const double t = S[q]; S[q] = S[o]; S[o] = t;
          }
        }
      }
      __syncwarp();
    }
  }
  const size_t base = (size_t)I * kCoarseWidth;
  bool diag = false;
  for (int q = lane; q < nu; q += 32) {
    tcol[base + q] = K[q];
    tval[base + q] = S[q];
    if (K[q] == I) {
      diag = true;
      if (!(S[q] > 0.0)) atomicOr(status, ST_NONPOSITIVE);
      cdinv[I] = 1.0 / S[q];
    }
  }
  if (!__any_sync(0xffffffffu, diag) && lane == 0) {
    atomicOr(status, ST_NONPOSITIVE);
    cdinv[I] = 1.0 / 0.0;
  }
  if (lane == 0) cnt[I] = nu;
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

// first nonzero of each system's rows: rowptr[sys_start[g]]
__global__ void k_nz_starts(int n_sys, const int *__restrict__ sys_start, const int *__restrict__ rowptr,
                            int *__restrict__ nz_start) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g <= n_sys) nz_start[g] = rowptr[sys_start[g]];
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
  extern __shared__ double dense_sm[];   // kDenseSmem bytes
  const int g = blockIdx.x;
  const int r0 = sys_start[g], m = sys_start[g + 1] - r0;
  if (m == 0 || m > kDenseMax || off[g + 1] - off[g] != (long long)m * m) return;   // not terminal here
  double *A = dense_sm, *B = dense_sm + m * m;
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
    // Before pivot p, row p of A is zero left of p and column j > p of B is
    // still e_j, so only A's columns > p and B's columns <= p change: m
    // entries a row instead of 2m - 1 (the skipped updates subtract zeros)
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      if (j > p) A[p * m + j] /= piv;
      else B[p * m + j] /= piv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (m - 1) * m; e += blockDim.x) {
      const int ii = e / m, jj = e % m;
      const int i = ii < p ? ii : ii + 1;
      const double f = A[i * m + p];
      if (jj < m - 1 - p) {
        const int j = p + 1 + jj;
        A[i * m + j] -= f * A[p * m + j];
      } else {
        const int j = jj - (m - 1 - p);
        B[i * m + j] -= f * B[p * m + j];
      }
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


// Row product of a coarse level: LN lanes per CSR row, lane l takes entries
// l, l+LN, ... and the partial sums meet in a fixed shuffle tree.  All 32
// lanes of the warp must call it together (rows past the end pass valid =
// false).  Coarse levels are latency-bound: 8 lanes per row keep each lane's
// chain of dependent loads short (measured on GB300: 2 lanes per row, which
// halves the FP64 instructions, made the FP64 sweeps 1.6x slower).
template <class T>
__host__ __device__ constexpr int row_lanes() { return 8; }

template <int LN, class T>
__device__ __forceinline__ T lane_reduce(T s) {
#pragma unroll
  for (int o = LN / 2; o >= 1; o /= 2) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <int LN, class T>
__device__ __forceinline__ T row_csr(int i, bool valid, int lane, const int *__restrict__ rowptr,
                                     const int *__restrict__ col, const T *__restrict__ val,
                                     const T *__restrict__ x) {
  T s = 0;
  if (valid)
    for (int k = rowptr[i] + lane; k < rowptr[i + 1]; k += LN) s = fma(val[k], x[col[k]], s);
  return lane_reduce<LN>(s);
}

// The same row product split in two for programmatic dependent launch: the
// first pf<T>() entries of each lane (matrix data, written by no kernel of the
// cycle) are loaded before pdl_wait(), the x gathers after it.  Entries are
// multiplied in the same order as row_csr, so the sum is identical.  FP32
// rows take six entries a lane (48 of the classical coarse levels' 40-46
// entries a row in flight at once; four and eight were measured slower),
// FP64 rows four.
template <class T>
__host__ __device__ constexpr int pf() { return sizeof(T) == 4 ? 6 : 4; }
template <class T>
struct RowPF {
  int k, ke;
  int c[pf<T>()];
  T v[pf<T>()];
};
template <int LN, class T>
__device__ __forceinline__ void row_prefetch(RowPF<T> &f, int i, bool valid, int lane, const int *__restrict__ rowptr,
                                             const int *__restrict__ col, const T *__restrict__ val) {
  f.k = valid ? rowptr[i] + lane : 0;
  f.ke = valid ? rowptr[i + 1] : 0;
#pragma unroll
  for (int u = 0; u < pf<T>(); ++u) {
    const int k = f.k + LN * u;
    f.c[u] = k < f.ke ? col[k] : 0;
    f.v[u] = k < f.ke ? val[k] : (T)0;
  }
}
template <int LN, class T>
__device__ __forceinline__ T row_finish(const RowPF<T> &f, const int *__restrict__ col, const T *__restrict__ val,
                                        const T *__restrict__ x) {
  T s = 0;
#pragma unroll
  for (int u = 0; u < pf<T>(); ++u)
    if (f.k + LN * u < f.ke) s = fma(f.v[u], x[f.c[u]], s);
  for (int k = f.k + LN * pf<T>(); k < f.ke; k += LN) s = fma(val[k], x[col[k]], s);
  return lane_reduce<LN>(s);
}

template <class T>
__device__ __forceinline__ T jac_first_row(T b, T sinv) { return (T)kOmega * sinv * b; }
template <class T>
__device__ __forceinline__ T jac_row(T xin, T sinv, T b, T ax) { return fma((T)kOmega * sinv, b - ax, xin); }

template <class T>
__global__ void k_jac_first(int n, const T *__restrict__ b, const T *__restrict__ sinv, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i < n) x[i] = jac_first_row(b[i], sinv[i]);
}

// r = b - A x on a coarse level, row_lanes<T>() lanes per row (used with the
// restriction as a separate kernel where aggregates are large: the fused
// kernel walks an aggregate's members four at a time)
template <class T>
__global__ void __launch_bounds__(256) k_resid_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                                   const T *__restrict__ val, const T *__restrict__ b,
                                                   const T *__restrict__ x, T *__restrict__ r) {
  constexpr int LN = row_lanes<T>();
  const int lane = threadIdx.x & (LN - 1);
  const int i = blockIdx.x * (256 / LN) + threadIdx.x / LN;
  const bool valid = i < n;
  RowPF<T> f;
  row_prefetch<LN>(f, i, valid, lane, rowptr, col, val);
  pdl_wait();
  pdl_trigger();
  const T bi = valid && lane == 0 ? b[i] : (T)0;   // in flight with the gathers
  const T s = row_finish<LN>(f, col, val, x);
  if (valid && lane == 0) r[i] = bi - s;
}

// x_out = x_in + omega D_l1^-1 (b - A x_in) on a coarse level, row_lanes<T>()
// lanes per row (256 / LN rows per block); rows of systems solved densely here
// are skipped
template <class T>
__global__ void __launch_bounds__(256) k_jac_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                                 const T *__restrict__ val, const T *__restrict__ sinv,
                                                 const T *__restrict__ b, const T *__restrict__ xin,
                                                 T *__restrict__ xout, const uint8_t *__restrict__ skip) {
  constexpr int LN = row_lanes<T>();
  const int lane = threadIdx.x & (LN - 1);
  const int i = blockIdx.x * (256 / LN) + threadIdx.x / LN;
  const bool valid = i < n;
  RowPF<T> f;
  row_prefetch<LN>(f, i, valid, lane, rowptr, col, val);
  const bool own = valid && lane == 0 && !skip[i];
  const T si = own ? sinv[i] : (T)0;
  pdl_wait();
  pdl_trigger();
  const T bi = own ? b[i] : (T)0, xi = own ? xin[i] : (T)0;   // in flight with the gathers
  const T s = row_finish<LN>(f, col, val, xin);
  if (own) xout[i] = jac_row(xi, si, bi, s);
}

// same sweep in the sliced-ELL layout (level 0), one thread per row
template <class T, int U>
__global__ void k_jac_sell(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                           const int *__restrict__ scol, const T *__restrict__ sval, const T *__restrict__ sinv,
                           const T *__restrict__ b, const T *__restrict__ xin, T *__restrict__ xout,
                           const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i >= n || skip[i]) return;
  xout[i] = jac_row(xin[i], sinv[i], b[i], sell_row<T, U>(i, rowptr, slice_ptr, scol, sval, xin));
}

template <class T, int U>
__global__ void k_resid_sell(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                             const int *__restrict__ scol, const T *__restrict__ sval, const T *__restrict__ b,
                             const T *__restrict__ x, T *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i >= n) return;
  r[i] = b[i] - sell_row<T, U>(i, rowptr, slice_ptr, scol, sval, x);
}

// The last finest-level sweep of the V-cycle inside CG (FP64 CG, or the FP32
// CG inside refinement): z = the sweep, and r.z per system formed on the way
// (r is the level's right-hand side), exactly as the separate r.z kernel
// would: one row per thread of a 256-row tile, the tile's block sum, the last
// tile of a system adding the tile partials in order and setting
// beta = (r.z)' / (r.z) and rho = (r.z)'.
template <class T, int U>
__global__ void __launch_bounds__(256) k_jac_sell_rz(const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                                     const int *__restrict__ scol, const T *__restrict__ sval,
                                                     const T *__restrict__ sinv, const T *__restrict__ r,
                                                     const T *__restrict__ xin, T *__restrict__ z,
                                                     const uint8_t *__restrict__ skip, Tiles tl, double *partials,
                                                     unsigned *counter, KrylovScalars *ks, int *n_done) {
  const int t = blockIdx.x;
  const int sys = tl.sys[t];
  const int i = tl.row0[t] + threadIdx.x;
  const bool valid = i < tl.row1[t];
  pdl_wait();
  pdl_trigger();
  double rz = 0.0;
  if (valid) {
    T zi;
    if (skip[i]) {
      zi = z[i];   // solved densely on this level
    } else {
      zi = jac_row(xin[i], sinv[i], r[i], sell_row<T, U>(i, rowptr, slice_ptr, scol, sval, xin));
      z[i] = zi;
    }
    rz = (double)fma(r[i], zi, (T)0);
  }
  if (ks[sys].done) return;   // uniform in the block: one system per tile
  double v[1] = {rz}, out[1];
  if (seg_sum<256, 1>(v, partials, counter, tl, t, sys, out) && threadIdx.x == 0) {
    KrylovScalars &k = ks[sys];
    k.beta = out[0] / k.rz;
    k.rz = out[0];
    if (!(out[0] > 0.0)) { k.breakdown = 1; k.done = 1; atomicAdd(n_done, 1); }
  }
}

// b_c[I] = sum of r over the members of aggregate I (row order)
template <class T>
__device__ __forceinline__ T restrict_row(int I, const int *__restrict__ mptr, const int *__restrict__ mem,
                                          const T *__restrict__ r) {
  T acc = 0;
  for (int p = mptr[I]; p < mptr[I + 1]; ++p) acc += r[mem[p]];
  return acc;
}


// classical levels: bc = R r and the coarse level's zero-start sweep tc =
// omega D_l1^-1 bc, row_lanes<T>() lanes per coarse row
template <class T>
__global__ void __launch_bounds__(256) k_rs_restrict(int nc, const int *__restrict__ rrow, const int *__restrict__ rcol,
                                                     const T *__restrict__ rval, const T *__restrict__ r,
                                                     const T *__restrict__ sinv_c, T *__restrict__ bc,
                                                     T *__restrict__ tc) {
  constexpr int LN = row_lanes<T>();
  const int lane = threadIdx.x & (LN - 1);
  const int I = blockIdx.x * (256 / LN) + threadIdx.x / LN;
  const bool valid = I < nc;
  RowPF<T> f;
  row_prefetch<LN>(f, I, valid, lane, rrow, rcol, rval);
  const T si = valid ? sinv_c[I] : (T)0;
  pdl_wait();
  pdl_trigger();
  const T s = row_finish<LN>(f, rcol, rval, r);
  if (valid && lane == 0) {
    bc[I] = s;
    tc[I] = jac_first_row(s, si);
  }
}

// classical levels: x += P xc, one thread per fine row (at most four entries)
template <class T>
__global__ void k_rs_prolong(int n, const int *__restrict__ prow, const int *__restrict__ pcol,
                             const T *__restrict__ pval, const T *__restrict__ xc, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = i < n ? prow[i] : 0, e = i < n ? prow[i + 1] : 0;
  pdl_wait();
  pdl_trigger();
  if (i >= n || b == e) return;
  T s = 0;
  for (int k = b; k < e; ++k) s = fma(pval[k], xc[pcol[k]], s);
  x[i] += s;
}

template <class T>
__global__ void k_prolong(int n, const int *__restrict__ agg, const T *__restrict__ xc, T *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = i < n ? agg[i] : -1;
  pdl_wait();
  pdl_trigger();
  if (J >= 0) x[i] += xc[J];
}

// Restriction fused with the first (zero-start) sweep of the coarse level:
// bc = P^T r, tc = omega D_l1^-1 bc.
template <class T>
__global__ void k_restrict_first(int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                                 const T *__restrict__ r, const T *__restrict__ sinv_c, T *__restrict__ bc,
                                 T *__restrict__ tc) {
  // the aggregate's first members and the scaling (written by no kernel of
  // the cycle) before the dependency wait; the sum keeps the member order
  constexpr int PF = 12;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int p0 = I < nc ? mptr[I] : 0, p1 = I < nc ? mptr[I + 1] : 0;
  int m[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) m[u] = p0 + u < p1 ? mem[p0 + u] : 0;
  const T si = I < nc ? sinv_c[I] : (T)0;
  pdl_wait();
  pdl_trigger();
  if (I >= nc) return;
  T v = 0;
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (p0 + u < p1) v += r[m[u]];
  for (int p = p0 + PF; p < p1; ++p) v += r[mem[p]];
  bc[I] = v;
  tc[I] = jac_first_row(v, si);
}

// Residual of a coarse level, restricted and turned into the next level's
// first sweep, in one pass: one warp per coarse row I, its member rows taken
// four at a time (8 lanes each); lane 0 adds the member residuals in member
// order, exactly as restrict_row does with a stored residual.
template <class T>
__global__ void __launch_bounds__(256) k_resid_restrict8(int nc, const int *__restrict__ mptr,
                                                         const int *__restrict__ mem, const int *__restrict__ rowptr,
                                                         const int *__restrict__ col, const T *__restrict__ val,
                                                         const T *__restrict__ b, const T *__restrict__ x,
                                                         const T *__restrict__ sinv_c, T *__restrict__ bc,
                                                         T *__restrict__ tc) {
  const int I = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int wl = threadIdx.x & 31, grp = wl >> 3, lane = wl & 7;
  // first member chunk's matrix rows before the dependency wait
  const int p0 = I < nc ? mptr[I] : 0, p1 = I < nc ? mptr[I + 1] : 0;
  RowPF<T> f;
  {
    const bool valid = p0 + grp < p1;
    row_prefetch<8>(f, valid ? mem[p0 + grp] : 0, valid, lane, rowptr, col, val);
  }
  pdl_wait();
  pdl_trigger();
  if (I >= nc) return;   // whole warps leave together
  T acc = 0;
  for (int base = p0; base < p1; base += 4) {
    const bool valid = base + grp < p1;
    const int i = valid ? mem[base + grp] : 0;
    const T s = base == p0 ? row_finish<8>(f, col, val, x) : row_csr<8>(i, valid, lane, rowptr, col, val, x);
    const T r = valid ? b[i] - s : (T)0;
    const int cnt = min(4, p1 - base);
    for (int q = 0; q < cnt; ++q) {
      const T rq = __shfl_sync(0xffffffffu, r, 8 * q);
      acc += rq;
    }
  }
  if (wl == 0) {
    bc[I] = acc;
    tc[I] = jac_first_row(acc, sinv_c[I]);
  }
}

// Prolongation fused with the first post-smoothing sweep of a coarse level:
// the corrected iterate x + P xc is formed on the fly for every entry read,
// t = (x + P xc) + omega D_l1^-1 (b - A (x + P xc)).
template <class T>
__global__ void __launch_bounds__(256) k_prolong_jac8(int n, const int *__restrict__ rowptr,
                                                      const int *__restrict__ col, const T *__restrict__ val,
                                                      const T *__restrict__ sinv, const T *__restrict__ b,
                                                      const T *__restrict__ x, const int *__restrict__ agg,
                                                      const T *__restrict__ xc, T *__restrict__ t,
                                                      const uint8_t *__restrict__ skip) {
  const int lane = threadIdx.x & 7;
  const int i = blockIdx.x * 32 + (threadIdx.x >> 3);
  const bool valid = i < n;
  RowPF<T> f;
  row_prefetch<8>(f, i, valid, lane, rowptr, col, val);
  constexpr int PF = pf<T>();
  int fa[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) fa[u] = f.k + 8 * u < f.ke ? agg[f.c[u]] : -1;
  pdl_wait();
  pdl_trigger();
  T s = 0;
#pragma unroll
  for (int u = 0; u < PF; ++u)
    if (f.k + 8 * u < f.ke) {
      const int j = f.c[u], J = fa[u];
      const T xj = J >= 0 ? x[j] + xc[J] : x[j];
      s = fma(f.v[u], xj, s);
    }
  for (int k = f.k + 8 * PF; k < f.ke; k += 8) {
    const int j = col[k];
    const int J = agg[j];
    const T xj = J >= 0 ? x[j] + xc[J] : x[j];
    s = fma(val[k], xj, s);
  }
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  if (valid && lane == 0 && !skip[i]) {
    const int J = agg[i];
    const T xi = J >= 0 ? x[i] + xc[J] : x[i];
    t[i] = jac_row(xi, sinv[i], b[i], s);
  }
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
  const bool term = m > 0 && off[g + 1] - off[g] == (long long)m * m;
  pdl_wait();
  pdl_trigger();
  if (!term) return;   // not terminal here
  const T *M = inv + off[g];
  for (int i = threadIdx.x; i < m; i += blockDim.x) x[r0 + i] = dense_row(i, m, M, b + r0);
}

// The lower part of the V-cycle in one kernel, out of shared memory: one
// thread block per system copies its rows of the tail levels (matrix, l1
// scaling, aggregates, members, dense inverse of its terminal block) into
// shared memory, walks the levels down and up with a block barrier between
// phases, and writes the first tail level's x back.  Same row arithmetic in
// the same order as the grid kernels, so the result is identical.
constexpr int kTailLevels = 10;
constexpr int kTailThreads = 1024;              // 128 groups of 8 lanes
constexpr size_t kTailSmem = 200 * 1024;        // dynamic shared memory cap

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

// cp.async of one 4- or 8-byte element, global -> shared (Ampere and later)
template <class E>
__device__ __forceinline__ void cp_async(E *dst, const E *src) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(E) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// bytes one system's level takes in the tail's shared memory: m rows, z
// nonzeros, mc rows of the next level, terminal or not
template <class T>
__host__ __device__ inline size_t tail_level_bytes(int m, int z, int mc, bool term) {
  size_t b = a16(4 * ((size_t)m + 1)) + a16(4 * (size_t)z) + a16(sizeof(T) * (size_t)z) + 4 * a16(sizeof(T) * (size_t)m);
  if (term) b += a16(sizeof(T) * (size_t)m * m);
  else b += a16(4 * (size_t)m) + a16(4 * ((size_t)mc + 1)) + a16(4 * (size_t)m);
  return b;
}

template <class T>
struct TailLevel {   // one level, whole batch (global memory)
  const int *sys_start, *nz_start, *rowptr, *col, *agg, *mptr, *mem;
  const T *val, *sinv, *inv;
  const long long *inv_off;   // null if no system is terminal here
  T *x, *b;
};
template <class T>
struct TailDesc {
  TailLevel<T> lv[kTailLevels];
  int nlev;
  unsigned smem;
};
template <class T>
struct TailLoc {   // one level of this block's system (shared memory)
  int m, mc, term;
  int *rp, *col, *agg, *mp, *mem;
  T *val, *sinv, *x, *b, *t, *inv;
};

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(TailDesc<T> d, int *status) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ TailLoc<T> loc[kTailLevels];
  __shared__ long long hdr[kTailLevels][10];   // per level: the scalars below
  __shared__ int nl;                           // levels this system has in the tail
  constexpr int NG = kTailThreads / 8;
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 7, grp = threadIdx.x >> 3;
  // 1. the system's offsets on every tail level, one load per thread
  //    0,1 rows [r0, r1); 2,3 nonzeros [z0, z1); 4,5 inverse [i0, i1);
  //    6,7 next level's rows [c0, c1); 8,9 members [q0, q1) (step 2)
  if (threadIdx.x < 8 * d.nlev) {
    const int k = threadIdx.x >> 3, j = threadIdx.x & 7;
    const TailLevel<T> &G = d.lv[k];
    long long v = 0;
    switch (j) {
      case 0: v = G.sys_start[g]; break;
      case 1: v = G.sys_start[g + 1]; break;
      case 2: v = G.nz_start[g]; break;
      case 3: v = G.nz_start[g + 1]; break;
      case 4: v = G.inv_off ? G.inv_off[g] : 0; break;
      case 5: v = G.inv_off ? G.inv_off[g + 1] : 0; break;
      case 6: v = k + 1 < d.nlev ? d.lv[k + 1].sys_start[g] : 0; break;
      default: v = k + 1 < d.nlev ? d.lv[k + 1].sys_start[g + 1] : 0; break;
    }
    hdr[k][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * d.nlev) {   // members of the next level's rows
    const int k = threadIdx.x >> 1, j = threadIdx.x & 1;
    const long long m = hdr[k][1] - hdr[k][0];
    const bool term = m > 0 && hdr[k][5] - hdr[k][4] == m * m;
    hdr[k][8 + j] = (!term && m > 0 && k + 1 < d.nlev) ? d.lv[k].mptr[hdr[k][6 + j]] : 0;
  }
  // 2. shared-memory layout
  if (threadIdx.x == 0) {
    size_t off = 0;
    int k = 0;
    for (; k < d.nlev; ++k) {
      const int m = (int)(hdr[k][1] - hdr[k][0]);
      if (m == 0) break;
      const int z = (int)(hdr[k][3] - hdr[k][2]);
      const bool term = hdr[k][5] - hdr[k][4] == (long long)m * m;
      const int mc = (!term && k + 1 < d.nlev) ? (int)(hdr[k][7] - hdr[k][6]) : 0;
      TailLoc<T> &L = loc[k];
      L.m = m; L.mc = mc; L.term = term;
      auto take = [&](size_t bytes) { unsigned char *p = sm + off; off += a16(bytes); return p; };
      L.rp = (int *)take(4 * ((size_t)m + 1));
      L.col = (int *)take(4 * (size_t)z);
      L.val = (T *)take(sizeof(T) * (size_t)z);
      L.sinv = (T *)take(sizeof(T) * (size_t)m);
      L.x = (T *)take(sizeof(T) * (size_t)m);
      L.b = (T *)take(sizeof(T) * (size_t)m);
      L.t = (T *)take(sizeof(T) * (size_t)m);
      if (term) {
        L.inv = (T *)take(sizeof(T) * (size_t)m * m);
        L.agg = L.mp = L.mem = nullptr;
      } else {
        L.inv = nullptr;
        L.agg = (int *)take(4 * (size_t)m);
        L.mp = (int *)take(4 * ((size_t)mc + 1));
        L.mem = (int *)take(4 * (size_t)m);
      }
      if (term) { ++k; break; }
    }
    nl = k;
    if (off > d.smem) {   // cannot happen: the host sized d.smem from the same layout
      atomicOr(status, ST_TAIL_SMEM);
      nl = -1;
    }
  }
  __syncthreads();
  if (nl <= 0) {
    pdl_wait();
    return;
  }
  // 3. asynchronous copies global -> shared (no register round trip, all in
  //    flight together), then the indices made local to the system
  for (int k = 0; k < nl; ++k) {
    const TailLevel<T> &G = d.lv[k];
    const TailLoc<T> &L = loc[k];
    const int r0 = (int)hdr[k][0], z0 = (int)hdr[k][2], m = L.m;
    const int z = (int)(hdr[k][3] - z0);
    for (int i = threadIdx.x; i <= m; i += blockDim.x) cp_async(&L.rp[i], &G.rowptr[r0 + i]);
    for (int q = threadIdx.x; q < z; q += blockDim.x) {
      cp_async(&L.col[q], &G.col[z0 + q]);
      cp_async(&L.val[q], &G.val[z0 + q]);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) cp_async(&L.sinv[i], &G.sinv[r0 + i]);
    if (L.term) {
      const T *M = G.inv + hdr[k][4];
      for (int q = threadIdx.x; q < m * m; q += blockDim.x) cp_async(&L.inv[q], &M[q]);
    } else {
      const int c0 = (int)hdr[k][6];
      const int q0 = (int)hdr[k][8], nm = (int)(hdr[k][9] - q0);
      for (int i = threadIdx.x; i < m; i += blockDim.x) cp_async(&L.agg[i], &G.agg[r0 + i]);
      for (int I = threadIdx.x; I <= L.mc; I += blockDim.x) cp_async(&L.mp[I], &G.mptr[c0 + I]);
      for (int p = threadIdx.x; p < nm; p += blockDim.x) cp_async(&L.mem[p], &G.mem[q0 + p]);
    }
  }
  // the right-hand side comes from the preceding kernel
  pdl_wait();
  pdl_trigger();
  {
    const int r0 = (int)hdr[0][0];
    for (int i = threadIdx.x; i < loc[0].m; i += blockDim.x) cp_async(&loc[0].b[i], &d.lv[0].b[r0 + i]);
  }
  cp_async_wait_all();
  __syncthreads();
  for (int k = 0; k < nl; ++k) {
    const TailLoc<T> &L = loc[k];
    const int r0 = (int)hdr[k][0], z0 = (int)hdr[k][2], m = L.m;
    const int z = (int)(hdr[k][3] - z0);
    for (int i = threadIdx.x; i <= m; i += blockDim.x) L.rp[i] -= z0;
    for (int q = threadIdx.x; q < z; q += blockDim.x) L.col[q] -= r0;
    if (!L.term) {
      const int c0 = (int)hdr[k][6], q0 = (int)hdr[k][8], nm = (int)(hdr[k][9] - q0);
      for (int i = threadIdx.x; i < m; i += blockDim.x) L.agg[i] = L.agg[i] >= 0 ? L.agg[i] - c0 : -1;
      for (int I = threadIdx.x; I <= L.mc; I += blockDim.x) L.mp[I] -= q0;
      for (int p = threadIdx.x; p < nm; p += blockDim.x) L.mem[p] -= r0;
    }
  }
  __syncthreads();
  // one op per row, 8 lanes per row, uniform loop bound
  auto rows8 = [&](const TailLoc<T> &L, const T *x, auto &&emit) {
    for (int base = 0; base < L.m; base += NG) {
      const int i = base + grp;
      const bool valid = i < L.m;
      const T s = row_csr<8>(i, valid, lane, L.rp, L.col, L.val, x);
      if (valid && lane == 0) emit(i, s);
    }
  };
  int last = nl - 1;   // deepest level with a coarse correction below it
  for (int k = 0; k < nl; ++k) {
    const TailLoc<T> &L = loc[k];
    if (L.term) {
      for (int i = threadIdx.x; i < L.m; i += blockDim.x) L.x[i] = dense_row(i, L.m, L.inv, L.b);
      __syncthreads();
      last = k - 1;
      break;
    }
    for (int i = threadIdx.x; i < L.m; i += blockDim.x) L.t[i] = jac_first_row(L.b[i], L.sinv[i]);
    __syncthreads();
    rows8(L, L.t, [&](int i, T s) { L.x[i] = jac_row(L.t[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
    rows8(L, L.x, [&](int i, T s) { L.t[i] = L.b[i] - s; });
    __syncthreads();
    if (k + 1 < nl) {
      const TailLoc<T> &C = loc[k + 1];
      for (int I = threadIdx.x; I < C.m; I += blockDim.x) C.b[I] = restrict_row(I, L.mp, L.mem, L.t);
    }
    __syncthreads();
  }
  for (int k = last; k >= 0; --k) {
    const TailLoc<T> &L = loc[k];
    if (k + 1 < nl) {
      const T *xc = loc[k + 1].x;
      for (int i = threadIdx.x; i < L.m; i += blockDim.x)
        if (L.agg[i] >= 0) L.x[i] += xc[L.agg[i]];
    }
    __syncthreads();
    rows8(L, L.x, [&](int i, T s) { L.t[i] = jac_row(L.x[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
    rows8(L, L.t, [&](int i, T s) { L.x[i] = jac_row(L.t[i], L.sinv[i], L.b[i], s); });
    __syncthreads();
  }
  {
    const TailLoc<T> &L = loc[0];
    T *gx = d.lv[0].x + d.lv[0].sys_start[g];
    for (int i = threadIdx.x; i < L.m; i += blockDim.x) gx[i] = L.x[i];
  }
}

// ---- the finest level in scaled variables, matrix in FP16 (VAG_MIXED_F16) ----
// With S = D^-1/2 and h = S A S (FP16), the level works on x~ = S^-1 x and
// b~ = S b: a sweep is x~ += omega D_h^-1 (b~ - h x~) with the l1 scaling of h,
// the residual handed to the restriction is S^-1 (b~ - h x~) = b - A x, the
// coarse correction enters as x~ += S^-1 P x_c, and z = S x~ on the way out.

__global__ void k_scale_setup(int n, const double *__restrict__ dinv, double *__restrict__ s0d,
                              float *__restrict__ s0f, double *__restrict__ sm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = sqrt(1.0 / dinv[i]);   // sqrt(a_ii)
  s0d[i] = d;
  s0f[i] = (float)d;
  sm[i] = 1.0 / d;                        // the D^-1/2 of the FP16 copy
}

// l1 scaling of the stored FP16 rows: 1 / sum_j |h_ij|
__global__ void k_l1_inv_h(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                           const __half *__restrict__ sval, float *__restrict__ sinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int len = rowptr[i + 1] - rowptr[i];
  const int base = slice_ptr[i >> 5] + (i & 31);
  float a = 0.f;
  for (int k = 0; k < len; ++k) a += fabsf(__half2float(sval[base + 32 * k]));
  sinv[i] = 1.f / a;
}

// b~ = S r (FP64 in, FP32 out)
__global__ void k_to_f32_scaled(int n, const double *__restrict__ r, const double *__restrict__ s0d,
                                float *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double si = i < n ? s0d[i] : 1.0;
  pdl_wait();
  pdl_trigger();
  if (i < n) b[i] = (float)(r[i] / si);
}

// z = S x~ (FP32 in, FP64 out)
__global__ void k_to_f64_scaled(int n, const float *__restrict__ x, const double *__restrict__ s0d,
                                double *__restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double si = i < n ? s0d[i] : 1.0;
  pdl_wait();
  pdl_trigger();
  if (i < n) z[i] = (double)x[i] / si;
}

template <int U>
__global__ void k_jac_sell_h(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                             const int *__restrict__ scol, const __half *__restrict__ sval,
                             const float *__restrict__ sinv, const float *__restrict__ b,
                             const float *__restrict__ xin, float *__restrict__ xout, const uint8_t *__restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i >= n || skip[i]) return;
  xout[i] = jac_row(xin[i], sinv[i], b[i], sell_row<float, U, __half>(i, rowptr, slice_ptr, scol, sval, xin));
}

// unscaled residual b - A x = S^-1 (b~ - h x~) for the restriction
template <int U>
__global__ void k_resid_sell_h(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                               const int *__restrict__ scol, const __half *__restrict__ sval,
                               const float *__restrict__ s0f, const float *__restrict__ b,
                               const float *__restrict__ x, float *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i >= n) return;
  r[i] = s0f[i] * (b[i] - sell_row<float, U, __half>(i, rowptr, slice_ptr, scol, sval, x));
}

// a system solved densely on the finest level, in scaled variables:
// x~ = S^-1 A^-1 S^-1 b~ (S^-1 = diag(s0f))
__global__ void k_dense_apply_scaled(const int *__restrict__ sys_start, const long long *__restrict__ off,
                                     const float *__restrict__ inv, const float *__restrict__ s0f,
                                     const float *__restrict__ b, float *x) {
  const int g = blockIdx.x;
  const int r0 = sys_start[g], m = sys_start[g + 1] - r0;
  const bool term = m > 0 && off[g + 1] - off[g] == (long long)m * m;
  pdl_wait();
  pdl_trigger();
  if (!term) return;
  const float *M = inv + off[g];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float acc = 0.f;
    for (int j = 0; j < m; ++j) acc = fmaf(M[i * m + j], s0f[r0 + j] * b[r0 + j], acc);
    x[r0 + i] = s0f[r0 + i] * acc;
  }
}

// x~ += S^-1 P x_c
__global__ void k_prolong_scaled(int n, const int *__restrict__ agg, const float *__restrict__ s0f,
                                 const float *__restrict__ xc, float *x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = i < n ? agg[i] : -1;
  const float si = i < n ? s0f[i] : 0.f;
  pdl_wait();
  pdl_trigger();
  if (J >= 0) x[i] += si * xc[J];
}

// b = a / s (FP32), the scaled-variable conversions of VAG_MIXED_F16 for a
// V-cycle called on FP32 vectors
__global__ void k_div32(int n, const float *__restrict__ a, const float *__restrict__ s, float *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float si = i < n ? s[i] : 1.f;
  pdl_wait();
  pdl_trigger();
  if (i < n) b[i] = a[i] / si;
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_to_f64(int n, const float *__restrict__ a, double *__restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (i < n) b[i] = (double)a[i];
}

}  // namespace


// Build the hierarchy for the current matrix values (called before every
// AMG solve: the numeric phase may have changed them).
void amg_setup(System *s, bool f32, bool f16, bool classical) {
  if (classical && f16) fail(VAG_EINVAL, "the FP16 finest level is for the aggregation hierarchy only");
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
  if (!s->amg_pin) VAG_CUDA(cudaMallocHost(&s->amg_pin, 4 * sizeof(int)));
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
        VAG_CUDA(cudaFuncSetAttribute(k_dense_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem));
        k_dense_inverse<<<ns, TB, kDenseSmem, st>>>(L.d_sys_start, L.rowptr, L.col, L.val, L.inv_off, L.inv,
                                                   s->status);
        note_launches(1);
        VAG_CHECK_LAUNCH();
        if (read_status(s) & ST_NONPOSITIVE) fail(VAG_EINVAL, "AMG: a terminal block is not positive definite");
      }
      if (all) break;
    }
    if (classical) {   // C/F splitting, interpolation, Galerkin R A P
      AmgLevel C;
      rs_coarsen(s, A.levels[lvl], C, alloc);
      trace_mark(st, "level: classical coarsening + Galerkin product");
      A.levels.push_back(C);
      continue;
    }
    AmgLevel &L = A.levels[lvl];
    const int n = L.n;
    uint8_t *strong = static_cast<uint8_t *>(alloc(L.nnz));
    int8_t *state = static_cast<int8_t *>(alloc(n));
    int8_t *next = static_cast<int8_t *>(alloc(n));
    unsigned long long *m1 = static_cast<unsigned long long *>(alloc(8 * (size_t)n));
    float *sd = static_cast<float *>(alloc(4 * (size_t)std::max(n, 1)));
    k_sqrt_diag<<<grid_for(n, TB), TB, 0, st>>>(n, L.dinv, sd);
    k_strength<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, L.val, sd, L.skip, strong, state,
                                               L.d_sys_start, ns, lvl > 0 ? 1 : 0);
    note_launches(2);
    trace_mark(st, "level: terminal blocks + strength");
    // MIS(2) rounds (state and next alternate), polled after 8 rounds and
    // then every 4 (a round after the last decision changes nothing)
    for (int r = 0, poll = 8; r < 64;) {
      k_mis_max1<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, L.d_sys_start, ns, m1,
                                                 undecided);
      k_mis_max2_decide<<<grid_for(n, TB), TB, 0, st>>>(n, L.rowptr, L.col, strong, state, m1, L.d_sys_start,
                                                         ns, next, undecided);
      note_launches(2);
      std::swap(state, next);
      if (++r < poll && r < 64) continue;
      VAG_CUDA(cudaMemcpyAsync(und_host, undecided, sizeof(int), cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaStreamSynchronize(st));
      if (*und_host == 0) break;
      poll += 4;
    }
    if (*und_host != 0) fail(VAG_ECUDA, "AMG: MIS(2) did not finish in 64 rounds");
    trace_mark(st, "level: MIS(2)");
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
    scan_exclusive(cnt, L.mptr, nc, st, false);   // at most n members: no need to wait for the total
    L.mem = static_cast<int *>(alloc(4 * (size_t)std::max(n, 1)));
    k_member_fill<<<grid_for(n, TB), TB, 0, st>>>(n, L.agg, L.mptr, cursor, L.mem);
    k_sort_members<<<grid_for(nc, TB), TB, 0, st>>>(nc, L.mptr, L.mem);
    note_launches(2);
    trace_mark(st, "level: aggregates + members");
    // Galerkin coarse matrix (coarse levels are swept in CSR, 8 lanes per row)
    AmgLevel C;
    C.n = nc;
    C.rowptr = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
    C.dinv = static_cast<double *>(alloc(8 * (size_t)std::max(nc, 1)));
    int *tcol;
    double *tval;
    VAG_CUDA(cudaMallocAsync(&tcol, 4 * (size_t)std::max(nc, 1) * kCoarseWidth, st));
    VAG_CUDA(cudaMallocAsync(&tval, 8 * (size_t)std::max(nc, 1) * kCoarseWidth, st));
    VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));
    k_coarse_build<<<grid_for(nc, kBuildWarps), 32 * kBuildWarps, 0, st>>>(nc, L.mptr, L.mem, L.rowptr, L.col, L.val,
                                                                            L.agg, tcol, tval, cnt, C.dinv, s->status);
    note_launches(1);
    scan_exclusive(cnt, C.rowptr, nc, st, false);
    C.d_sys_start = static_cast<int *>(alloc(4 * ((size_t)ns + 1)));
    k_coarse_starts<<<grid_for(ns + 1, TB), TB, 0, st>>>(ns, L.d_sys_start, rscan, C.d_sys_start);
    note_launches(1);
    // one wait for the coarse nonzero count, the status and the row starts
    C.sys_start.assign(ns + 1, 0);
    VAG_CUDA(cudaMemcpyAsync(&s->amg_pin[0], C.rowptr + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaMemcpyAsync(&s->amg_pin[1], s->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaMemcpyAsync(C.sys_start.data(), C.d_sys_start, 4 * (ns + 1), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    C.nnz = s->amg_pin[0];
    const int cst = s->amg_pin[1];
    if (cst & ST_ROW_OVERFLOW) fail(VAG_EMESH, "AMG: a coarse row couples too many aggregates");
    if (cst & ST_NONPOSITIVE) fail(VAG_EINVAL, "AMG: non-positive coarse diagonal");
    C.col = static_cast<int *>(alloc(4 * (size_t)std::max<int64_t>(C.nnz, 1)));
    C.val = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(C.nnz, 1)));
    k_coarse_compact<<<grid_for(nc, TB), TB, 0, st>>>(nc, tcol, tval, C.rowptr, C.col, C.val);
    note_launches(1);
    VAG_CUDA(cudaFreeAsync(tcol, st));
    VAG_CUDA(cudaFreeAsync(tval, st));
    trace_mark(st, "level: Galerkin product");
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
  if (!A.levels.empty()) A.levels[0].r = static_cast<double *>(alloc(8 * (size_t)std::max(A.levels[0].n, 1)));
  // FP32 copy of the hierarchy (the mixed-precision path)
  A.f32 = f32;
  A.f16 = false;
  A.classical = classical;
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
    A.f16 = f16;
    if (A.f16) {
      const int n0 = s->n_rows;
      A.s0d = static_cast<double *>(alloc(8 * (size_t)std::max(n0, 1)));
      A.s0f = static_cast<float *>(alloc(4 * (size_t)std::max(n0, 1)));
      double *sm = static_cast<double *>(alloc(8 * (size_t)std::max(n0, 1)));
      A.sval16 = static_cast<__half *>(alloc(2 * (size_t)std::max<int64_t>(s->sell_nnz, 1)));
      A.sinv16 = static_cast<float *>(alloc(4 * (size_t)std::max(n0, 1)));
      k_scale_setup<<<grid_for(n0, TB), TB, 0, st>>>(n0, s->dinv, A.s0d, A.s0f, sm);
      note_launches(1);
      sell_values_scaled_f16(s, sm, A.sval16);
      k_l1_inv_h<<<grid_for(n0, TB), TB, 0, st>>>(n0, s->rowptr, s->slice_ptr, A.sval16, A.sinv16);
      note_launches(1);
    }
    for (size_t l = 0; l < A.levels.size(); ++l) {
      AmgLevel &L = A.levels[l];
      if (l == 0) {
        L.sval32 = A.sval32;
      } else {
        L.val32 = cast(L.val, L.nnz);
      }
      L.sinv32 = cast(L.sinv, L.n);
      L.inv32 = L.any_term ? cast(L.inv, L.n_inv) : nullptr;
      if (L.prow) {
        L.pval32 = cast(L.pval, L.p_nnz);
        L.rval32 = cast(L.rval, L.r_nnz);
      }
      L.x32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.b32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
      L.t32 = static_cast<float *>(alloc(4 * (size_t)std::max(L.n, 1)));
    }
    if (!A.levels.empty()) A.levels[0].r32 = static_cast<float *>(alloc(4 * (size_t)std::max(A.levels[0].n, 1)));
  }
  // first nonzero of each system on every coarse level (the tail's layout)
  for (size_t l = 1; l < A.levels.size(); ++l) {
    AmgLevel &L = A.levels[l];
    L.d_nz_start = static_cast<int *>(alloc(4 * ((size_t)ns + 1)));
    k_nz_starts<<<grid_for(ns + 1, TB), TB, 0, st>>>(ns, L.d_sys_start, L.rowptr, L.d_nz_start);
    note_launches(1);
    L.nz_start.assign(ns + 1, 0);
    VAG_CUDA(cudaMemcpyAsync(L.nz_start.data(), L.d_nz_start, 4 * ((size_t)ns + 1), cudaMemcpyDeviceToHost, st));
  }
  VAG_CUDA(cudaStreamSynchronize(st));
  // FP32 hierarchy: first level from which every system's remaining levels
  // fit the tail's shared memory; from there the V-cycle runs in one kernel.
  // (Not for FP64: one SM issues about two FP64 FMAs per clock on GB300, so
  // FP64 work must spread over the whole GPU.)
  A.tail_start = -1;   // the one-kernel tail walks aggregates: not for classical levels
  for (size_t l0 = 1; f32 && !classical && l0 < A.levels.size() && A.tail_start < 0; ++l0) {
    if ((int)(A.levels.size() - l0) > kTailLevels) continue;
    size_t need[2] = {0, 0};
    for (int g = 0; g < ns; ++g) {
      size_t b64 = 0, b32 = 0;
      for (size_t l = l0; l < A.levels.size(); ++l) {
        const AmgLevel &L = A.levels[l];
        const int m = L.sys_start[g + 1] - L.sys_start[g];
        if (m == 0) break;
        const int z = L.nz_start[g + 1] - L.nz_start[g];
        const bool term = m <= kDenseMax;
        const int mc = (!term && l + 1 < A.levels.size())
                           ? A.levels[l + 1].sys_start[g + 1] - A.levels[l + 1].sys_start[g] : 0;
        b64 += tail_level_bytes<double>(m, z, mc, term);
        b32 += tail_level_bytes<float>(m, z, mc, term);
        if (term) break;
      }
      need[0] = std::max(need[0], b64);
      need[1] = std::max(need[1], b32);
    }
    if (need[f32 ? 1 : 0] <= kTailSmem) {
      A.tail_start = (int)l0;
      A.tail_smem[0] = need[0];
      A.tail_smem[1] = need[1];
    }
  }
  if (A.tail_start >= 0) {   // opt in to more than 48 KB of dynamic shared memory
    if (f32)
      VAG_CUDA(cudaFuncSetAttribute(k_vcycle_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem));
    else
      VAG_CUDA(cudaFuncSetAttribute(k_vcycle_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTailSmem));
  }
  VAG_CHECK_LAUNCH();
  trace_mark(st, "smoother scaling, work vectors, FP32 copy");
  if (trace_enabled()) {
    std::fprintf(stderr, "[vag trace] AMG hierarchy: %zu levels, tail from level %d (%zu bytes of shared memory)\n",
                 A.levels.size(), A.tail_start, A.tail_smem[f32 ? 1 : 0]);
    for (size_t l = 0; l < A.levels.size(); ++l) {
      const AmgLevel &L = A.levels[l];
      int mx = 0;
      for (int g = 0; g < ns; ++g) mx = std::max(mx, L.sys_start[g + 1] - L.sys_start[g]);
      std::fprintf(stderr, "  level %zu: rows %d (largest system %d), nnz %lld%s%s\n", l, L.n, mx, (long long)L.nnz,
                   L.any_term ? ", terminal systems" : "", L.all_term ? " (all)" : "");
    }
  }
  A.built = true;
}

// Level arrays of one precision.
template <class T>
struct LV {
  const T *val, *sinv, *inv, *sval;
  T *x, *b, *t, *r;
  const T *pv, *rv;   // classical levels: values of P and R
};
template <class T>
static LV<T> lv(System *s, AmgLevel &L);
template <>
LV<double> lv<double>(System *, AmgLevel &L) {
  return {L.val, L.sinv, L.inv, L.sval, L.x, L.b, L.t, L.r, L.pval, L.rval};
}
template <>
LV<float> lv<float>(System *, AmgLevel &L) {
  return {L.val32, L.sinv32, L.inv32, L.sval32, L.x32, L.b32, L.t32, L.r32, L.pval32, L.rval32};
}   // val32 on coarse levels, sval32 on level 0

// The levels from lvl down, V(2,2) from a zero initial guess, in one kernel.
// Systems that end at a level are solved exactly there; the others are
// smoothed, restricted, corrected from the next level and smoothed again.
template <class T>
static void tail(System *s, int lvl, cudaStream_t st) {
  Amg &A = s->amg;
  TailDesc<T> d{};
  d.nlev = (int)A.levels.size() - lvl;
  if (d.nlev > kTailLevels) fail(VAG_ECUDA, "AMG: too many levels below the tail start");
  for (int k = 0; k < d.nlev; ++k) {
    AmgLevel &L = A.levels[lvl + k];
    const LV<T> v = lv<T>(s, L);
    d.lv[k] = TailLevel<T>{L.d_sys_start, L.d_nz_start, L.rowptr, L.col, L.agg, L.mptr, L.mem, v.val, v.sinv,
                           v.inv, L.any_term ? L.inv_off : nullptr, v.x, v.b};
  }
  const size_t smem = A.tail_smem[sizeof(T) == 4 ? 1 : 0];
  d.smem = (unsigned)smem;
  launch_pdl(k_vcycle_tail<T>, s->seg.n_sys, kTailThreads, smem, st, d, s->status);
  note_launches(1);
}

// x = V(b): one V-cycle from a zero initial guess, one sweep before and after
// the coarse correction on level 0 and two on coarse levels.  Systems that
// end at this level are solved exactly; the others are smoothed, restricted,
// corrected from the next level and smoothed again.  On coarse levels the
// first sweep t = omega D_l1^-1 b has already been made by the restriction
// that produced b.
// cg: level 0 of the FP64 V-cycle inside CG: its first sweep t = omega
// D_l1^-1 r was made by the CG update, and its last sweep also forms r.z
// (returns true when it did)
template <class T>
static bool vcycle(System *s, int lvl, const T *b, T *x, cudaStream_t st, bool cg = false,
                   KrylovScalars *cg_ks = nullptr, int *cg_done = nullptr) {
  Amg &A = s->amg;
  AmgLevel &L = A.levels[lvl];
  if (lvl > 0 && lvl == A.tail_start) {   // b, x are this level's own b, x
    tail<T>(s, lvl, st);
    return false;
  }
  const LV<T> v = lv<T>(s, L);
  const int n = L.n;
  const int g = grid_for(n, TB);
  if (L.any_term) {
    if (sizeof(T) == 4 && lvl == 0 && A.f16)
      launch_pdl(k_dense_apply_scaled, s->seg.n_sys, 64, 0, st, (const int *)L.d_sys_start,
                 (const long long *)L.inv_off, (const float *)L.inv32, (const float *)A.s0f, (const float *)b,
                 (float *)x);
    else
      launch_pdl(k_dense_apply<T>, s->seg.n_sys, 64, 0, st, (const int *)L.d_sys_start,
                 (const long long *)L.inv_off, v.inv, b, x);
    note_launches(1);
  }
  if (L.all_term) return false;
  AmgLevel &C = A.levels[lvl + 1];
  const LV<T> c = lv<T>(s, C);
  constexpr int LN = row_lanes<T>();
  const int gL = grid_for(n, 256 / LN);   // LN lanes per row
  // finest level: the autotuned loads in flight of the sliced-ELL row loop
  auto jac_sell = s->sell_u == 2 ? k_jac_sell<T, 2> : s->sell_u == 8 ? k_jac_sell<T, 8> : k_jac_sell<T, 4>;
  auto resid_sell = s->sell_u == 2 ? k_resid_sell<T, 2> : s->sell_u == 8 ? k_resid_sell<T, 8> : k_resid_sell<T, 4>;
  const bool h16 = sizeof(T) == 4 && lvl == 0 && A.f16;   // scaled FP16 finest level
  auto jac_h = s->sell_u == 2 ? k_jac_sell_h<2> : s->sell_u == 8 ? k_jac_sell_h<8> : k_jac_sell_h<4>;
  if (h16) {
    const float *bb = (const float *)b;
    float *xx = (float *)x, *tt = A.levels[0].t32;
    const LV<float> c32 = lv<float>(s, C);
    auto resid_h = s->sell_u == 2 ? k_resid_sell_h<2> : s->sell_u == 8 ? k_resid_sell_h<8> : k_resid_sell_h<4>;
    launch_pdl(k_jac_first<float>, g, TB, 0, st, n, bb, (const float *)A.sinv16, tt);
    launch_pdl(resid_h, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr, (const int *)L.scol,
               (const __half *)A.sval16, (const float *)A.s0f, bb, (const float *)tt, L.r32);
    launch_pdl(k_restrict_first<float>, grid_for(C.n, TB), TB, 0, st, C.n, (const int *)L.mptr, (const int *)L.mem,
               (const float *)L.r32, c32.sinv, c32.b, c32.t);
    note_launches(3);
  } else if (lvl == 0) {
    // level 0: sliced ELL, one thread per row; one sweep from zero, t =
    // omega D_l1^-1 b, then the residual b - A t for the restriction
    if (!cg) launch_pdl(k_jac_first<T>, g, TB, 0, st, n, b, v.sinv, v.t);
    launch_pdl(resid_sell, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr,
               (const int *)L.scol, v.sval, b, (const T *)v.t, v.r);
    if (A.classical)
      launch_pdl(k_rs_restrict<T>, grid_for(C.n, 256 / LN), 256, 0, st, C.n, (const int *)L.rrow,
                 (const int *)L.rcol, v.rv, (const T *)v.r, c.sinv, c.b, c.t);
    else
      launch_pdl(k_restrict_first<T>, grid_for(C.n, TB), TB, 0, st, C.n, (const int *)L.mptr, (const int *)L.mem,
                 (const T *)v.r, c.sinv, c.b, c.t);
    note_launches(cg ? 2 : 3);
  } else if (A.classical) {
    // classical coarse levels: second sweep, residual, restriction R
    launch_pdl(k_jac_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)v.t, x, (const uint8_t *)L.skip);
    launch_pdl(k_resid_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, b,
               (const T *)x, v.t);
    launch_pdl(k_rs_restrict<T>, grid_for(C.n, 256 / LN), 256, 0, st, C.n, (const int *)L.rrow, (const int *)L.rcol,
               v.rv, (const T *)v.t, c.sinv, c.b, c.t);
    note_launches(3);
  } else {
    // coarse levels: CSR, 8 lanes per row; residual and restriction fused
    launch_pdl(k_jac_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)v.t, x, (const uint8_t *)L.skip);
    if (n > 6 * C.n) {   // large aggregates: residual over all rows, then restriction
      launch_pdl(k_resid_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, b,
                 (const T *)x, v.t);
      launch_pdl(k_restrict_first<T>, grid_for(C.n, TB), TB, 0, st, C.n, (const int *)L.mptr, (const int *)L.mem,
                 (const T *)v.t, c.sinv, c.b, c.t);
      note_launches(3);
    } else {
      launch_pdl(k_resid_restrict8<T>, grid_for(C.n, 8), 256, 0, st, C.n, (const int *)L.mptr, (const int *)L.mem,
                 (const int *)L.rowptr, (const int *)L.col, v.val, b, (const T *)x, c.sinv, c.b, c.t);
      note_launches(2);
    }
  }
  vcycle<T>(s, lvl + 1, c.b, c.x, st);
  // post-smoothing: level 0 adds the coarse correction to t and makes one
  // sweep from it into x; coarse levels make two sweeps, the first applying
  // the coarse correction as it reads x
  if (h16) {
    const float *bb = (const float *)b;
    float *xx = (float *)x, *tt = A.levels[0].t32;
    launch_pdl(k_prolong_scaled, g, TB, 0, st, n, (const int *)L.agg, (const float *)A.s0f,
               (const float *)A.levels[1].x32, tt);
    launch_pdl(jac_h, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr, (const int *)L.scol,
               (const __half *)A.sval16, (const float *)A.sinv16, bb, (const float *)tt, xx, (const uint8_t *)L.skip);
    note_launches(2);
  } else if (lvl == 0) {
    if (A.classical)
      launch_pdl(k_rs_prolong<T>, g, TB, 0, st, n, (const int *)L.prow, (const int *)L.pcol, v.pv, (const T *)c.x,
                 v.t);
    else
      launch_pdl(k_prolong<T>, g, TB, 0, st, n, (const int *)L.agg, (const T *)c.x, v.t);
    if (cg) {   // the last sweep forms r.z for the Krylov loop (cg_ks, cg_done)
      auto jr = s->sell_u == 2 ? k_jac_sell_rz<T, 2> : s->sell_u == 8 ? k_jac_sell_rz<T, 8> : k_jac_sell_rz<T, 4>;
      const Tiles tl{s->seg.tile_sys, s->seg.tile_row0, s->seg.tile_row1, s->seg.sys_tile0, s->seg.sys_grp0,
                     s->seg.n_tiles, s->seg.n_sys};
      launch_pdl(jr, s->seg.n_tiles, 256, 0, st, (const int *)L.rowptr, (const int *)L.slice_ptr,
                 (const int *)L.scol, (const T *)v.sval, (const T *)v.sinv, (const T *)b, (const T *)v.t, (T *)x,
                 (const uint8_t *)L.skip, tl, s->partials, s->counter, cg_ks, cg_done);
      note_launches(2);
      return true;
    }
    launch_pdl(jac_sell, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr, (const int *)L.scol,
               v.sval, v.sinv, b, (const T *)v.t, x, (const uint8_t *)L.skip);
    note_launches(2);
  } else if (A.classical) {
    // coarse correction x += P x_c, then two sweeps
    launch_pdl(k_rs_prolong<T>, g, TB, 0, st, n, (const int *)L.prow, (const int *)L.pcol, v.pv, (const T *)c.x, x);
    launch_pdl(k_jac_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)x, v.t, (const uint8_t *)L.skip);
    launch_pdl(k_jac_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)v.t, x, (const uint8_t *)L.skip);
    note_launches(3);
  } else {
    launch_pdl(k_prolong_jac8<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)x, (const int *)L.agg, (const T *)c.x, v.t, (const uint8_t *)L.skip);
    launch_pdl(k_jac_csr<T>, gL, 256, 0, st, n, (const int *)L.rowptr, (const int *)L.col, v.val, v.sinv, b,
               (const T *)v.t, x, (const uint8_t *)L.skip);
    note_launches(2);
  }
  return false;
}

void amg_apply(System *s, const double *r, double *z, cudaStream_t st) {
  Amg &A = s->amg;
  if (!A.f32) {
    vcycle<double>(s, 0, r, z, st);
    return;
  }
  AmgLevel &L0 = A.levels[0];
  const int n = L0.n;
  if (A.f16) {   // scaled variables on the finest level
    launch_pdl(k_to_f32_scaled, grid_for(n, TB), TB, 0, st, n, r, (const double *)A.s0d, L0.b32);
    vcycle<float>(s, 0, L0.b32, L0.x32, st);
    launch_pdl(k_to_f64_scaled, grid_for(n, TB), TB, 0, st, n, (const float *)L0.x32, (const double *)A.s0d, z);
    note_launches(2);
    return;
  }
  launch_pdl(k_to_f32, grid_for(n, TB), TB, 0, st, (int64_t)n, r, L0.b32);
  vcycle<float>(s, 0, L0.b32, L0.x32, st);
  launch_pdl(k_to_f64, grid_for(n, TB), TB, 0, st, n, (const float *)L0.x32, z);
  note_launches(2);
}

void amg_apply_f32(System *s, const float *r, float *z, cudaStream_t st) {
  Amg &A = s->amg;
  if (!A.f32) fail(VAG_EINVAL, "amg_apply_f32 needs the FP32 hierarchy");
  AmgLevel &L0 = A.levels[0];
  const int n = L0.n;
  if (A.f16) {   // scaled variables on the finest level: b~ = S r, z = S x~
    launch_pdl(k_div32, grid_for(n, TB), TB, 0, st, n, r, (const float *)A.s0f, L0.b32);
    vcycle<float>(s, 0, L0.b32, L0.x32, st);
    launch_pdl(k_div32, grid_for(n, TB), TB, 0, st, n, (const float *)L0.x32, (const float *)A.s0f, z);
    note_launches(2);
    return;
  }
  vcycle<float>(s, 0, r, z, st);
}

bool amg_apply_cg(System *s, const double *r, double *z, cudaStream_t st) {
  if (s->amg.f32 || s->amg.levels.empty() || s->amg.levels[0].all_term) return false;
  return vcycle<double>(s, 0, r, z, st, true, s->ks, s->n_done);
}

bool amg_apply_f32_cg(System *s, const float *r, float *z, cudaStream_t st, KrylovScalars *ks, int *n_done) {
  const Amg &A = s->amg;
  if (!A.f32 || A.f16 || A.levels.empty() || A.levels[0].all_term) return false;
  return vcycle<float>(s, 0, r, z, st, true, ks, n_done);
}

const float *amg_first_sweep_scale_f32(System *s, float *&t0, float &omega) {
  const Amg &A = s->amg;
  if (!A.f32 || A.f16 || A.levels.empty() || A.levels[0].all_term) return nullptr;
  t0 = A.levels[0].t32;
  omega = (float)kOmega;
  return A.levels[0].sinv32;
}

const double *amg_first_sweep_scale(System *s, double *&t0, double &omega) {
  if (s->amg.f32 || s->amg.levels.empty() || s->amg.levels[0].all_term) return nullptr;
  t0 = s->amg.levels[0].t;
  omega = kOmega;
  return s->amg.levels[0].sinv;
}

// Mean duration of one finest-level sweep (x_out = x_in + omega D_l1^-1
// (b - A x_in)) of the last hierarchy, FP64 or FP32, launched as in the
// V-cycle.
double time_smoother(System *s, int reps) {
  Amg &A = s->amg;
  if (!A.built || A.levels.empty() || A.f16) fail(VAG_EINVAL, "no FP64 or FP32 AMG hierarchy: solve with AMG first");
  AmgLevel &L = A.levels[0];
  cudaStream_t st = s->ctx->stream;
  const int n = L.n, g = grid_for(n, TB);
  if (A.f32) {
    auto jac = s->sell_u == 2 ? k_jac_sell<float, 2> : s->sell_u == 8 ? k_jac_sell<float, 8> : k_jac_sell<float, 4>;
    auto sweep32 = [&](const float *xin, float *xout) {
      launch_pdl(jac, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr, (const int *)L.scol,
                 (const float *)L.sval32, (const float *)L.sinv32, (const float *)L.b32, xin, xout,
                 (const uint8_t *)L.skip);
      note_launches(1);
    };
    VAG_CUDA(cudaMemsetAsync(L.x32, 0, sizeof(float) * n, st));
    VAG_CUDA(cudaMemsetAsync(L.b32, 0, sizeof(float) * n, st));
    sweep32(L.x32, L.t32);   // warm-up
    VAG_CUDA(cudaEventRecord(s->ev0, st));
    for (int r = 0; r < reps; ++r) {
      if (r & 1) sweep32(L.t32, L.x32);
      else sweep32(L.x32, L.t32);
    }
    VAG_CUDA(cudaEventRecord(s->ev1, st));
    VAG_CUDA(cudaEventSynchronize(s->ev1));
    float ms = 0.f;
    VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
    return (double)ms / reps;
  }
  if (!s->kz) fail(VAG_EINVAL, "no FP64 AMG hierarchy: solve with AMG first");
  auto sweep = [&](const double *xin, double *xout) {
    auto jac = s->sell_u == 2 ? k_jac_sell<double, 2> : s->sell_u == 8 ? k_jac_sell<double, 8> : k_jac_sell<double, 4>;
    launch_pdl(jac, g, TB, 0, st, n, (const int *)L.rowptr, (const int *)L.slice_ptr,
               (const int *)L.scol, (const double *)L.sval, (const double *)L.sinv, (const double *)s->kr, xin, xout,
               (const uint8_t *)L.skip);
    note_launches(1);
  };
  VAG_CUDA(cudaMemsetAsync(s->kz, 0, sizeof(double) * n, st));
  sweep(s->kz, s->kp);   // warm-up
  VAG_CUDA(cudaEventRecord(s->ev0, st));
  for (int r = 0; r < reps; ++r) {
    if (r & 1) sweep(s->kp, s->kz);
    else sweep(s->kz, s->kp);
  }
  VAG_CUDA(cudaEventRecord(s->ev1, st));
  VAG_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  VAG_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  return (double)ms / reps;
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
