// Classical (Ruge-Stueben-type) coarsening for the AMG hierarchy: the
// counterpart of the classical AMG (Hypre's BoomerAMG) that the paper's
// solver experiments (Sec. 5.3-5.4) found robust in the fracture/matrix
// permeability ratio.  Written from the classical construction (Ruge and
// Stueben, "Algebraic multigrid", 1987; Stueben, "A review of algebraic
// multigrid", 2001) with the parallel PMIS splitting (De Sterck, Yang, Heys,
// SIAM J. Matrix Anal. Appl. 27, 2006).  Per level, all on the device:
//  strength   i depends strongly on j != i when -a_ij >= theta max_{k != i}
//             (-a_ik) (negative couplings; positive ones never count);
//  measure    the number of rows that depend strongly on i; the eliminated
//             VAG matrix is symmetric, so whether j depends on i is read from
//             row i's entry a_ij and row j's largest negative coupling, with
//             no transpose of the strength graph;
//  PMIS       rows no row depends on are fine from the start; then, in
//             rounds, an undecided row whose key (measure, a hash of its
//             system-local index, the index) is the largest among its
//             undecided strong neighbours (either direction) becomes coarse,
//             and undecided rows that depend on a new coarse row become fine;
//  2nd pass   a fine row with strong connections but no coarse one becomes
//             coarse, so every such row interpolates from at least one;
//  P          direct interpolation: coarse rows copy their value; a fine row
//             i takes w_ij = -alpha_i a_ij / (a_ii + sum_{k != i} a_ik^+) from
//             its strong coarse neighbours (at most kPmax, the largest
//             |a_ij|, ties by index), alpha_i = (sum of all its negative
//             couplings) / (sum over the chosen ones), so that P maps the
//             constant to the constant on zero-row-sum rows; rows without
//             strong connections interpolate from nothing (the smoother
//             handles them);
//  R = P^T    transposed with its rows sorted by fine index;
//  Galerkin   A_c = R A P, one coarse row per warp, every entry summed in a
//             fixed sequence order and the row's columns in the order they
//             first appear (deterministic: a system's hierarchy depends on
//             that system alone, so it is bitwise the same in a batch).
#include <climits>
#include <functional>
#include <vector>

#include "vag_internal.cuh"

namespace vag {
namespace {

constexpr int TB = 256;
constexpr double kRsTheta = 0.25;
constexpr int kPmax = 4;
constexpr int kMaxRounds = 64;

__device__ __forceinline__ uint32_t rs_hash(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x;
}

__device__ __forceinline__ int rs_sys_of_row(int i, const int *__restrict__ start, int n_sys) {
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// largest negative coupling -a_ik over k != i (0 when there is none)
__global__ void k_rs_maxneg(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, double *__restrict__ maxneg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
    if (col[k] != i && -val[k] > m) m = -val[k];
  maxneg[i] = m;
}

// i depends strongly on j through the entry a (= a_ij = a_ji)
__device__ __forceinline__ bool rs_strong(double a, double maxneg_row) {
  return maxneg_row > 0.0 && -a >= kRsTheta * maxneg_row;
}

// state: 0 undecided, 1 coarse, -1 fine, -2 fine without strong connections
// (interpolates from nothing), -3 row of a system solved densely here
__global__ void k_rs_init(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                          const double *__restrict__ val, const double *__restrict__ maxneg,
                          const uint8_t *__restrict__ skip, const int *__restrict__ sys_start, int n_sys,
                          unsigned long long *__restrict__ key, int8_t *__restrict__ state,
                          uint8_t *__restrict__ sflag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (skip[i]) {
    key[i] = 0;
    state[i] = -3;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) sflag[k] = 0;
    return;
  }
  bool depends = false;
  unsigned infl = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = col[k];
    uint8_t f = 0;
    if (j != i) {
      const bool dij = rs_strong(val[k], maxneg[i]);   // i depends on j
      const bool dji = rs_strong(val[k], maxneg[j]);   // j depends on i
      depends |= dij;
      infl += dji;
      f = (uint8_t)(dij | (dji << 1));
    }
    sflag[k] = f;   // the strength of the entry, both ways, for the PMIS rounds
  }
  const int loc = i - sys_start[rs_sys_of_row(i, sys_start, n_sys)];
  key[i] = ((unsigned long long)(infl < 65535u ? infl : 65535u) << 48) |
           ((unsigned long long)(rs_hash((uint32_t)loc) & 0xffffu) << 32) | (uint32_t)loc;
  state[i] = (!depends && infl == 0) ? -2 : (infl == 0 ? -1 : 0);
}

// PMIS round, first half: undecided rows that are the largest among their
// undecided strong neighbours become coarse
__global__ void k_rs_pmis_c(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const uint8_t *__restrict__ sflag, const unsigned long long *__restrict__ key,
                            const int8_t *__restrict__ st_in, int8_t *__restrict__ st_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int8_t s = st_in[i];
  if (s != 0) {
    st_out[i] = s;
    return;
  }
  const unsigned long long ki = key[i];
  bool top = true;
  for (int k = rowptr[i]; k < rowptr[i + 1] && top; ++k) {
    if (!sflag[k]) continue;   // not strong either way (or the diagonal)
    const int j = col[k];
    if (st_in[j] == 0 && key[j] > ki) top = false;
  }
  st_out[i] = top ? 1 : 0;
}

// second half: undecided rows that depend on a coarse row become fine; the
// rest are counted
__global__ void k_rs_pmis_f(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const uint8_t *__restrict__ sflag, const int8_t *__restrict__ st_in,
                            int8_t *__restrict__ st_out, int *undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int8_t o = 1;
  if (i < n) {
    const int8_t s = st_in[i];
    o = s;
    if (s == 0) {
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        if ((sflag[k] & 1) && st_in[col[k]] == 1) {   // i depends on a coarse row
          o = -1;
          break;
        }
      }
    }
    st_out[i] = o;
  }
  // one atomic per warp for the rows still undecided
  const unsigned m = __ballot_sync(0xffffffffu, o == 0);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(undecided, __popc(m));
}

// second pass: a fine row that depends on rows but on no coarse one becomes
// coarse
__global__ void k_rs_second_pass(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                                 const double *__restrict__ val, const double *__restrict__ maxneg,
                                 const int8_t *__restrict__ st_in, int8_t *__restrict__ st_out,
                                 int *__restrict__ cflag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int8_t s = st_in[i];
  if (s == -1) {
    bool depends = false, has_c = false;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = col[k];
      if (j == i || !rs_strong(val[k], maxneg[i])) continue;
      depends = true;
      has_c |= st_in[j] == 1;
    }
    if (depends && !has_c) s = 1;
  }
  st_out[i] = s;
  cflag[i] = s == 1;
}

// the chosen coarse neighbours of fine row i: its strong coarse neighbours,
// at most kPmax of them with the largest |a_ij| (ties by smaller index);
// returned as CSR positions in CSR order
__device__ __forceinline__ int rs_choose(int i, const int *__restrict__ rowptr, const int *__restrict__ col,
                                         const double *__restrict__ val, const double *__restrict__ maxneg,
                                         const int8_t *__restrict__ st, int (&pick)[kPmax]) {
  int m = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const int j = col[k];
    if (j == i || st[j] != 1 || !rs_strong(val[k], maxneg[i])) continue;
    const double a = fabs(val[k]);
    if (m < kPmax) {
      pick[m++] = k;
      continue;
    }
    // replace the weakest pick (on a tie the one of larger index) if this
    // one is strictly stronger
    int wq = 0;
    for (int q = 1; q < kPmax; ++q) {
      const double aq = fabs(val[pick[q]]), aw = fabs(val[pick[wq]]);
      if (aq < aw || (aq == aw && col[pick[q]] > col[pick[wq]])) wq = q;
    }
    if (a > fabs(val[pick[wq]])) pick[wq] = k;
  }
  for (int p = 1; p < m; ++p)   // CSR order
    for (int q = p; q > 0 && pick[q - 1] > pick[q]; --q) {
      const int t = pick[q];
      pick[q] = pick[q - 1];
      pick[q - 1] = t;
    }
  return m;
}

__global__ void k_rs_p_count(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ maxneg,
                             const int8_t *__restrict__ st, int *__restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int8_t s = st[i];
  int c = 0;
  if (s == 1) {
    c = 1;
  } else if (s == -1) {
    int pick[kPmax];
    c = rs_choose(i, rowptr, col, val, maxneg, st, pick);
  }
  cnt[i] = c;
}

__global__ void k_rs_p_fill(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ maxneg,
                            const int8_t *__restrict__ st, const int *__restrict__ cidx,
                            const int *__restrict__ prow, int *__restrict__ pcol, double *__restrict__ pval,
                            int *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int8_t s = st[i];
  const int o = prow[i];
  if (s == 1) {
    pcol[o] = cidx[i];
    pval[o] = 1.0;
    return;
  }
  if (s != -1) return;
  int pick[kPmax];
  const int m = rs_choose(i, rowptr, col, val, maxneg, st, pick);
  if (m != prow[i + 1] - o) {
    atomicOr(status, ST_BAD_INDEX);
    return;
  }
  double aii = 0.0, neg = 0.0, pos = 0.0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const double a = val[k];
    if (col[k] == i) aii += a;
    else if (a < 0.0) neg += a;
    else pos += a;
  }
  double cneg = 0.0;
  for (int q = 0; q < m; ++q) cneg += val[pick[q]];
  const double diag = aii + pos;
  if (!(diag > 0.0) || !(cneg < 0.0)) {
    atomicOr(status, ST_NONPOSITIVE);
    return;
  }
  const double alpha = neg / cneg;
  for (int q = 0; q < m; ++q) {
    pcol[o + q] = cidx[col[pick[q]]];
    pval[o + q] = -alpha * val[pick[q]] / diag;
  }
}

// R = P^T: counts per coarse row, entries placed by an atomic cursor, then
// each row sorted by fine index (so its content does not depend on the order
// of the atomics)
__global__ void k_rs_r_count(int n, const int *__restrict__ prow, const int *__restrict__ pcol, int *rcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = prow[i]; k < prow[i + 1]; ++k) atomicAdd(&rcnt[pcol[k]], 1);
}

__global__ void k_rs_r_fill(int n, const int *__restrict__ prow, const int *__restrict__ pcol,
                            const double *__restrict__ pval, const int *__restrict__ rrow, int *cursor,
                            int *__restrict__ rcol, double *__restrict__ rval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = prow[i]; k < prow[i + 1]; ++k) {
    const int I = pcol[k];
    const int q = rrow[I] + atomicAdd(&cursor[I], 1);
    rcol[q] = i;
    rval[q] = pval[k];
  }
}

__global__ void k_rs_r_sort(int nc, const int *__restrict__ rrow, int *rcol, double *rval) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  for (int p = rrow[I] + 1; p < rrow[I + 1]; ++p) {
    const int c = rcol[p];
    const double v = rval[p];
    int q = p - 1;
    while (q >= rrow[I] && rcol[q] > c) {
      rcol[q + 1] = rcol[q];
      rval[q + 1] = rval[q];
      --q;
    }
    rcol[q + 1] = c;
    rval[q + 1] = v;
  }
}

// A_c = R A P row by row, each warp taking coarse rows I, I + (warps in the
// grid), ...: for every entry r_Ii of row I of R (in order), the entries a_ik
// of row i of A 32 at a time, each lane walking row k of P (at most kPmax
// entries) one entry per round; the contributions r_Ii a_ik p_kJ meet in a
// shared-memory hash keyed by J, lanes that hit the same slot are grouped
// and the lowest adds their values in lane order, so every entry is summed in
// the order (entry of R, chunk of A's row, entry of P, lane), fixed by the
// data.  A column enters the row's list when it first appears, the columns
// new in one round in the order of their lowest lane (a ballot prefix), so
// the list order is fixed by the data too.  A row may use at most HASH/2
// slots (ST_ROW_OVERFLOW otherwise).  Its (column, sum) pairs are written in
// list order to the row's padded slot zcol/zval[I*HASH/2 ..], the table is
// cleared through the list, the count goes to zcnt[I] and 1/z_II to zdinv;
// k_rs_compact packs the rows.
template <int HASH, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_rs_rap(int nrows, const int *__restrict__ rrow,
                                                       const int *__restrict__ rcol, const double *__restrict__ rval,
                                                       const int *__restrict__ arow, const int *__restrict__ acol,
                                                       const double *__restrict__ aval,
                                                       const int *__restrict__ prow, const int *__restrict__ pcol,
                                                       const double *__restrict__ pval, int *__restrict__ zcnt,
                                                       int *__restrict__ zcol, double *__restrict__ zval,
                                                       double *__restrict__ zdinv, int *status) {
  constexpr int CAP = HASH / 2;
  __shared__ int keys[WARPS][HASH];
  __shared__ double sums[WARPS][HASH];
  __shared__ int used[WARPS][CAP];
  __shared__ double vals[WARPS][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  int *K = keys[w];
  double *S = sums[w];
  int *U = used[w];
  for (int h = lane; h < HASH; h += 32) {
    K[h] = -1;
    S[h] = 0.0;
  }
  __syncwarp();
  const int stride = gridDim.x * WARPS;
  for (int I = blockIdx.x * WARPS + w; I < nrows; I += stride) {   // a whole warp takes each row
    int nu = 0;                 // columns listed so far (the same in every lane)
    bool overflow = false;
    // one round: each lane offers (J, v) (J < 0: nothing)
    auto add = [&](int J, double v) {
      int slot = -1;
      bool claimed = false;
      if (J >= 0) {
        unsigned h = ((unsigned)J * 2654435761u) & (HASH - 1);
        for (int probe = 0; probe < HASH; ++probe, h = (h + 1) & (HASH - 1)) {
          const int cur = ((volatile int *)K)[h];
          if (cur == J) { slot = (int)h; break; }
          if (cur == -1) {
            const int old = atomicCAS(&K[h], -1, J);
            if (old == -1) { slot = (int)h; claimed = true; break; }
            if (old == J) { slot = (int)h; break; }
          }
        }
        if (slot < 0) overflow = true;
      }
      vals[w][lane] = v;
      __syncwarp();
      const unsigned grp = __match_any_sync(0xffffffffu, slot >= 0 ? slot : -1 - lane);
      const bool is_new = (grp & __ballot_sync(0xffffffffu, claimed)) != 0;
      const bool leader = slot >= 0 && lane == __ffs(grp) - 1;
      const unsigned lead_new = __ballot_sync(0xffffffffu, leader && is_new);
      if (leader && is_new) {
        const int q = nu + __popc(lead_new & below);
        if (q < CAP) U[q] = slot;
      }
      nu += __popc(lead_new);
      if (leader) {
        double acc = S[slot];
        for (unsigned m = grp; m; m &= m - 1) acc += vals[w][__ffs(m) - 1];
        S[slot] = acc;
      }
      __syncwarp();
    };
    for (int kr = rrow[I]; kr < rrow[I + 1]; ++kr) {
      const int i = rcol[kr];
      const double r = rval[kr];
      const int ab = arow[i], ae = arow[i + 1];
      for (int c = ab; c < ae; c += 32) {
        const int k = c + lane;
        int eb = 0, len = 0;
        double a = 0.0;
        if (k < ae) {
          const int j = acol[k];
          a = r * aval[k];
          eb = prow[j];
          len = prow[j + 1] - eb;
        }
        const int mlen = __reduce_max_sync(0xffffffffu, len);
        for (int e = 0; e < mlen; ++e) add(e < len ? pcol[eb + e] : -1, e < len ? a * pval[eb + e] : 0.0);
      }
    }
    __syncwarp();
    const bool bad = __any_sync(0xffffffffu, overflow) || nu > CAP;
    if (bad) {
      if (lane == 0) {
        atomicOr(status, ST_ROW_OVERFLOW);
        zcnt[I] = 0;
      }
      // the list is incomplete: clear the whole table
      for (int h = lane; h < HASH; h += 32) {
        K[h] = -1;
        S[h] = 0.0;
      }
      __syncwarp();
      continue;
    }
    if (lane == 0) zcnt[I] = nu;
    const size_t base = (size_t)I * CAP;   // the row's padded slot; compacted afterwards
    bool diag = false;
    for (int q = lane; q < nu; q += 32) {
      const int h = U[q];
      const int J = K[h];
      const double z = S[h];
      zcol[base + q] = J;
      zval[base + q] = z;
      K[h] = -1;
      S[h] = 0.0;
      if (zdinv && J == I) {
        diag = true;
        if (!(z > 0.0)) atomicOr(status, ST_NONPOSITIVE);
        zdinv[I] = 1.0 / z;
      }
    }
    if (zdinv && !__any_sync(0xffffffffu, diag) && lane == 0) {
      atomicOr(status, ST_NONPOSITIVE);
      zdinv[I] = 1.0 / 0.0;
    }
    __syncwarp();
  }
}

// grids of k_rs_rap: enough warps to fill the GPU a few times over, each
// warp then walks many rows
static int rap_blocks(int nrows, int warps) {
  const int want = (nrows + warps - 1) / warps;
  const int cap = num_sms() * 32;
  return std::max(1, std::min(want, cap));
}

template <int CAP>
__global__ void k_rs_compact(int nc, const int *__restrict__ tcol, const double *__restrict__ tval,
                             const int *__restrict__ rowptr, int *__restrict__ col, double *__restrict__ val) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const size_t base = (size_t)I * CAP;
  for (int q = 0; q < rowptr[I + 1] - rowptr[I]; ++q) {
    col[rowptr[I] + q] = tcol[base + q];
    val[rowptr[I] + q] = tval[base + q];
  }
}

__global__ void k_rs_coarse_starts(int n_sys, const int *__restrict__ sys_start, const int *__restrict__ cscan,
                                   int *csys_start) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g <= n_sys) csys_start[g] = cscan[sys_start[g]];
}

// stream-ordered temporaries of the context's pool, freed on every path
struct RsTemps {
  Ctx *c;
  std::vector<void *> p;
  ~RsTemps() {
    for (void *q : p) ctx_free(c, q);
  }
  void *operator()(size_t bytes) {
    void *q = ctx_alloc(c, bytes ? bytes : 1);
    p.push_back(q);
    return q;
  }
};

}  // namespace

void rs_coarsen(System *s, AmgLevel &L, AmgLevel &C, const std::function<void *(size_t)> &alloc) {
  cudaStream_t st = s->ctx->stream;
  const int n = L.n, ns = s->seg.n_sys;
  RsTemps tmp{s->ctx, {}};
  trace_mark(st, "  classical: enter");
  double *maxneg = static_cast<double *>(tmp(8 * (size_t)std::max(n, 1)));
  unsigned long long *key = static_cast<unsigned long long *>(tmp(8 * (size_t)std::max(n, 1)));
  int8_t *sa = static_cast<int8_t *>(tmp(std::max(n, 1)));
  int8_t *sb = static_cast<int8_t *>(tmp(std::max(n, 1)));
  int *undecided = static_cast<int *>(tmp(sizeof(int)));
  const int g = grid_for(n, TB);
  k_rs_maxneg<<<g, TB, 0, st>>>(n, L.rowptr, L.col, L.val, maxneg);
  uint8_t *sflag = static_cast<uint8_t *>(tmp((size_t)std::max<int64_t>(L.nnz, 1)));
  k_rs_init<<<g, TB, 0, st>>>(n, L.rowptr, L.col, L.val, maxneg, L.skip, L.d_sys_start, ns, key, sa, sflag);
  note_launches(2);
  VAG_CHECK_LAUNCH();
  trace_mark(st, "  classical: strength + measure");
  // PMIS rounds (two kernels each, states ping-pong), polled every 4 rounds
  int *und_host = s->n_done_host;   // pinned int
  bool finished = false;
  for (int r = 0; r < kMaxRounds; ++r) {
    VAG_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int), st));
    k_rs_pmis_c<<<g, TB, 0, st>>>(n, L.rowptr, L.col, sflag, key, sa, sb);
    k_rs_pmis_f<<<g, TB, 0, st>>>(n, L.rowptr, L.col, sflag, sb, sa, undecided);
    note_launches(2);
    if ((r & 3) != 3) continue;
    VAG_CUDA(cudaMemcpyAsync(und_host, undecided, sizeof(int), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
    if (*und_host == 0) {
      finished = true;
      break;
    }
  }
  if (!finished) fail(VAG_ECUDA, "AMG: the PMIS splitting did not finish");
  trace_mark(st, "  classical: PMIS rounds");
  int *cflag = static_cast<int *>(tmp(4 * (size_t)std::max(n, 1)));
  int *cidx = static_cast<int *>(tmp(4 * ((size_t)n + 1)));
  k_rs_second_pass<<<g, TB, 0, st>>>(n, L.rowptr, L.col, L.val, maxneg, sa, sb, cflag);
  note_launches(1);
  scan_exclusive(cflag, cidx, n, st, false);
  const int8_t *state = sb;
  // P: row counts, then one read-back of the coarse count and of P's
  // nonzeros (R = P^T has as many)
  int *pcnt = static_cast<int *>(tmp(4 * ((size_t)n + 1)));
  L.prow = static_cast<int *>(alloc(4 * ((size_t)n + 1)));
  k_rs_p_count<<<g, TB, 0, st>>>(n, L.rowptr, L.col, L.val, maxneg, state, pcnt);
  note_launches(1);
  scan_exclusive(pcnt, L.prow, n, st, false);
  int *pin = s->amg_pin;   // pinned
  VAG_CUDA(cudaMemcpyAsync(&pin[0], cidx + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaMemcpyAsync(&pin[1], L.prow + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  const int nc = pin[0];
  L.p_nnz = pin[1];
  L.pcol = static_cast<int *>(alloc(4 * (size_t)std::max<int64_t>(L.p_nnz, 1)));
  L.pval = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(L.p_nnz, 1)));
  VAG_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), st));   // checked after the Galerkin product
  k_rs_p_fill<<<g, TB, 0, st>>>(n, L.rowptr, L.col, L.val, maxneg, state, cidx, L.prow, L.pcol, L.pval, s->status);
  note_launches(1);
  // R = P^T
  int *rcnt = static_cast<int *>(tmp(4 * ((size_t)nc + 1)));
  int *cursor = static_cast<int *>(tmp(4 * ((size_t)nc + 1)));
  L.rrow = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
  VAG_CUDA(cudaMemsetAsync(rcnt, 0, 4 * ((size_t)nc + 1), st));
  VAG_CUDA(cudaMemsetAsync(cursor, 0, 4 * ((size_t)nc + 1), st));
  k_rs_r_count<<<g, TB, 0, st>>>(n, L.prow, L.pcol, rcnt);
  note_launches(1);
  scan_exclusive(rcnt, L.rrow, nc, st, false);
  L.r_nnz = L.p_nnz;
  L.rcol = static_cast<int *>(alloc(4 * (size_t)std::max<int64_t>(L.r_nnz, 1)));
  L.rval = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(L.r_nnz, 1)));
  k_rs_r_fill<<<g, TB, 0, st>>>(n, L.prow, L.pcol, L.pval, L.rrow, cursor, L.rcol, L.rval);
  k_rs_r_sort<<<grid_for(nc, TB), TB, 0, st>>>(nc, L.rrow, L.rcol, L.rval);
  note_launches(2);
  VAG_CHECK_LAUNCH();
  L.nc = nc;
  trace_mark(st, "  classical: second pass, P, R");
  // Galerkin A_c = R A P in one pass into rows padded to kRapHash/2 columns,
  // then packed
  constexpr int kRapHash = 512, kRapWarps = 4, kRapCap = kRapHash / 2;
  C.n = nc;
  C.rowptr = static_cast<int *>(alloc(4 * ((size_t)nc + 1)));
  C.dinv = static_cast<double *>(alloc(8 * (size_t)std::max(nc, 1)));
  int *cc = static_cast<int *>(tmp(4 * ((size_t)nc + 1)));
  int *tcol = static_cast<int *>(tmp(4 * (size_t)std::max(nc, 1) * kRapCap));
  double *tval = static_cast<double *>(tmp(8 * (size_t)std::max(nc, 1) * kRapCap));
  const int gc = rap_blocks(nc, kRapWarps);
  k_rs_rap<kRapHash, kRapWarps><<<gc, 32 * kRapWarps, 0, st>>>(nc, L.rrow, L.rcol, L.rval, L.rowptr, L.col, L.val,
                                                               L.prow, L.pcol, L.pval, cc, tcol, tval, C.dinv,
                                                               s->status);
  note_launches(1);
  scan_exclusive(cc, C.rowptr, nc, st, false);
  VAG_CUDA(cudaMemcpyAsync(&pin[0], C.rowptr + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaMemcpyAsync(&pin[1], s->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  C.nnz = pin[0];
  {
    const int stv = pin[1];
    if (stv & ST_BAD_INDEX) fail(VAG_ECUDA, "AMG: internal interpolation count mismatch");
    if (stv & ST_ROW_OVERFLOW) fail(VAG_EMESH, "AMG: a coarse row couples too many coarse rows");
    if (stv & ST_NONPOSITIVE)
      fail(VAG_EINVAL, "AMG: a fine row has no usable coarse couplings or a coarse diagonal is not positive");
  }
  C.col = static_cast<int *>(alloc(4 * (size_t)std::max<int64_t>(C.nnz, 1)));
  C.val = static_cast<double *>(alloc(8 * (size_t)std::max<int64_t>(C.nnz, 1)));
  k_rs_compact<kRapCap><<<grid_for(nc, TB), TB, 0, st>>>(nc, tcol, tval, C.rowptr, C.col, C.val);
  note_launches(1);
  trace_mark(st, "  classical: Galerkin R A P");
  C.d_sys_start = static_cast<int *>(alloc(4 * ((size_t)ns + 1)));
  k_rs_coarse_starts<<<grid_for(ns + 1, TB), TB, 0, st>>>(ns, L.d_sys_start, cidx, C.d_sys_start);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  C.sys_start.assign(ns + 1, 0);
  VAG_CUDA(cudaMemcpyAsync(C.sys_start.data(), C.d_sys_start, 4 * ((size_t)ns + 1), cudaMemcpyDeviceToHost, st));
  const int stv = read_status(s);   // synchronises
  if (stv & ST_BAD_INDEX) fail(VAG_ECUDA, "AMG: internal sparse-product count mismatch");
  if (stv & ST_NONPOSITIVE) fail(VAG_EINVAL, "AMG: non-positive coarse diagonal");
}

}  // namespace vag
