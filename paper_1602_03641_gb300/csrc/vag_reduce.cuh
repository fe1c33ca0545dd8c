// Deterministic block and grid reductions (fixed summation order for a fixed
// grid: per-block partials, then the last block to finish sums the partials
// in index order).
#pragma once
#include "vag_internal.cuh"

namespace vag {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh /* NT/32 doubles */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

// Writes K per-block values to partials[K*blockIdx.x + k]; returns true in
// every thread of the last block to arrive, after which `out[k]` (thread 0)
// holds the grid totals in a fixed order.
template <int NT, int K>
__device__ __forceinline__ bool grid_sum(const double (&v)[K], double *partials, unsigned *counter,
                                         double (&out)[K]) {
  __shared__ double sh[NT / 32];
  __shared__ bool last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bs[k] = block_sum<NT>(v[k], sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[K * blockIdx.x + k] = bs[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) acc += __ldcg(&partials[K * b + k]);
    out[k] = block_sum<NT>(acc, sh);
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Row tiles of a batch: tile t covers rows [row0[t], row1[t]) of system
// sys[t]; sys_tile0 gives the first tile of each system (n_sys+1 entries).
// The tiles of a system form groups of kSegGroup consecutive tiles (the last
// one shorter); grp0 gives each system's first group (n_sys+1 entries).
constexpr int kSegGroup = 32;
struct Tiles {
  const int *sys, *row0, *row1, *sys_tile0;
  const int *grp0;
  int n_tiles, n_sys;
};

// Sums K values per system in two levels, so that no counter sees more than
// about kSegGroup or n_tiles / kSegGroup arrivals (a system of 8 000 tiles
// otherwise queues 8 000 atomics on one address): per-tile block sums go to
// partials[K*t + k]; the last tile of a group to arrive adds the group's
// tile partials in tile order into partials[K*(n_tiles + g) + k]; the last
// group of system `sys` to finish adds its group partials in group order and
// returns true in all its threads with out[] valid in thread 0.  The grouping
// depends on the system alone, so the sums do too.  Counters: counter[sys]
// per system, counter[n_sys + 1 + g] per group.
template <int NT, int K>
__device__ __forceinline__ bool seg_sum(const double (&v)[K], double *partials, unsigned *counter, const Tiles &tl,
                                        int t, int sys, double (&out)[K]) {
  __shared__ double sh[NT / 32];
  __shared__ bool last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bs[k] = block_sum<NT>(v[k], sh);
  const int t0 = tl.sys_tile0[sys], t1 = tl.sys_tile0[sys + 1];
  const int gl = (t - t0) / kSegGroup;                 // group within the system
  const int ga = t0 + gl * kSegGroup;                  // its tiles [ga, gb)
  const int gb = min(ga + kSegGroup, t1);
  const int g = tl.grp0[sys] + gl;                     // its storage index
  const int ng = tl.grp0[sys + 1] - tl.grp0[sys];
  unsigned *gctr = counter + tl.n_sys + 1;
  double *gpart = partials + (size_t)K * tl.n_tiles;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)K * t + k] = bs[k];
    __threadfence();
    const unsigned ticket = atomicAdd(&gctr[g], 1u);
    last = (ticket == (unsigned)(gb - ga - 1));
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double gs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = ga + threadIdx.x; b < gb; b += NT) acc += __ldcg(&partials[(size_t)K * b + k]);
    gs[k] = block_sum<NT>(acc, sh);
  }
  if (threadIdx.x == 0) {
    gctr[g] = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) gpart[(size_t)K * g + k] = gs[k];
    __threadfence();
    const unsigned ticket = atomicAdd(&counter[sys], 1u);
    last = (ticket == (unsigned)(ng - 1));
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int g0 = tl.grp0[sys];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < ng; b += NT) acc += __ldcg(&gpart[(size_t)K * (g0 + b) + k]);
    out[k] = block_sum<NT>(acc, sh);
  }
  if (threadIdx.x == 0) counter[sys] = 0u;
  return true;
}

}  // namespace vag
