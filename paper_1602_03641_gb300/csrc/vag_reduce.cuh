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
struct Tiles {
  const int *sys, *row0, *row1, *sys_tile0;
};

// Sums K values per system: per-tile block sums go to partials[K*t + k]; the
// last tile of system `sys` to arrive adds its system's partials in tile
// order and returns true in all its threads with out[] valid in thread 0.
template <int NT, int K>
__device__ __forceinline__ bool seg_sum(const double (&v)[K], double *partials, unsigned *counter, const Tiles &tl,
                                        int t, int sys, double (&out)[K]) {
  __shared__ double sh[NT / 32];
  __shared__ bool last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bs[k] = block_sum<NT>(v[k], sh);
  const int t0 = tl.sys_tile0[sys], t1 = tl.sys_tile0[sys + 1];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)K * t + k] = bs[k];
    __threadfence();
    const unsigned ticket = atomicAdd(&counter[sys], 1u);
    last = (ticket == (unsigned)(t1 - t0 - 1));
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = t0 + threadIdx.x; b < t1; b += NT) acc += __ldcg(&partials[(size_t)K * b + k]);
    out[k] = block_sum<NT>(acc, sh);
  }
  if (threadIdx.x == 0) counter[sys] = 0u;
  return true;
}

}  // namespace vag
