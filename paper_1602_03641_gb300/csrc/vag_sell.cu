// Sliced-ELL copy (slices of 32 consecutive rows, column-major inside a
// slice) of the eliminated system, for thread-per-row SpMV: the 32 threads of
// a warp read entry k of their 32 rows as one contiguous 256-byte (FP64) or
// 128-byte (FP32) segment, and a row costs exactly one FMA per stored entry
// (no cross-lane reduction -- on GB300 the FP64 pipe, not HBM, limits a
// lane-split CSR SpMV).  Entries of a row keep their CSR order, so a row sum
// is the same sequence of FMAs whatever the slice layout.
#include <functional>

#include "vag_internal.cuh"

namespace vag {
namespace {

constexpr int TB = 256;

__global__ void k_slice_width(int n, int n_slices, const int *__restrict__ rowptr, int *__restrict__ width) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= n_slices) return;
  int w = 0;
  const int r1 = min(n, (sl + 1) * 32);
  for (int r = sl * 32; r < r1; ++r) w = max(w, rowptr[r + 1] - rowptr[r]);
  width[sl] = 32 * w;
}

__global__ void k_sell_cols(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                            const int *__restrict__ slice_ptr, int *__restrict__ scol) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int b = rowptr[row], e = rowptr[row + 1];
  const int base = slice_ptr[row >> 5] + (row & 31);
  for (int k = 0; k < e - b; ++k) scol[base + 32 * k] = col[b + k];
}

// padding slots point at the row itself (their values are 0)
__global__ void k_sell_pad(int n, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                           int *__restrict__ scol) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= ((n + 31) / 32) * 32) return;
  const int sl = row >> 5;
  const int w = (slice_ptr[sl + 1] - slice_ptr[sl]) / 32;
  const int len = row < n ? rowptr[row + 1] - rowptr[row] : 0;
  const int base = slice_ptr[sl] + (row & 31);
  for (int k = len; k < w; ++k) scol[base + 32 * k] = row < n ? row : 0;
}

template <class T>
__device__ __forceinline__ T to_store(double v) { return (T)v; }
template <>
__device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }

template <class T>
__global__ void k_sell_vals(int n, const int *__restrict__ rowptr, const double *__restrict__ val,
                            const double *__restrict__ scale, const int *__restrict__ col,
                            const int *__restrict__ slice_ptr, T *__restrict__ sval) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int b = rowptr[row], e = rowptr[row + 1];
  const int base = slice_ptr[row >> 5] + (row & 31);
  const double sr = scale ? scale[row] : 1.0;
  for (int k = 0; k < e - b; ++k) {
    const double v = scale ? sr * val[b + k] * scale[col[b + k]] : val[b + k];
    sval[base + 32 * k] = to_store<T>(v);
  }
  // padding up to the slice width: value 0 (its column is the row itself)
  const int w = (slice_ptr[(row >> 5) + 1] - slice_ptr[row >> 5]) >> 5;
  for (int k = e - b; k < w; ++k) sval[base + 32 * k] = to_store<T>(0.0);
}

}  // namespace

// Sliced-ELL structure of any CSR matrix (n rows): slice_ptr [n_slices+1]
// and scol [total]; returns total.  The caller supplies the allocator.
int64_t sell_structure(cudaStream_t st, int n, const int *rowptr, const int *col, int **slice_ptr_out,
                       int **scol_out, const std::function<void *(size_t)> &alloc) {
  const int n_slices = (n + 31) / 32;
  int *slice_ptr = static_cast<int *>(alloc(sizeof(int) * ((size_t)n_slices + 1)));
  int *width;
  VAG_CUDA(cudaMallocAsync(&width, sizeof(int) * ((size_t)n_slices + 1), st));
  k_slice_width<<<grid_for(n_slices, TB), TB, 0, st>>>(n, n_slices, rowptr, width);
  note_launches(1);
  VAG_CHECK_LAUNCH();
  const int64_t total = n_slices ? scan_exclusive(width, slice_ptr, n_slices, st) : 0;
  if (!n_slices) VAG_CUDA(cudaMemsetAsync(slice_ptr, 0, sizeof(int), st));
  VAG_CUDA(cudaFreeAsync(width, st));
  int *scol = static_cast<int *>(alloc(sizeof(int) * (size_t)std::max<int64_t>(total, 1)));
  if (n > 0) {
    k_sell_cols<<<grid_for(n, TB), TB, 0, st>>>(n, rowptr, col, slice_ptr, scol);
    k_sell_pad<<<grid_for((int64_t)n_slices * 32, TB), TB, 0, st>>>(n, rowptr, slice_ptr, scol);
    note_launches(2);
    VAG_CHECK_LAUNCH();
  }
  *slice_ptr_out = slice_ptr;
  *scol_out = scol;
  return total;
}

void build_sell(System *s) {
  s->n_slices = (s->n_rows + 31) / 32;
  s->sell_nnz = sell_structure(s->ctx->stream, s->n_rows, s->rowptr, s->col, &s->slice_ptr, &s->scol,
                               [s](size_t bytes) { return sys_alloc_bytes(s, bytes); });
  s->sval = sys_alloc<double>(s, (size_t)std::max<int64_t>(s->sell_nnz, 1));
}

void sell_values(System *s) {
  cudaStream_t st = s->ctx->stream;
  k_sell_vals<double><<<grid_for(s->n_rows, TB), TB, 0, st>>>(s->n_rows, s->rowptr, s->val, nullptr, s->col,
                                                               s->slice_ptr, s->sval);
  note_launches(1);
  VAG_CHECK_LAUNCH();
}

// FP32 copy of D^{-1/2} A D^{-1/2} (scale = D^{-1/2}, FP64) for the inner
// solve of the mixed-precision path.
void sell_values_scaled_f32(System *s, const double *scale, float *out) {
  cudaStream_t st = s->ctx->stream;
  k_sell_vals<float><<<grid_for(s->n_rows, TB), TB, 0, st>>>(s->n_rows, s->rowptr, s->val, scale, s->col,
                                                              s->slice_ptr, out);
  note_launches(1);
  VAG_CHECK_LAUNCH();
}

void sell_values_f32(System *s, float *out) { sell_values_scaled_f32(s, nullptr, out); }

// FP16 copy of D^{-1/2} A D^{-1/2} (scale = D^{-1/2}, FP64): unit diagonal,
// off-diagonal entries in [-1, 1], so FP16 keeps about three digits of each.
void sell_values_scaled_f16(System *s, const double *scale, __half *out) {
  cudaStream_t st = s->ctx->stream;
  k_sell_vals<__half><<<grid_for(s->n_rows, TB), TB, 0, st>>>(s->n_rows, s->rowptr, s->val, scale, s->col,
                                                               s->slice_ptr, out);
  note_launches(1);
  VAG_CHECK_LAUNCH();
}

}  // namespace vag
