// vag_spmv_dot_noalloc: y = A x and x.y on caller-owned CSR arrays, with no
// device allocation at all.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// want the product -- code running inside their own stream-capture region,
// allocator-restricted host threads (e.g. a real-time serving loop that
// forbids allocation after start-up), or embedders whose memory is fully
// reserved by another runtime.  Every other entry point of this library
// allocates its scratch with cudaMalloc/cudaMallocAsync; this one keeps its
// scratch (one partial sum per thread block plus an arrival counter) in a
// file-scope __device__ array of fixed size that every GPU which loads the
// library holds until the process exits.
//
// In host code `g_na_partials` / `g_na_counter` are host-side stand-ins for
// the device symbols, not device addresses: their device addresses are looked
// up once per device with cudaGetSymbolAddress (with that device current) and
// cached.  That lookup happens on the first call on each device, so make the
// first call on a device before any stream capture that includes it.  The
// cache lives as long as the process: after cudaDeviceReset the module is
// loaded again and the cached addresses may be stale, so a process that resets
// a device must not call this entry point again on it.
//
// The scratch is shared by every call on a device and keeps the contents of
// the last call.  The arrival counter must start at zero: each call clears it
// with a stream-ordered memset before its kernel, and the last block resets it.
// Calls whose kernels overlap on the GPU (for example issued on two streams
// without ordering) race on the scratch and give wrong results; order them.
#include <mutex>

#include "vag_internal.cuh"
#include "vag_reduce.cuh"

namespace {

constexpr int kNT = 256;                                   // threads per block
constexpr int kLanes = 8;                                  // lanes per CSR row
constexpr int kRowsPerBlock = kNT / kLanes;                // 32 rows per block
constexpr int kMaxBlocks = VAG_NOALLOC_MAX_ROWS / kRowsPerBlock;
static_assert(VAG_NOALLOC_MAX_ROWS % kRowsPerBlock == 0, "row limit must fill whole blocks");

__device__ __align__(256) double g_na_partials[kMaxBlocks];   // 1 MiB
__device__ __align__(256) unsigned int g_na_counter[64];

struct DeviceScratch {
  double *partials = nullptr;
  unsigned int *counter = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// Looks up (once per device, with that device current) the device addresses
// of the static scratch.
cudaError_t scratch_for(int dev, DeviceScratch *out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  DeviceScratch &s = g_scratch[dev];
  if (!s.partials) {
    void *p = nullptr, *c = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_partials);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&c, g_na_counter);
    if (e != cudaSuccess) return e;
    s.partials = static_cast<double *>(p);
    s.counter = static_cast<unsigned int *>(c);
  }
  *out = s;
  return cudaSuccess;
}

// One block per 32 rows (8 lanes per row), so the grid never exceeds the
// static partial-sum array for n <= VAG_NOALLOC_MAX_ROWS.
__global__ void __launch_bounds__(kNT) k_spmv_dot_static(int n, const int *__restrict__ rowptr,
                                                        const int *__restrict__ col, const double *__restrict__ val,
                                                        const double *__restrict__ x, double *__restrict__ y,
                                                        double *partials, unsigned int *counter, double *xdoty) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int row = blockIdx.x * kRowsPerBlock + threadIdx.x / kLanes;
  double s = 0.0;
  if (row < n) {
    const int b = rowptr[row], e = rowptr[row + 1];
    for (int k = b + lane; k < e; k += kLanes) s = fma(val[k], __ldg(&x[col[k]]), s);
  }
#pragma unroll
  for (int o = kLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  double dp = 0.0;
  if (row < n && lane == 0) {
    y[row] = s;
    dp = x[row] * s;
  }
  double v[1] = {dp}, out[1];
  if (vag::grid_sum<kNT, 1>(v, partials, counter, out) && threadIdx.x == 0) *xdoty = out[0];
}

}  // namespace

extern "C" vag_status vag_spmv_dot_noalloc(int32_t n_rows, const int32_t *rowptr, const int32_t *col,
                                           const double *val, const double *x, double *y, double *xdoty,
                                           void *stream) {
  if (n_rows < 0 || n_rows > VAG_NOALLOC_MAX_ROWS) return VAG_EINVAL;
  if (!rowptr || !xdoty || (n_rows > 0 && (!col || !val || !x || !y))) return VAG_EINVAL;
  // rows read x[col[k]] while other rows write y: the two must not overlap
  if (n_rows > 0) {
    const uintptr_t xb = reinterpret_cast<uintptr_t>(x), yb = reinterpret_cast<uintptr_t>(y);
    const uintptr_t len = sizeof(double) * (uintptr_t)n_rows;
    if (xb < yb + len && yb < xb + len) return VAG_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VAG_ECUDA;
  DeviceScratch sc;
  if (scratch_for(dev, &sc) != cudaSuccess) return VAG_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sc.counter, 0, sizeof(unsigned int), st) != cudaSuccess) return VAG_ECUDA;
  const int grid = n_rows > 0 ? (n_rows + kRowsPerBlock - 1) / kRowsPerBlock : 1;
  k_spmv_dot_static<<<grid, kNT, 0, st>>>(n_rows, rowptr, col, val, x, y, sc.partials, sc.counter, xdoty);
  vag::note_launches(1);
  return cudaGetLastError() == cudaSuccess ? VAG_OK : VAG_ECUDA;
}
