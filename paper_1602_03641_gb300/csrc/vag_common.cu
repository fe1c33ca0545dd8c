// Shared device utilities: budget-checked allocation, exclusive scan, status.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "vag_internal.cuh"

namespace vag {

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool t_capturing = false;
void set_capturing(bool on) { t_capturing = on; }
void note_launches(unsigned long long n) {
  if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ trace ---
// With the environment variable VAG_TRACE set, the phases of each API call
// are marked with a device event and a host clock reading on the call's
// stream, and printed to stderr when the call ends (device time between
// consecutive marks, and host time spent issuing them).  Off by default;
// marks are skipped while a graph is being captured.
namespace {
struct TraceMark {
  const char *label;
  cudaEvent_t ev;
  std::chrono::steady_clock::time_point host;
};
thread_local std::vector<TraceMark> t_marks;
bool trace_on() {
  static const bool on = std::getenv("VAG_TRACE") != nullptr;
  return on;
}
}  // namespace

bool trace_enabled() { return trace_on(); }

void trace_mark(cudaStream_t st, const char *label) {
  if (!trace_on() || t_capturing) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, st);
  t_marks.push_back({label, e, std::chrono::steady_clock::now()});
}

void trace_report(const char *call) {
  if (!trace_on() || t_marks.empty()) return;
  cudaEventSynchronize(t_marks.back().ev);
  std::fprintf(stderr, "[vag trace] %s\n", call);
  for (size_t i = 1; i < t_marks.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t_marks[i - 1].ev, t_marks[i].ev);
    const double host = std::chrono::duration<double, std::milli>(t_marks[i].host - t_marks[i - 1].host).count();
    std::fprintf(stderr, "  %-34s device %9.3f ms   host %9.3f ms\n", t_marks[i].label, ms, host);
  }
  for (auto &m : t_marks) cudaEventDestroy(m.ev);
  t_marks.clear();
}

void *ctx_alloc(Ctx *c, size_t bytes) {
  void *p = nullptr;
  cudaError_t e = c->pool ? cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(VAG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}

void ctx_free(Ctx *c, void *p) {
  if (!p) return;
  if (c->pool) cudaFreeAsync(p, c->stream);
  else cudaFree(p);
}

void *sys_alloc_bytes(System *s, size_t bytes) {
  Ctx *c = s->ctx;
  bytes = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);   // a zero-size array still gets a valid pointer
  if (c->budget && c->in_use + bytes > c->budget)
    fail(VAG_EBUDGET, "device memory budget exceeded (" + std::to_string(c->in_use + bytes) +
                          " > " + std::to_string(c->budget) + " bytes)");
  void *p = ctx_alloc(c, bytes);
  s->allocs.push_back({p, bytes});
  s->bytes += bytes;
  c->in_use += bytes;
  return p;
}

void sys_free_all(System *s) {
  for (auto &a : s->allocs) ctx_free(s->ctx, a.ptr);
  if (s->ctx) s->ctx->in_use -= s->bytes;
  s->allocs.clear();
  s->bytes = 0;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 0x7fffffff) g = 0x7fffffff;
  return (int)g;
}

int read_status(System *s) {
  int st = 0;
  VAG_CUDA(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->ctx->stream));
  VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  return st;
}

// ------------------------------------------------------------------ scan ----
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_sum(int v, int *total) {
  __shared__ int warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  return incl - v + warp_tot[warp];
}

__global__ void scan_tiles(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ tile_sums,
                           int n) {
  __shared__ int tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    sum += v[i];
  }
  int off = block_exclusive_sum(sum, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = off;
    off += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void add_tile_offsets(int *__restrict__ out, const int *__restrict__ offs, int n) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int add = offs[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    int64_t idx = base + i;
    if (idx < n) out[idx] += add;
  }
}

__global__ void write_total(int *out, int n, const int *tile_sums_scanned, int ntiles,
                            const int *tile_sums) {
  out[n] = tile_sums_scanned[ntiles - 1] + tile_sums[ntiles - 1];
}

void scan_rec(const int *in, int *out, int n, cudaStream_t st) {
  // out has room for n+1 entries; writes exclusive prefix and out[n] = total.
  int ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  int *sums = nullptr;
  VAG_CUDA(cudaMallocAsync(&sums, sizeof(int) * (2 * ntiles + 1), st));
  int *sums_scan = sums + ntiles;
  scan_tiles<<<ntiles, kScanThreads, 0, st>>>(in, out, sums, n);
  VAG_CHECK_LAUNCH();
  note_launches(2);   // scan_tiles + write_total
  if (ntiles > 1) {
    scan_rec(sums, sums_scan, ntiles, st);
    add_tile_offsets<<<ntiles, kScanThreads, 0, st>>>(out, sums_scan, n);
    VAG_CHECK_LAUNCH();
    note_launches(1);
  } else {
    VAG_CUDA(cudaMemsetAsync(sums_scan, 0, sizeof(int), st));
  }
  write_total<<<1, 1, 0, st>>>(out, n, sums_scan, ntiles, sums);
  VAG_CHECK_LAUNCH();
  VAG_CUDA(cudaFreeAsync(sums, st));
}
}  // namespace

int scan_exclusive(const int *in, int *out, int n, cudaStream_t st, bool want_total) {
  if (n == 0) {
    VAG_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
    return 0;
  }
  scan_rec(in, out, n, st);
  if (!want_total) return -1;
  int total = 0;
  VAG_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  return total;
}

}  // namespace vag
