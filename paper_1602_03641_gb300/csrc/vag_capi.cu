// extern "C" entry points of libvag (declared in include/vag.h): argument
// checks, host/device staging, and the mapping of internal errors to status
// codes.  No exception crosses this boundary.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "vag_internal.cuh"
#include "vag_topo.h"

using namespace vag;

namespace {

template <class F>
vag_status guarded(Ctx *c, F &&f) {
  try {
    f();
    if (c) c->last_error.clear();
    return VAG_OK;
  } catch (const Error &e) {
    if (c) c->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    if (c) c->last_error = "host allocation failed";
    return VAG_ENOMEM;
  } catch (...) {
    if (c) c->last_error = "unexpected internal error";
    return VAG_ECUDA;
  }
}

// NVTX range around an API call (visible to Nsight tools; a no-op without one)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

void check_mem(int mem) {
  if (mem != VAG_MEM_HOST && mem != VAG_MEM_DEVICE) fail(VAG_EINVAL, "mem must be VAG_MEM_HOST or VAG_MEM_DEVICE");
}

cudaMemcpyKind to_dev(int mem) { return mem == VAG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind from_dev(int mem) { return mem == VAG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

template <class T>
T *upload(System *s, const T *src, size_t n, int mem, const char *what) {
  if (n && !src) fail(VAG_EINVAL, std::string(what) + " is NULL");
  T *d = sys_alloc<T>(s, n);
  if (n) VAG_CUDA(cudaMemcpyAsync(d, src, sizeof(T) * n, to_dev(mem), s->ctx->stream));
  return d;
}

template <class T>
void copy_in(System *s, T *dst, const T *src, size_t n, int mem, const char *what) {
  if (n && !src) fail(VAG_EINVAL, std::string(what) + " is NULL");
  if (n) VAG_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n, to_dev(mem), s->ctx->stream));
}

// Peaceman wells of one or more systems, validated on the host and put in
// the union's fracture-face numbering.
struct WellsHost {
  std::vector<int> ff;
  std::vector<double> wi, pw, q, cin;
  bool fixes_level = false;   // some perforation has WI > 0
};

template <class T>
void fetch(std::vector<T> &dst, const T *src, size_t n, int mem, cudaStream_t st, const char *what) {
  if (n && !src) fail(VAG_EINVAL, std::string(what) + " is NULL");
  const size_t old = dst.size();
  dst.resize(old + n);
  if (!n) return;
  if (mem == VAG_MEM_HOST) {
    std::copy(src, src + n, dst.begin() + old);
  } else {
    VAG_CUDA(cudaMemcpyAsync(dst.data() + old, src, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
  }
}

void gather_wells(WellsHost &w, const vag_props &p, int mem, int nf_sys, int ff_off, cudaStream_t st) {
  if (p.n_perf < 0) fail(VAG_EINVAL, "n_perf < 0");
  if (p.n_perf == 0) return;
  const size_t n = (size_t)p.n_perf, b = w.ff.size();
  fetch(w.ff, p.well_ff, n, mem, st, "well_ff");
  fetch(w.wi, p.well_wi, n, mem, st, "well_wi");
  fetch(w.pw, p.well_pw, n, mem, st, "well_pw");
  fetch(w.q, p.well_q, n, mem, st, "well_q");
  fetch(w.cin, p.well_cin, n, mem, st, "well_cin");
  std::vector<int> seen(w.ff.begin() + b, w.ff.end());
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) fail(VAG_EINVAL, "a fracture face is perforated twice");
  for (size_t i = b; i < b + n; ++i) {
    if (w.ff[i] < 0 || w.ff[i] >= nf_sys) fail(VAG_EINVAL, "well_ff out of range");
    if (!(w.wi[i] >= 0.0) || !std::isfinite(w.wi[i])) fail(VAG_EINVAL, "well_wi must be finite and >= 0");
    if (!std::isfinite(w.pw[i]) || !std::isfinite(w.q[i]) || !std::isfinite(w.cin[i]))
      fail(VAG_EINVAL, "well_pw, well_q and well_cin must be finite");
    if (w.wi[i] > 0.0) w.fixes_level = true;
    w.ff[i] += ff_off;
  }
}

void upload_wells(System *s, const WellsHost &w) {
  const int n = (int)w.ff.size();
  if (n > s->perf_cap) {
    s->well_ff = sys_alloc<int>(s, n);
    s->well_wi = sys_alloc<double>(s, n);
    s->well_pw = sys_alloc<double>(s, n);
    s->well_q = sys_alloc<double>(s, n);
    s->well_cin = sys_alloc<double>(s, n);
    s->Fw = sys_alloc<double>(s, n);
    s->perf_cap = n;
  }
  if (!s->ff_perf) s->ff_perf = sys_alloc<int>(s, s->nf > 0 ? s->nf : 1);
  cudaStream_t st = s->ctx->stream;
  if (n) {
    VAG_CUDA(cudaMemsetAsync(s->Fw, 0, sizeof(double) * n, st));   // no well rates before a solve
    VAG_CUDA(cudaMemcpyAsync(s->well_ff, w.ff.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    VAG_CUDA(cudaMemcpyAsync(s->well_wi, w.wi.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    VAG_CUDA(cudaMemcpyAsync(s->well_pw, w.pw.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    VAG_CUDA(cudaMemcpyAsync(s->well_q, w.q.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    VAG_CUDA(cudaMemcpyAsync(s->well_cin, w.cin.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  // fracture face -> perforation (or -1), for the transport map
  std::vector<int> fp((size_t)(s->nf > 0 ? s->nf : 1), -1);
  for (int i = 0; i < n; ++i) fp[w.ff[i]] = i;
  VAG_CUDA(cudaMemcpyAsync(s->ff_perf, fp.data(), sizeof(int) * fp.size(), cudaMemcpyHostToDevice, st));
  VAG_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
  s->n_perf = n;
}

// Shapes of a general mesh: keep the per-cell array only when some cell is
// not a hexahedron (the symbolic phase then groups the cells by shape).
void set_shapes(System *s, int8_t *shape, unsigned mask, bool tri) {
  s->tri_ff = s->tri_ff || tri;
  s->cell_shape = mask == (1u << topo::HEX) ? nullptr : shape;
}

template <class T>
void copy_out(const System *s, T *dst, const T *src, size_t n, int mem) {
  if (dst && n) VAG_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n, from_dev(mem), s->ctx->stream));
}

void use_device(Ctx *c) { VAG_CUDA(cudaSetDevice(c->device)); }

// Segment starts of a batch (host vectors already filled) copied to the device.
void upload_segments(System *s) {
  Segments &g = s->seg;
  const int n1 = g.n_sys + 1;
  g.d_node_start = upload(s, g.node_start.data(), n1, VAG_MEM_HOST, "node_start");
  g.d_ff_start = upload(s, g.ff_start.data(), n1, VAG_MEM_HOST, "ff_start");
  g.d_cell_start = upload(s, g.cell_start.data(), n1, VAG_MEM_HOST, "cell_start");
  g.d_row_start = sys_alloc<int>(s, n1);
  VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
}

__global__ void k_add_offset(int *a, int64_t n, int off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && a[i] >= 0) a[i] += off;   // -1 marks an unused node slot
}

void free_ctx(vag_ctx *ctx) {
  if (ctx->c.stream) cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.own_stream) {
    cudaStreamSynchronize(ctx->c.own_stream);
    cudaStreamDestroy(ctx->c.own_stream);
  }
  if (ctx->c.pool) cudaMemPoolDestroy(ctx->c.pool);
  delete ctx;
}

// A system counts against its context; a context whose destruction was
// requested while systems were alive is freed with its last system.
void destroy_system(vag_system *sys) {
  if (!sys) return;
  System *s = &sys->s;
  Ctx *c = s->ctx;
  if (c && c->stream) cudaStreamSynchronize(c->stream);
  if (s->pcg_graph) cudaGraphExecDestroy(s->pcg_graph);
  if (s->mx.graph) cudaGraphExecDestroy(s->mx.graph);
  if (s->mx.graph_amg) cudaGraphExecDestroy(s->mx.graph_amg);
  if (s->pcg_graph_amg) cudaGraphExecDestroy(s->pcg_graph_amg);
  if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
  if (s->bicg_graph) cudaGraphExecDestroy(s->bicg_graph);
  if (s->pcg_graph_cheb) cudaGraphExecDestroy(s->pcg_graph_cheb);
  amg_free(s);
  if (s->ks_host) cudaFreeHost(s->ks_host);
  if (s->n_done_host) cudaFreeHost(s->n_done_host);
  if (s->amg_pin) cudaFreeHost(s->amg_pin);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  sys_free_all(s);
  const bool counted = s->counted;
  delete sys;
  if (c && counted) {
    c->live_systems -= 1;
    if (c->destroy_requested && c->live_systems == 0) free_ctx(c->owner);
  }
}

}  // namespace

extern "C" {

vag_status vag_ctx_create(int device, size_t mem_budget_bytes, vag_ctx **out) {
  if (!out) return VAG_EINVAL;
  *out = nullptr;
  std::unique_ptr<vag_ctx> c(new (std::nothrow) vag_ctx());
  if (!c) return VAG_ENOMEM;
  vag_status st = guarded(&c->c, [&] {
    int n = 0;
    VAG_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) fail(VAG_EINVAL, "no such CUDA device");
    c->c.device = device;
    c->c.budget = mem_budget_bytes;
    c->c.owner = c.get();
    VAG_CUDA(cudaSetDevice(device));
    VAG_CUDA(cudaStreamCreateWithFlags(&c->c.own_stream, cudaStreamNonBlocking));
    c->c.stream = c->c.own_stream;
    // a private stream-ordered pool that keeps freed memory for reuse, so
    // systems assembled one after another do not pay for cudaMalloc/cudaFree
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    if (cudaMemPoolCreate(&c->c.pool, &pp) == cudaSuccess) {
      unsigned long long keep = ~0ull;
      cudaMemPoolSetAttribute(c->c.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      c->c.pool = nullptr;   // fall back to cudaMalloc
    }
  });
  if (st != VAG_OK) return st;
  *out = c.release();
  return VAG_OK;
}

void vag_ctx_destroy(vag_ctx *ctx) {
  if (!ctx || ctx->c.destroy_requested) return;
  ctx->c.destroy_requested = true;
  if (ctx->c.live_systems == 0) free_ctx(ctx);
}

vag_status vag_ctx_set_stream(vag_ctx *ctx, void *stream) {
  if (!ctx) return VAG_EINVAL;
  return guarded(&ctx->c, [&] {
    // work (and pool allocations) ordered on the old stream must be complete
    // before the new stream uses or frees them
    VAG_CUDA(cudaStreamSynchronize(ctx->c.stream));
    if (stream == nullptr) {
      ctx->c.stream = ctx->c.own_stream;
      return;
    }
    // the legacy default stream cannot be captured into CUDA graphs
    if (stream == (void *)cudaStreamLegacy || stream == (void *)0)
      fail(VAG_EINVAL, "pass a created stream, not the legacy default stream");
    ctx->c.stream = (cudaStream_t)stream;
  });
}

const char *vag_last_error(const vag_ctx *ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

size_t vag_ctx_bytes_in_use(const vag_ctx *ctx) { return ctx ? ctx->c.in_use : 0; }

unsigned long long vag_launch_count(void) { return launches_so_far(); }

vag_status vag_assemble(vag_ctx *ctx, const vag_mesh *mesh, const vag_props *props, const vag_dirichlet *bc,
                        int mem, vag_system **out) {
  NvtxRange nvtx_range("vag_assemble");
  if (!ctx) return VAG_EINVAL;
  if (out) *out = nullptr;
  std::unique_ptr<vag_system> sys;
  vag_status st = guarded(&ctx->c, [&] {
    if (!mesh || !props || !bc || !out) fail(VAG_EINVAL, "null argument");
    check_mem(mem);
    if (mesh->n_nodes <= 0 || mesh->n_cells <= 0 || mesh->n_ff < 0) fail(VAG_EINVAL, "bad mesh sizes");
    if (bc->n_dir < 0) fail(VAG_EINVAL, "n_dir < 0");
    if (!(props->mu > 0.0)) fail(VAG_EINVAL, "mu must be positive");
    // int32 indices: every control volume, and every cell's 8 node slots and
    // fracture face's 4 node slots, must be addressable
    if ((int64_t)mesh->n_nodes + mesh->n_ff + mesh->n_cells > 0x7fffffffLL || 8LL * mesh->n_cells > 0x7fffffffLL ||
        4LL * mesh->n_ff > 0x7fffffffLL)
      fail(VAG_EINVAL, "mesh too large");
    use_device(&ctx->c);
    sys.reset(new vag_system());
    System *s = &sys->s;
    if (ctx->c.destroy_requested) fail(VAG_EINVAL, "context already destroyed");
    s->ctx = &ctx->c;
    s->counted = true;
    ctx->c.live_systems += 1;
    s->nv = mesh->n_nodes;
    s->nc = mesh->n_cells;
    s->nf = mesh->n_ff;
    s->nd = bc->n_dir;
    s->n_cv = s->nv + s->nf + s->nc;
    s->mu = props->mu;
    VAG_CUDA(cudaEventCreate(&s->ev0));
    VAG_CUDA(cudaEventCreate(&s->ev1));
    trace_mark(s->ctx->stream, "start");
    s->status = sys_alloc<int>(s, 4);
    s->xyz = upload(s, mesh->xyz, 3 * (size_t)s->nv, mem, "xyz");
    if (mesh->cell_nodes) {   // hexahedral fast path
      s->cell_nodes = upload(s, mesh->cell_nodes, 8 * (size_t)s->nc, mem, "cell_nodes");
      s->ff_nodes = upload(s, mesh->ff_nodes, 4 * (size_t)s->nf, mem, "ff_nodes");
    } else {                  // general polyhedral descriptor
      s->cell_nodes = sys_alloc<int>(s, 8 * (size_t)s->nc);
      s->ff_nodes = sys_alloc<int>(s, 4 * (size_t)s->nf);
      int8_t *shape = sys_alloc<int8_t>(s, (size_t)s->nc);
      bool tri = false;
      const unsigned mask = general_to_cells(s->ctx, *mesh, mem, s->cell_nodes, s->ff_nodes, shape, &tri);
      set_shapes(s, shape, mask, tri);
    }
    {
      WellsHost w;
      gather_wells(w, *props, mem, s->nf, 0, s->ctx->stream);
      if (s->nd == 0 && !w.fixes_level)
        fail(VAG_EINVAL, "at least one Dirichlet node or a well perforation with WI > 0 is required");
      upload_wells(s, w);
    }
    s->dir_nodes = upload(s, bc->nodes, (size_t)s->nd, mem, "dirichlet nodes");
    s->dir_vals = upload(s, bc->values, (size_t)s->nd, mem, "dirichlet values");
    s->lam = upload(s, props->lambda_m, 6 * (size_t)s->nc, mem, "lambda_m");
    s->lamf = upload(s, props->lambda_f, (size_t)s->nf, mem, "lambda_f");
    s->df = upload(s, props->d_f, (size_t)s->nf, mem, "d_f");
    Segments &g = s->seg;
    g.n_sys = 1;
    g.node_start = {0, s->nv};
    g.ff_start = {0, s->nf};
    g.cell_start = {0, s->nc};
    g.dir_start = {0, s->nd};
    upload_segments(s);
    trace_mark(s->ctx->stream, "upload");
    symbolic_phase(s);
    trace_mark(s->ctx->stream, "symbolic phase");
    build_tiles(s);
    build_sell(s);
    trace_mark(s->ctx->stream, "row tiles + SELL structure");
    numeric_phase(s);
    trace_mark(s->ctx->stream, "numeric phase");
    trace_report("vag_assemble");
  });
  if (st != VAG_OK) {
    destroy_system(sys.release());
    return st;
  }
  *out = sys.release();
  return VAG_OK;
}

vag_status vag_assemble_batch(vag_ctx *ctx, int32_t n_sys, const vag_mesh *meshes, const vag_props *props,
                              const vag_dirichlet *bcs, int mem, vag_system **out) {
  NvtxRange nvtx_range("vag_assemble_batch");
  if (!ctx) return VAG_EINVAL;
  if (out) *out = nullptr;
  std::unique_ptr<vag_system> sys;
  vag_status st = guarded(&ctx->c, [&] {
    if (!meshes || !props || !bcs || !out || n_sys <= 0) fail(VAG_EINVAL, "null argument or n_sys <= 0");
    check_mem(mem);
    int64_t nv = 0, nc = 0, nf = 0, nd = 0;
    for (int i = 0; i < n_sys; ++i) {
      const vag_mesh &m = meshes[i];
      if (m.n_nodes <= 0 || m.n_cells <= 0 || m.n_ff < 0) fail(VAG_EINVAL, "bad mesh sizes in system " + std::to_string(i));
      if (bcs[i].n_dir < 0) fail(VAG_EINVAL, "system " + std::to_string(i) + ": n_dir < 0");
      if (!(props[i].mu > 0.0)) fail(VAG_EINVAL, "mu must be positive");
      if (props[i].mu != props[0].mu) fail(VAG_EINVAL, "all systems of a batch must share mu");
      nv += m.n_nodes; nc += m.n_cells; nf += m.n_ff; nd += bcs[i].n_dir;
    }
    if (nv + nf + nc > 0x7fffffffLL || 8 * nc > 0x7fffffffLL || 4 * nf > 0x7fffffffLL) fail(VAG_EINVAL, "batch too large");
    use_device(&ctx->c);
    sys.reset(new vag_system());
    System *s = &sys->s;
    if (ctx->c.destroy_requested) fail(VAG_EINVAL, "context already destroyed");
    s->ctx = &ctx->c;
    s->counted = true;
    ctx->c.live_systems += 1;
    s->nv = (int)nv; s->nc = (int)nc; s->nf = (int)nf; s->nd = (int)nd;
    s->n_cv = s->nv + s->nf + s->nc;
    s->mu = props[0].mu;
    VAG_CUDA(cudaEventCreate(&s->ev0));
    VAG_CUDA(cudaEventCreate(&s->ev1));
    s->status = sys_alloc<int>(s, 4);
    Segments &g = s->seg;
    g.n_sys = n_sys;
    g.node_start.assign(n_sys + 1, 0); g.ff_start.assign(n_sys + 1, 0);
    g.cell_start.assign(n_sys + 1, 0); g.dir_start.assign(n_sys + 1, 0);
    for (int i = 0; i < n_sys; ++i) {
      g.node_start[i + 1] = g.node_start[i] + meshes[i].n_nodes;
      g.ff_start[i + 1] = g.ff_start[i] + meshes[i].n_ff;
      g.cell_start[i + 1] = g.cell_start[i] + meshes[i].n_cells;
      g.dir_start[i + 1] = g.dir_start[i] + bcs[i].n_dir;
    }
    s->xyz = sys_alloc<double>(s, 3 * (size_t)nv);
    s->cell_nodes = sys_alloc<int>(s, 8 * (size_t)nc);
    s->ff_nodes = sys_alloc<int>(s, 4 * (size_t)nf);
    s->dir_nodes = sys_alloc<int>(s, (size_t)nd);
    s->dir_vals = sys_alloc<double>(s, (size_t)nd);
    s->lam = sys_alloc<double>(s, 6 * (size_t)nc);
    s->lamf = sys_alloc<double>(s, (size_t)nf);
    s->df = sys_alloc<double>(s, (size_t)nf);
    cudaStream_t str = ctx->c.stream;
    int8_t *shape = sys_alloc<int8_t>(s, (size_t)nc);
    VAG_CUDA(cudaMemsetAsync(shape, 0, (size_t)nc, str));   // topo::HEX == 0
    static_assert(topo::HEX == 0, "fast-path cells are marked by a zero fill");
    unsigned mask = 1u << topo::HEX;
    bool tri = false;
    WellsHost wells;
    for (int i = 0; i < n_sys; ++i) {
      const vag_mesh &m = meshes[i];
      const int v0 = g.node_start[i], c0 = g.cell_start[i], f0 = g.ff_start[i], d0 = g.dir_start[i];
      copy_in(s, s->xyz + 3 * (size_t)v0, m.xyz, 3 * (size_t)m.n_nodes, mem, "xyz");
      if (m.cell_nodes) {
        copy_in(s, s->cell_nodes + 8 * (size_t)c0, m.cell_nodes, 8 * (size_t)m.n_cells, mem, "cell_nodes");
        copy_in(s, s->ff_nodes + 4 * (size_t)f0, m.ff_nodes, 4 * (size_t)m.n_ff, mem, "ff_nodes");
      } else {
        bool t = false;
        mask |= general_to_cells(s->ctx, m, mem, s->cell_nodes + 8 * (size_t)c0, s->ff_nodes + 4 * (size_t)f0,
                                 shape + c0, &t);
        tri = tri || t;
      }
      {   // each system needs its own pressure level
        const bool had = wells.fixes_level;
        wells.fixes_level = false;
        gather_wells(wells, props[i], mem, m.n_ff, f0, str);
        if (bcs[i].n_dir == 0 && !wells.fixes_level)
          fail(VAG_EINVAL, "system " + std::to_string(i) +
                               " has neither a Dirichlet node nor a well perforation with WI > 0");
        wells.fixes_level = wells.fixes_level || had;
      }
      copy_in(s, s->dir_nodes + d0, bcs[i].nodes, (size_t)bcs[i].n_dir, mem, "dirichlet nodes");
      copy_in(s, s->dir_vals + d0, bcs[i].values, (size_t)bcs[i].n_dir, mem, "dirichlet values");
      copy_in(s, s->lam + 6 * (size_t)c0, props[i].lambda_m, 6 * (size_t)m.n_cells, mem, "lambda_m");
      copy_in(s, s->lamf + f0, props[i].lambda_f, (size_t)m.n_ff, mem, "lambda_f");
      copy_in(s, s->df + f0, props[i].d_f, (size_t)m.n_ff, mem, "d_f");
      if (v0) {   // node ids of system i become union ids
        k_add_offset<<<grid_for(8 * (int64_t)m.n_cells, 256), 256, 0, str>>>(s->cell_nodes + 8 * (size_t)c0,
                                                                            8 * (int64_t)m.n_cells, v0);
        if (m.n_ff)
          k_add_offset<<<grid_for(4 * (int64_t)m.n_ff, 256), 256, 0, str>>>(s->ff_nodes + 4 * (size_t)f0,
                                                                           4 * (int64_t)m.n_ff, v0);
        k_add_offset<<<grid_for(bcs[i].n_dir, 256), 256, 0, str>>>(s->dir_nodes + d0, bcs[i].n_dir, v0);
        note_launches(m.n_ff ? 3 : 2);
        VAG_CHECK_LAUNCH();
      }
    }
    set_shapes(s, shape, mask, tri);
    upload_wells(s, wells);
    upload_segments(s);
    symbolic_phase(s);
    build_tiles(s);
    build_sell(s);
    numeric_phase(s);
  });
  if (st != VAG_OK) {
    destroy_system(sys.release());
    return st;
  }
  *out = sys.release();
  return VAG_OK;
}

vag_status vag_system_get_batch(const vag_system *sys, int32_t *n_sys, int32_t *node_start, int32_t *ff_start,
                                int32_t *cell_start, int32_t *row_start) {
  if (!sys) return VAG_EINVAL;
  const Segments &g = sys->s.seg;
  if (n_sys) *n_sys = g.n_sys;
  for (int i = 0; i <= g.n_sys; ++i) {
    if (node_start) node_start[i] = g.node_start[i];
    if (ff_start) ff_start[i] = g.ff_start[i];
    if (cell_start) cell_start[i] = g.cell_start[i];
    if (row_start) row_start[i] = g.row_start[i];
  }
  return VAG_OK;
}

vag_status vag_solve_get_infos(const vag_system *sys, vag_solve_info *infos) {
  if (!sys || !infos) return VAG_EINVAL;
  const System *s = &sys->s;
  if (!s->solved) {
    if (s->ctx) s->ctx->last_error = "no solve yet";
    return VAG_EINVAL;
  }
  solve_infos(s, infos);
  return VAG_OK;
}

vag_status vag_transport_get_dts(const vag_system *sys, double *dt_max, double *dt) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  if (s->dts_host.size() < 2 * (size_t)s->seg.n_sys) {
    if (s->ctx) s->ctx->last_error = "no transport yet";
    return VAG_EINVAL;
  }
  for (int g = 0; g < s->seg.n_sys; ++g) {
    if (dt_max) dt_max[g] = s->dts_host[2 * g];
    if (dt) dt[g] = s->dts_host[2 * g + 1];
  }
  return VAG_OK;
}

vag_status vag_update_props(vag_system *sys, const vag_props *props, int mem) {
  NvtxRange nvtx_range("vag_update_props");
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  return guarded(s->ctx, [&] {
    if (!props) fail(VAG_EINVAL, "null props");
    check_mem(mem);
    if (!(props->mu > 0.0)) fail(VAG_EINVAL, "mu must be positive");
    use_device(s->ctx);
    copy_in(s, s->lam, props->lambda_m, 6 * (size_t)s->nc, mem, "lambda_m");
    copy_in(s, s->lamf, props->lambda_f, (size_t)s->nf, mem, "lambda_f");
    copy_in(s, s->df, props->d_f, (size_t)s->nf, mem, "d_f");
    WellsHost w;
    gather_wells(w, *props, mem, s->nf, 0, s->ctx->stream);
    if (s->nd == 0 && !w.fixes_level)
      fail(VAG_EINVAL, "at least one Dirichlet node or a well perforation with WI > 0 is required");
    upload_wells(s, w);
    s->mu = props->mu;
    numeric_phase(s);
    s->solved = false;
    s->have_flux = false;
  });
}

vag_status vag_peaceman_wi(int32_t n, const double *dx, const double *dz, const double *d_f,
                           const double *lambda_f, const double *r_w, double mu, double *wi_out) {
  if (n < 0 || (n > 0 && (!dx || !dz || !d_f || !lambda_f || !r_w || !wi_out)) || !(mu > 0.0)) return VAG_EINVAL;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> wi((size_t)n);
  for (int32_t i = 0; i < n; ++i) {
    const double a = dx[i], h = dz[i], w = d_f[i];
    if (!(a > 0.0) || !(h > 0.0) || !(w > 0.0) || !(lambda_f[i] > 0.0) || !(r_w[i] > 0.0)) return VAG_EINVAL;
    const double C = (4.0 / 3.0) * (a * h / w + a * w / h + h * w / a);
    const double D = 0.5 * std::sqrt(a * a + w * w);
    const double lr = std::log(D / r_w[i]) - two_pi * h / C;   // log(r_0 / r_w)
    if (!(lr > 0.0)) return VAG_EINVAL;
    wi[(size_t)i] = two_pi * h * lambda_f[i] / (mu * lr);
  }
  std::copy(wi.begin(), wi.end(), wi_out);
  return VAG_OK;
}

void vag_system_destroy(vag_system *sys) { destroy_system(sys); }

vag_status vag_system_get_info(const vag_system *sys, vag_system_info *info) {
  if (!sys || !info) return VAG_EINVAL;
  const System *s = &sys->s;
  info->n_nodes = s->nv;
  info->n_cells = s->nc;
  info->n_ff = s->nf;
  info->n_dir = s->nd;
  info->n_rows = s->n_rows;
  info->nnz = s->nnz;
  info->n_frac_cells = s->n_fc;
  info->n_cv = s->n_cv;
  info->nnz_transport = s->nnz_t;
  info->device_bytes = s->bytes;
  return VAG_OK;
}

vag_status vag_solve(vag_system *sys, const vag_solve_opts *opts, double *u_out, vag_solve_info *info) {
  NvtxRange nvtx_range("vag_solve");
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  vag_solve_info local{};
  vag_solve_info *inf = info ? info : &local;
  vag_status st = guarded(s->ctx, [&] {
    if (!opts) fail(VAG_EINVAL, "null options");
    check_mem(opts->mem);
    if (!(opts->rtol > 0.0) || opts->maxit <= 0) fail(VAG_EINVAL, "rtol must be > 0 and maxit > 0");
    if (opts->precision != VAG_FP64 && opts->precision != VAG_MIXED && opts->precision != VAG_MIXED_F16 &&
        opts->precision != VAG_FP64_PC32)
      fail(VAG_EINVAL, "unknown precision");
    const bool amg = opts->precond == VAG_PC_AMG || opts->precond == VAG_PC_AMG_RS;
    if (opts->precision == VAG_MIXED_F16 && opts->precond != VAG_PC_AMG)
      fail(VAG_EINVAL, "VAG_MIXED_F16 stores the aggregation AMG finest level in FP16: it needs VAG_PC_AMG");
    if (opts->precision == VAG_FP64_PC32 && !amg)
      fail(VAG_EINVAL, "VAG_FP64_PC32 preconditions by the FP32 AMG hierarchy: it needs an AMG preconditioner");
    if (!(opts->inner_rtol >= 0.0 && opts->inner_rtol < 1.0)) fail(VAG_EINVAL, "inner_rtol must be in [0, 1)");
    if (opts->precond != VAG_PC_JACOBI && opts->precond != VAG_PC_CHEBYSHEV && !amg)
      fail(VAG_EINVAL, "unknown preconditioner");
    if (opts->precond == VAG_PC_CHEBYSHEV && opts->precision != VAG_FP64)
      fail(VAG_EINVAL, "VAG_PC_CHEBYSHEV runs in FP64 only");
    use_device(s->ctx);
    trace_mark(s->ctx->stream, "start");
    // VAG_MIXED(_F16): FP64 refinement around FP32 CG (Jacobi: on the scaled
    // system; AMG: preconditioned by the FP32 hierarchy); VAG_FP64_PC32: FP64
    // CG preconditioned by the FP32 hierarchy
    if (opts->krylov != VAG_KRYLOV_CG && opts->krylov != VAG_KRYLOV_BICGSTAB && opts->krylov != VAG_KRYLOV_GMRES)
      fail(VAG_EINVAL, "unknown Krylov method");
    if (opts->krylov == VAG_KRYLOV_BICGSTAB) {
      if (opts->precision == VAG_MIXED && !amg) fail(VAG_EINVAL, "BiCGStab with VAG_MIXED needs an AMG preconditioner");
      bicgstab_solve(s, opts, inf);
    } else if (opts->krylov == VAG_KRYLOV_GMRES) {
      if (opts->precision == VAG_MIXED && !amg) fail(VAG_EINVAL, "GMRES with VAG_MIXED needs an AMG preconditioner");
      gmres_solve(s, opts, inf);
    } else if (opts->precision == VAG_MIXED && opts->precond == VAG_PC_JACOBI) {
      mixed_solve(s, opts, inf);
    } else if ((opts->precision == VAG_MIXED || opts->precision == VAG_MIXED_F16) && amg) {
      mixed_amg_solve(s, opts, inf);
    } else {
      pcg_solve(s, opts, inf);
    }
    copy_out(s, u_out, s->u, (size_t)s->n_cv, opts->mem);
    trace_mark(s->ctx->stream, "copy out");
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
    trace_report("vag_solve");
    if (inf->status == VAG_EBREAKDOWN) fail(VAG_EBREAKDOWN, "CG breakdown: p^T A p <= 0 or NaN");
    if (inf->status == VAG_ENOTCONVERGED)
      fail(VAG_ENOTCONVERGED, "CG reached maxit above rtol (last iterate written)");
  });
  return st;
}

vag_status vag_kernel_time(vag_system *sys, int kernel, int32_t reps, double *ms_per_launch) {
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  return guarded(s->ctx, [&] {
    if (!ms_per_launch || reps < 1) fail(VAG_EINVAL, "null output or reps < 1");
    use_device(s->ctx);
    switch (kernel) {
      case VAG_KERNEL_SPMV: *ms_per_launch = time_spmv(s, reps); break;
      case VAG_KERNEL_SMOOTH: *ms_per_launch = time_smoother(s, reps); break;
      case VAG_KERNEL_TRANSPORT_STEP: *ms_per_launch = time_transport_step(s, reps); break;
      case VAG_KERNEL_SPMV32: *ms_per_launch = time_spmv32(s, reps); break;
      case VAG_KERNEL_CELL_LOCAL: *ms_per_launch = time_cell_local(s, reps); break;
      default: fail(VAG_EINVAL, "unknown kernel");
    }
    VAG_CHECK_LAUNCH();
  });
}

vag_status vag_spmv(vag_system *sys, const double *x, double *y, int mem) {
  NvtxRange nvtx_range("vag_spmv");
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  return guarded(s->ctx, [&] {
    if (!x || !y) fail(VAG_EINVAL, "null vector");
    check_mem(mem);
    use_device(s->ctx);
    cudaStream_t st = s->ctx->stream;
    if (mem == VAG_MEM_DEVICE) {
      spmv_f64(s, x, y);   // stream-ordered: no host synchronisation
      return;
    } else {
      double *dx, *dy;
      const size_t n = s->n_rows;
      VAG_CUDA(cudaMallocAsync(&dx, sizeof(double) * n, st));
      VAG_CUDA(cudaMallocAsync(&dy, sizeof(double) * n, st));
      VAG_CUDA(cudaMemcpyAsync(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice, st));
      spmv_f64(s, dx, dy);
      VAG_CUDA(cudaMemcpyAsync(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
      VAG_CUDA(cudaFreeAsync(dx, st));
      VAG_CUDA(cudaFreeAsync(dy, st));
    }
    VAG_CUDA(cudaStreamSynchronize(st));
  });
}

vag_status vag_transport(vag_system *sys, const vag_transport_opts *o, double *c_inout, vag_transport_info *info) {
  NvtxRange nvtx_range("vag_transport");
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  vag_transport_info local{};
  vag_transport_info *inf = info ? info : &local;
  return guarded(s->ctx, [&] {
    if (!o || !c_inout) fail(VAG_EINVAL, "null argument");
    check_mem(o->mem);
    if (!s->have_flux) fail(VAG_EINVAL, "no fluxes: call vag_solve or vag_set_fluxes first");
    if (o->n_steps < 0) fail(VAG_EINVAL, "n_steps < 0");
    if (!(o->omega >= 0.0 && o->omega < 1.0)) fail(VAG_EINVAL, "omega must be in [0, 1)");
    if (!(o->cfl > 0.0) && !(o->dt > 0.0)) fail(VAG_EINVAL, "give cfl > 0 or dt > 0");
    use_device(s->ctx);
    cudaStream_t st = s->ctx->stream;
    trace_mark(st, "start");
    const size_t n = s->n_cv;
    // stage porosities, cbar and c
    if (!o->phi_m || (s->nf && !o->phi_f) || (s->nd && !o->cbar)) fail(VAG_EINVAL, "null porosity or cbar");
    double *stage;
    const size_t tot = (size_t)s->nc + s->nf + s->nd + (o->mem == VAG_MEM_HOST ? n : 0);
    VAG_CUDA(cudaMallocAsync(&stage, sizeof(double) * (tot ? tot : 1), st));
    double *pm = stage, *pf = stage + s->nc, *cb = pf + s->nf;
    VAG_CUDA(cudaMemcpyAsync(pm, o->phi_m, sizeof(double) * s->nc, to_dev(o->mem), st));
    if (s->nf) VAG_CUDA(cudaMemcpyAsync(pf, o->phi_f, sizeof(double) * s->nf, to_dev(o->mem), st));
    VAG_CUDA(cudaMemcpyAsync(cb, o->cbar, sizeof(double) * s->nd, to_dev(o->mem), st));
    double *cdev = c_inout;
    if (o->mem == VAG_MEM_HOST) {
      cdev = cb + s->nd;
      VAG_CUDA(cudaMemcpyAsync(cdev, c_inout, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    try {
      transport_run(s, o, cdev, inf, pm, pf, cb);
    } catch (...) {
      cudaFreeAsync(stage, st);
      throw;
    }
    if (o->mem == VAG_MEM_HOST)
      VAG_CUDA(cudaMemcpyAsync(c_inout, cdev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaFreeAsync(stage, st));
    trace_mark(st, "copy out");
    VAG_CUDA(cudaStreamSynchronize(st));
    trace_report("vag_transport");
  });
}

vag_status vag_transport_step(vag_system *sys, const vag_transport_opts *opts, double *c_inout, double *dt_used,
                              vag_transport_info *info) {
  vag_transport_info local{};
  vag_transport_info *inf = info ? info : &local;
  const vag_status st = vag_transport(sys, opts, c_inout, inf);
  if (st == VAG_OK && dt_used) *dt_used = inf->dt;
  return st;
}

vag_status vag_export_system(const vag_system *sys, int32_t *rowptr, int32_t *col, double *val, double *rhs,
                             int32_t *row_dof, int mem) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    use_device(s->ctx);
    copy_out(s, rowptr, s->rowptr, (size_t)s->n_rows + 1, mem);
    copy_out(s, col, s->col, (size_t)s->nnz, mem);
    copy_out(s, val, s->val, (size_t)s->nnz, mem);
    copy_out(s, rhs, s->rhs, (size_t)s->n_rows, mem);
    copy_out(s, row_dof, s->dof_of_row, (size_t)s->n_rows, mem);
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  });
}

vag_status vag_export_fluxes(const vag_system *sys, double *Fcn, double *Fcf, double *Fff, int mem) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    if (!s->have_flux) fail(VAG_EINVAL, "no fluxes yet");
    use_device(s->ctx);
    copy_out(s, Fcn, s->Fcn, 8 * (size_t)s->nc, mem);
    copy_out(s, Fcf, s->Fcf, 6 * (size_t)s->nc, mem);
    copy_out(s, Fff, s->Fff, 4 * (size_t)s->nf, mem);
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  });
}

vag_status vag_export_cells(const vag_system *sys, int32_t *cell_nodes, int8_t *shape, int32_t *ff_nodes, int mem) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    use_device(s->ctx);
    if (cell_nodes) copy_out(s, cell_nodes, s->cell_nodes, 8 * (size_t)s->nc, mem);
    if (ff_nodes) copy_out(s, ff_nodes, s->ff_nodes, 4 * (size_t)s->nf, mem);
    if (shape) {
      if (s->cell_shape) {
        copy_out(s, shape, s->cell_shape, (size_t)s->nc, mem);
      } else if (mem == VAG_MEM_HOST) {
        std::memset(shape, topo::HEX, (size_t)s->nc);
      } else {
        VAG_CUDA(cudaMemsetAsync(shape, topo::HEX, (size_t)s->nc, s->ctx->stream));
      }
    }
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  });
}

vag_status vag_export_well_rates(const vag_system *sys, double *Fw, int mem) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    if (s->n_perf && !Fw) fail(VAG_EINVAL, "null array");
    use_device(s->ctx);
    copy_out(s, Fw, s->Fw, (size_t)s->n_perf, mem);
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  });
}

vag_status vag_set_fluxes(vag_system *sys, const double *Fcn, const double *Fcf, const double *Fff, int mem) {
  if (!sys) return VAG_EINVAL;
  System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    if (!Fcn || !Fcf || (s->nf && !Fff)) fail(VAG_EINVAL, "null flux array");
    use_device(s->ctx);
    if (!s->Fcn) {
      s->Fcn = sys_alloc<double>(s, 8 * (size_t)s->nc);
      s->Fcf = sys_alloc<double>(s, 6 * (size_t)s->nc);
      s->Fff = sys_alloc<double>(s, 4 * (size_t)(s->nf > 0 ? s->nf : 1));
    }
    copy_in(s, s->Fcn, Fcn, 8 * (size_t)s->nc, mem, "F_cell_nodes");
    copy_in(s, s->Fcf, Fcf, 6 * (size_t)s->nc, mem, "F_cell_faces");
    copy_in(s, s->Fff, Fff, 4 * (size_t)s->nf, mem, "F_frac");
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
    s->have_flux = true;
  });
}

vag_status vag_export_porous_volumes(const vag_system *sys, double *phi, int mem) {
  if (!sys) return VAG_EINVAL;
  const System *s = &sys->s;
  return guarded(s->ctx, [&] {
    check_mem(mem);
    if (!s->phi) fail(VAG_EINVAL, "no porous volumes yet: call vag_transport first");
    use_device(s->ctx);
    copy_out(s, phi, s->phi, (size_t)s->n_cv, mem);
    VAG_CUDA(cudaStreamSynchronize(s->ctx->stream));
  });
}

}  // extern "C"
