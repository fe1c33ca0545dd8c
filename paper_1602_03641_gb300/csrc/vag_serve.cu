// Request server: continuous batching of Darcy + transport requests.
//
// Each worker ("slot") owns a context (stream + memory pool) on the device.
// A free slot takes the oldest queued request and every other queued request
// with the same solver settings, as long as their estimated device memory
// fits what the budget has left, assembles them as one batch (disjoint
// union), solves, runs the transport steps and completes them.  Requests that
// arrive while batches are on the GPU wait only for the next free slot, and
// batches of different slots overlap on the device.  A request's result does
// not depend on the batch it lands in (see vag_assemble_batch).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "vag_cellmap.h"
#include "vag_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  // copies of the caller's inputs
  std::vector<double> xyz, lam, lamf, df, dirv, phim, phif, cbar, c0;
  std::vector<int32_t> cn, ffn, dirn;
  // the general descriptor, kept as given (validated at submit)
  bool general = false;
  int32_t n_cells = 0, n_ff = 0, n_faces = 0;
  std::vector<int32_t> fptr, fidx, cptr, cidx, ffid;
  // wells
  std::vector<int32_t> wff;
  std::vector<double> wwi, wpw, wq, wcin;
  double mu = 1.0, omega = 0.5, cfl = 0.9, rtol = 1e-8;
  int32_t n_steps = 0, maxit = 1000;
  int precision = VAG_FP64, precond = VAG_PC_JACOBI;
  double *u_out = nullptr, *c_out = nullptr;
  size_t est = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  vag_result res{};
  int32_t nv() const { return (int32_t)(xyz.size() / 3); }
  int32_t nc() const { return n_cells; }
  int32_t nf() const { return n_ff; }
  bool same_settings(const Req &o) const {
    return precision == o.precision && precond == o.precond && rtol == o.rtol && maxit == o.maxit &&
           n_steps == o.n_steps && omega == o.omega && cfl == o.cfl && mu == o.mu;
  }
};

// Device bytes a request needs while its batch runs (system, Krylov and
// transport buffers, plus the AMG hierarchy when used), with margin.
size_t estimate_bytes(const Req &r) {
  const double nc = r.nc(), nv = r.nv(), nf = r.nf();
  double b = 1400.0 * nc + 900.0 * nv + 1200.0 * nf;
  if (r.precond == VAG_PC_AMG) b *= 1.6;
  if (r.precond == VAG_PC_AMG_RS) b *= 2.2;   // denser coarse levels and P, R
  if (r.precond == VAG_PC_CHEBYSHEV) b *= 1.05;   // four more row vectors
  if (r.precision != VAG_FP64) b *= 1.25;
  return (size_t)(b * 1.2) + (1u << 20);
}

}  // namespace

struct vag_server {
  vag_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::map<uint64_t, std::shared_ptr<Req>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t reserved = 0, peak = 0;
  uint64_t submitted = 0, completed = 0, rejected = 0, in_flight = 0;
  std::vector<double> latencies;   // ms, completed requests
  Clock::time_point t_first_submit{}, t_last_done{};
  bool any_submit = false;
  std::vector<std::thread> workers;
  std::string last_error;

  void worker(int slot);
  void run_batch(vag_ctx *ctx, std::vector<std::shared_ptr<Req>> &batch);
};

void vag_server::run_batch(vag_ctx *ctx, std::vector<std::shared_ptr<Req>> &batch) {
  const int n = (int)batch.size();
  std::vector<vag_mesh> meshes(n);
  std::vector<vag_props> props(n);
  std::vector<vag_dirichlet> bcs(n);
  for (int i = 0; i < n; ++i) {
    Req &r = *batch[i];
    if (r.general)
      meshes[i] = vag_mesh{r.nv(), r.xyz.data(), r.nc(), nullptr, r.nf(), nullptr, r.n_faces, r.fptr.data(),
                           r.fidx.data(), r.cptr.data(), r.cidx.data(), r.ffid.data()};
    else
      meshes[i] = vag_mesh{r.nv(), r.xyz.data(), r.nc(), r.cn.data(), r.nf(), r.ffn.data()};
    props[i] = vag_props{r.lam.data(), r.lamf.data(), r.df.data(), r.mu, (int32_t)r.wff.size(), r.wff.data(),
                         r.wwi.data(), r.wpw.data(), r.wq.data(), r.wcin.data()};
    bcs[i] = vag_dirichlet{(int32_t)r.dirn.size(), r.dirn.data(), r.dirv.data()};
  }
  const Req &r0 = *batch[0];
  vag_system *sys = nullptr;
  vag_status st = vag_assemble_batch(ctx, n, meshes.data(), props.data(), bcs.data(), VAG_MEM_HOST, &sys);
  std::vector<vag_solve_info> infos(n);
  std::vector<double> u, c, dtmax(n), dt(n);
  std::vector<int32_t> ns(n + 1), fs(n + 1), cs(n + 1);
  vag_solve_info agg{};
  vag_transport_info tinf{};
  if (st == VAG_OK) {
    vag_system_info si{};
    vag_system_get_info(sys, &si);
    vag_system_get_batch(sys, nullptr, ns.data(), fs.data(), cs.data(), nullptr);
    u.resize(si.n_cv);
    vag_solve_opts so{r0.precision, r0.precond, r0.rtol, r0.maxit, VAG_MEM_HOST, VAG_KRYLOV_CG, 0.0};
    st = vag_solve(sys, &so, u.data(), &agg);
    if (st == VAG_OK || st == VAG_ENOTCONVERGED) vag_solve_get_infos(sys, infos.data());
    if (st == VAG_OK && r0.n_steps > 0) {
      const int NV = ns[n], NF = fs[n];
      std::vector<double> phim, phif, cbar;
      c.assign(si.n_cv, 0.0);
      for (int i = 0; i < n; ++i) {
        Req &r = *batch[i];
        phim.insert(phim.end(), r.phim.begin(), r.phim.end());
        phif.insert(phif.end(), r.phif.begin(), r.phif.end());
        cbar.insert(cbar.end(), r.cbar.begin(), r.cbar.end());
        if (!r.c0.empty()) {   // caller's c^0 in its own [nodes | ffaces | cells] order
          std::copy(r.c0.begin(), r.c0.begin() + r.nv(), c.begin() + ns[i]);
          std::copy(r.c0.begin() + r.nv(), r.c0.begin() + r.nv() + r.nf(), c.begin() + NV + fs[i]);
          std::copy(r.c0.begin() + r.nv() + r.nf(), r.c0.end(), c.begin() + NV + NF + cs[i]);
        }
      }
      vag_transport_opts to{phim.data(), phif.data(), cbar.data(), r0.omega, r0.cfl, 0.0, r0.n_steps, VAG_MEM_HOST};
      st = vag_transport(sys, &to, c.data(), &tinf);
      if (st == VAG_OK) vag_transport_get_dts(sys, dtmax.data(), dt.data());
    }
  }
  const std::string err = st == VAG_OK ? "" : vag_last_error(ctx);
  // results back into the callers' buffers, system by system
  if (sys && (st == VAG_OK || st == VAG_ENOTCONVERGED)) {
    const int NV = ns[n], NF = fs[n];
    for (int i = 0; i < n; ++i) {
      Req &r = *batch[i];
      auto put = [&](const std::vector<double> &src, double *dst) {
        if (!dst || src.empty()) return;
        std::copy(src.begin() + ns[i], src.begin() + ns[i + 1], dst);
        std::copy(src.begin() + NV + fs[i], src.begin() + NV + fs[i + 1], dst + r.nv());
        std::copy(src.begin() + NV + NF + cs[i], src.begin() + NV + NF + cs[i + 1], dst + r.nv() + r.nf());
      };
      put(u, r.u_out);
      if (r.n_steps > 0 && st == VAG_OK) put(c, r.c_out);
    }
  }
  if (sys) vag_system_destroy(sys);
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n; ++i) {
    Req &r = *batch[i];
    r.res.status = st;
    r.res.solve = infos[i];
    r.res.transport = tinf;
    r.res.transport.dt_max = dtmax[i];
    r.res.transport.dt = dt[i];
    r.res.batch_size = n;
    r.t_done = now;
    r.res.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
    r.res.queue_ms = std::chrono::duration<double, std::milli>(r.t_start - r.t_submit).count();
    r.done = true;
    reserved -= r.est;
    latencies.push_back(r.res.latency_ms);
    ++completed;
    --in_flight;
  }
  if (!err.empty()) last_error = err;
  t_last_done = now;
  cv_done.notify_all();
  cv_work.notify_all();   // memory came back
}

void vag_server::worker(int slot) {
  vag_ctx *ctx = nullptr;
  if (vag_ctx_create(opts.device, 0, &ctx) != VAG_OK) return;
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    {
      std::unique_lock<std::mutex> lock(mu);
      for (;;) {
        if (stop) break;
        if (!queue.empty()) {
          const size_t budget = opts.mem_budget_bytes;
          const auto &head = queue.front();
          if (!budget || reserved + head->est <= budget || in_flight == 0) break;
        }
        cv_work.wait(lock);
      }
      if (stop) break;
      // the oldest request and every compatible one that still fits
      const size_t budget = opts.mem_budget_bytes;
      auto head = queue.front();
      size_t take = 0;
      for (auto it = queue.begin(); it != queue.end() && (int)batch.size() < opts.max_batch;) {
        Req &r = **it;
        const bool fits = !budget || reserved + take + r.est <= budget || batch.empty();
        if (r.same_settings(*head) && fits) {
          take += r.est;
          batch.push_back(*it);
          it = queue.erase(it);
        } else {
          ++it;
        }
      }
      reserved += take;
      peak = std::max(peak, reserved);
      in_flight += batch.size();
      const auto now = Clock::now();
      for (auto &r : batch) r->t_start = now;
    }
    run_batch(ctx, batch);
  }
  vag_ctx_destroy(ctx);
  (void)slot;
}

extern "C" {

vag_status vag_server_create(const vag_server_opts *opts, vag_server **out) {
  if (!opts || !out) return VAG_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || opts->device < 0 || opts->device >= n) {
    cudaGetLastError();
    return VAG_ECUDA;
  }
  std::unique_ptr<vag_server> s(new (std::nothrow) vag_server());
  if (!s) return VAG_ENOMEM;
  s->opts = *opts;
  if (s->opts.slots <= 0) s->opts.slots = 2;
  if (s->opts.max_batch <= 0) s->opts.max_batch = 64;
  for (int i = 0; i < s->opts.slots; ++i) s->workers.emplace_back(&vag_server::worker, s.get(), i);
  *out = s.release();
  return VAG_OK;
}

vag_status vag_server_submit(vag_server *s, const vag_request *q, uint64_t *ticket) {
  if (!s || !q || !ticket) return VAG_EINVAL;
  const vag_mesh &m = q->mesh;
  const bool general = !m.cell_nodes;
  const vag_props &pp = q->props;
  if (pp.n_perf < 0 || (pp.n_perf > 0 && (!pp.well_ff || !pp.well_wi || !pp.well_pw || !pp.well_q || !pp.well_cin)))
    return VAG_EINVAL;
  bool level = q->bc.n_dir > 0;   // the pressure level is fixed by a Dirichlet node or a producing well
  for (int32_t i = 0; i < pp.n_perf; ++i) level = level || pp.well_wi[i] > 0.0;
  if (m.n_nodes <= 0 || m.n_cells <= 0 || m.n_ff < 0 || q->bc.n_dir < 0 || !level || !(q->props.mu > 0.0) ||
      !m.xyz || (!general && m.n_ff && !m.ff_nodes) ||
      (general && (m.n_faces <= 0 || !m.face_node_ptr || !m.face_node_idx || !m.cell_face_ptr ||
                   !m.cell_face_idx || (m.n_ff && !m.ff_face_ids))) ||
      !q->props.lambda_m ||
      (m.n_ff && (!q->props.lambda_f || !q->props.d_f)) || (q->bc.n_dir && (!q->bc.nodes || !q->bc.values)) ||
      q->n_steps < 0 || (q->n_steps > 0 && (!q->phi_m || (m.n_ff && !q->phi_f) || (q->bc.n_dir && !q->cbar))) || !(q->rtol > 0.0) || q->maxit <= 0)
    return VAG_EINVAL;
  auto r = std::make_shared<Req>();
  const size_t nv = m.n_nodes, nc = m.n_cells, nf = m.n_ff, nd = q->bc.n_dir;
  r->xyz.assign(m.xyz, m.xyz + 3 * nv);
  r->n_cells = m.n_cells;
  r->n_ff = m.n_ff;
  if (!general) {
    r->cn.assign(m.cell_nodes, m.cell_nodes + 8 * nc);
    if (nf) r->ffn.assign(m.ff_nodes, m.ff_nodes + 4 * nf);
  } else {   // the general descriptor: validated here (vag_cellmap.h), converted on the device
    const int64_t flen = m.face_node_ptr[m.n_faces], clen = m.cell_face_ptr[m.n_cells];
    if (flen < 0 || clen < 0) return VAG_EINVAL;
    int32_t out[8];
    int sh = 0;
    for (size_t K = 0; K < nc; ++K) {
      const int e = vag::cell_from_faces(m.face_node_ptr, m.face_node_idx, flen, m.cell_face_ptr, m.cell_face_idx,
                                         clen, m.n_faces, m.n_nodes, (int32_t)K, out, &sh);
      if (e != vag::HEXMAP_OK) return e == vag::HEXMAP_BAD_INDEX ? VAG_EINVAL : VAG_EMESH;
    }
    for (size_t i = 0; i < nf; ++i) {
      const int e = vag::face_nodes_of(m.face_node_ptr, m.face_node_idx, flen, m.n_faces, m.n_nodes,
                                       m.ff_face_ids[i], out);
      if (e != vag::HEXMAP_OK) return e == vag::HEXMAP_BAD_INDEX ? VAG_EINVAL : VAG_EMESH;
    }
    r->general = true;
    r->n_faces = m.n_faces;
    r->fptr.assign(m.face_node_ptr, m.face_node_ptr + m.n_faces + 1);
    r->fidx.assign(m.face_node_idx, m.face_node_idx + flen);
    r->cptr.assign(m.cell_face_ptr, m.cell_face_ptr + m.n_cells + 1);
    r->cidx.assign(m.cell_face_idx, m.cell_face_idx + clen);
    r->ffid.assign(m.ff_face_ids, m.ff_face_ids + nf);
  }
  if (pp.n_perf > 0) {
    r->wff.assign(pp.well_ff, pp.well_ff + pp.n_perf);
    r->wwi.assign(pp.well_wi, pp.well_wi + pp.n_perf);
    r->wpw.assign(pp.well_pw, pp.well_pw + pp.n_perf);
    r->wq.assign(pp.well_q, pp.well_q + pp.n_perf);
    r->wcin.assign(pp.well_cin, pp.well_cin + pp.n_perf);
  }
  r->lam.assign(q->props.lambda_m, q->props.lambda_m + 6 * nc);
  if (nf) {
    r->lamf.assign(q->props.lambda_f, q->props.lambda_f + nf);
    r->df.assign(q->props.d_f, q->props.d_f + nf);
  }
  r->dirn.assign(q->bc.nodes, q->bc.nodes + nd);
  r->dirv.assign(q->bc.values, q->bc.values + nd);
  if (q->n_steps > 0) {
    r->phim.assign(q->phi_m, q->phi_m + nc);
    if (nf) r->phif.assign(q->phi_f, q->phi_f + nf);
    r->cbar.assign(q->cbar, q->cbar + nd);
    if (q->c0) r->c0.assign(q->c0, q->c0 + nv + nf + nc);
  }
  r->mu = q->props.mu;
  r->omega = q->omega;
  r->cfl = q->cfl;
  r->n_steps = q->n_steps;
  r->precision = q->precision;
  r->precond = q->precond;
  r->rtol = q->rtol;
  r->maxit = q->maxit;
  r->u_out = q->u_out;
  r->c_out = q->c_out;
  r->est = estimate_bytes(*r);
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return VAG_EINVAL;
  if (s->opts.mem_budget_bytes && r->est > s->opts.mem_budget_bytes) {
    ++s->rejected;
    s->last_error = "request needs more device memory than the server budget";
    return VAG_EBUDGET;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = Clock::now();
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first_submit = r->t_submit;
  }
  s->queue.push_back(r);
  s->all[r->ticket] = r;
  ++s->submitted;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return VAG_OK;
}

vag_status vag_server_wait(vag_server *s, uint64_t ticket, int32_t timeout_ms, vag_result *out) {
  if (!s) return VAG_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return VAG_EINVAL;
  std::shared_ptr<Req> r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lock, pred);
  } else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) {
    return VAG_ETIMEOUT;
  }
  if (out) *out = r->res;
  s->all.erase(ticket);
  return VAG_OK;
}

vag_status vag_server_get_stats(vag_server *s, vag_server_stats *st) {
  if (!s || !st) return VAG_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  *st = vag_server_stats{};
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->rejected = s->rejected;
  st->in_queue = s->queue.size();
  st->in_flight = s->in_flight;
  st->bytes_reserved = s->reserved;
  st->peak_bytes = s->peak;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    const double span = std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count();
    st->solves_per_s = span > 0 ? s->completed / span : 0.0;
  }
  return VAG_OK;
}

const char *vag_server_last_error(const vag_server *s) { return s ? s->last_error.c_str() : "null server"; }

void vag_server_destroy(vag_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    // queued requests are cancelled
    for (auto &r : s->queue) {
      r->res.status = VAG_ETIMEOUT;
      r->done = true;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  s->cv_done.notify_all();
  delete s;
}

}  // extern "C"
