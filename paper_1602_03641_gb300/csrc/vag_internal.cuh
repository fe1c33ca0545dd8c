// Internal declarations of the VAG CUDA library (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "vag.h"

struct vag_ctx;

namespace vag {

// --------------------------------------------------------------- errors ----
struct Error {
  vag_status code;
  std::string msg;
};

[[noreturn]] inline void fail(vag_status code, const std::string &msg) { throw Error{code, msg}; }

#define VAG_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      ::vag::fail(VAG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

#define VAG_CHECK_LAUNCH() VAG_CUDA(cudaGetLastError())

// Device status bits (atomicOr'ed by kernels, read by the host).
enum : int {
  ST_BAD_INDEX = 1,        // an index outside its range
  ST_DUP_DIRICHLET = 2,    // a Dirichlet node listed twice
  ST_DUP_FFACE = 4,        // a fracture face listed twice
  ST_FFACE_NOT_FACE = 8,   // a fracture face that is no cell face
  ST_FACE_3CELLS = 16,     // a face shared by more than two cells
  ST_ROW_OVERFLOW = 32,    // a CSR row wider than the kernel's bound
  ST_HASH_FULL = 64,       // the fracture-face table overflowed
  ST_BAD_GEOMETRY = 128,   // a degenerate sub-tetrahedron or triangle
  ST_NONPOSITIVE = 256,    // a non-positive diagonal / porous volume
  ST_ISOLATED = 512,       // an unknown coupled to nothing (no diagonal)
  ST_NO_SLOT = 1024,       // a contribution without a CSR slot
  ST_TAIL_SMEM = 2048,     // a system's tail levels exceed the shared-memory plan
  ST_WAIT_TIMEOUT = 4096,  // a bounded barrier wait gave up
};

constexpr int kMaxRowWidth = 160;   // unique columns of one eliminated row
constexpr int kMaxRedBlocks = 4096; // blocks of a reduction kernel

// ------------------------------------------------------------ context ------
struct Ctx {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  int live_systems = 0;        // systems created from this context and not yet destroyed
  bool destroy_requested = false;
  struct ::vag_ctx *owner = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;   // stream-ordered pool for every device buffer of the context's systems
  std::string last_error;
  // autotuned loads in flight of the sliced-ELL row loop, per matrix size
  // class (floor(log2 rows)); see tune_sell
  std::vector<int> sell_unroll = std::vector<int>(32, 0);
};

// One device allocation owned by a system.
struct Alloc {
  void *ptr;
  size_t bytes;
};

// Krylov scalars kept on the device, one set per system of a batch.
struct KrylovScalars {
  double rz, pq, alpha, beta, rr, bb, tol2, res2;
  int iter, maxit, done, breakdown;
  int inner_total;             // mixed precision: inner iterations summed over refinements
  int stalled;                 // true residual stopped falling (rounding floor)
  double omega;                // BiCGStab: omega; rz holds rho = r0^.r, pq holds r0^.v
  int half;                    // BiCGStab: converged on s within the current iteration
};

// One level of the aggregation AMG hierarchy (level 0 aliases the system).
struct AmgLevel {
  int n = 0;
  int64_t nnz = 0;
  int *rowptr = nullptr, *col = nullptr;
  double *val = nullptr, *dinv = nullptr;
  double *sinv = nullptr;          // [n] smoother scaling 1 / sum_j |a_ij| (l1-Jacobi)
  std::vector<int> sys_start;      // host, n_sys+1: first row of each system
  int *d_sys_start = nullptr;
  std::vector<int> nz_start;       // host, n_sys+1: first nonzero of each system
  int *d_nz_start = nullptr;
  int *agg = nullptr;              // [n] aggregate (row of the next level) or -1
  // systems that end their hierarchy at this level (at most kDenseMax rows)
  // are solved densely here: per-row skip mask and dense inverses
  uint8_t *skip = nullptr;         // [n] row belongs to a terminal system
  bool any_term = false, all_term = false;
  double *inv = nullptr;           // dense inverses of the terminal blocks
  long long *inv_off = nullptr;    // [n_sys+1] offsets (0-sized for other systems)
  long long n_inv = 0;             // entries of inv
  int nc = 0;
  int *mptr = nullptr, *mem = nullptr;   // members of each aggregate, sorted
  double *x = nullptr, *b = nullptr, *t = nullptr;   // V-cycle work vectors
  // level 0 only: the residual after its single pre-sweep (the V-cycle's b
  // and x there are the caller's vectors)
  double *r = nullptr;
  float *r32 = nullptr;
  // sliced-ELL copy of level 0 (the system's own); coarse levels use CSR
  int *slice_ptr = nullptr, *scol = nullptr;
  double *sval = nullptr;
  float *sval32 = nullptr;
  int64_t sell_nnz = 0;
  // FP32 copy (mixed-precision path)
  float *val32 = nullptr, *sinv32 = nullptr, *inv32 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *t32 = nullptr;
  // classical hierarchy: interpolation P [n x nc] and restriction R = P^T
  // [nc x n] in CSR (FP64, FP32 copies for the mixed path)
  int *prow = nullptr, *pcol = nullptr, *rrow = nullptr, *rcol = nullptr;
  double *pval = nullptr, *rval = nullptr;
  float *pval32 = nullptr, *rval32 = nullptr;
  int64_t p_nnz = 0, r_nnz = 0;
};
struct Amg {
  std::vector<AmgLevel> levels;
  std::vector<void *> allocs;
  size_t bytes = 0;
  bool built = false;
  bool f32 = false;                // V-cycle in FP32
  bool classical = false;          // classical (Ruge-Stueben-type) levels instead of aggregation
  int tail_start = -1;             // first level run by the one-kernel tail
  size_t tail_smem[2] = {0, 0};    // its dynamic shared memory (FP64, FP32)
  float *sval32 = nullptr;         // FP32 sliced-ELL values of A (finest level)
  // VAG_MIXED_F16: the finest level in scaled variables (x~ = D^1/2 x),
  // h = D^-1/2 A D^-1/2 in FP16 (sliced ELL), its l1 scaling, and D^1/2
  bool f16 = false;
  __half *sval16 = nullptr;
  float *sinv16 = nullptr, *s0f = nullptr;
  double *s0d = nullptr;
};

// State of the mixed-precision solve (FP32 inner CG inside FP64 refinement).
struct Mixed {
  float *sval32 = nullptr;     // FP32 sliced-ELL values of S A S, S = D^{-1/2} (Jacobi)
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  float *z32 = nullptr;        // preconditioned inner residual (AMG)
  float *dval32 = nullptr;     // FP32 difference-form values of A, sliced ELL (AMG)
  float *rowsum32 = nullptr;   // [n_rows] its row sums
  bool dstale = true;
  cudaGraphExec_t graph_amg = nullptr;   // inner iterations with the V-cycle, rebuilt per solve
  size_t graph_amg_nodes = 0;
  double *sc = nullptr;        // S
  KrylovScalars *ks_in = nullptr;
  int *n_done_in = nullptr;
  bool stale = true;           // values older than the last numeric phase
  cudaGraphExec_t graph = nullptr;
};

// A batch of independent systems is assembled as the disjoint union of their
// meshes; each system's Krylov rows are contiguous.  Reductions run per row
// tile (one thread block each); the last tile of a system to finish sums the
// system's tile partials in tile order, so a system's arithmetic does not
// depend on the other systems of the batch.
struct Segments {
  int n_sys = 1;
  std::vector<int> node_start, ff_start, cell_start, dir_start, row_start;   // host, n_sys+1
  int *d_node_start = nullptr, *d_ff_start = nullptr, *d_cell_start = nullptr, *d_row_start = nullptr;
  int n_tiles = 0;
  std::vector<int> tile_start_h;     // first tile of each system, n_sys+1
  int *tile_sys = nullptr;           // [n_tiles]
  int *tile_row0 = nullptr;          // [n_tiles+1] (row range of tile t: [row0[t], row1[t]))
  int *tile_row1 = nullptr;
  int *sys_tile0 = nullptr;          // [n_sys+1] first tile of each system
  int *sys_grp0 = nullptr;           // [n_sys+1] first reduction group of each system
  int n_groups = 0;                  // reduction groups (kSegGroup tiles each, per system)
  int *cv_sys = nullptr;             // [n_cv] system of each control volume
};

struct System {
  Ctx *ctx = nullptr;
  bool counted = false;        // counted in ctx->live_systems
  std::vector<Alloc> allocs;
  size_t bytes = 0;

  // sizes
  int nv = 0, nc = 0, nf = 0, nd = 0;
  int n_rows = 0, n_row_nodes = 0, n_fc = 0;
  int64_t nnz = 0;
  int n_cv = 0;
  int64_t nnz_t = 0;
  double mu = 1.0;

  // mesh + data (device)
  double *xyz = nullptr;
  int *cell_nodes = nullptr;   // [8 nc] node slots (vag_topo.h), -1 where unused
  int *ff_nodes = nullptr;     // [4 nf] slot 3 = -1 for a triangle
  int8_t *cell_shape = nullptr;   // [nc] shape of each cell, nullptr when all are hexahedra
  int *shape_cells = nullptr;  // [nc] the cells grouped by shape, increasing within a shape
  int shape_start[5] = {0, 0, 0, 0, 0};   // (host) first entry of each shape in shape_cells
  bool tri_ff = false;         // some fracture face is a triangle
  // Peaceman wells (Sec. 5.5): perforated fracture faces
  int n_perf = 0;
  int *well_ff = nullptr;      // [n_perf] fracture-face index (distinct)
  double *well_wi = nullptr, *well_pw = nullptr, *well_q = nullptr, *well_cin = nullptr;   // [n_perf]
  double *Fw = nullptr;        // [n_perf] rate leaving the face into the well
  int *ff_perf = nullptr;      // [nf] perforation of each fracture face, or -1
  int perf_cap = 0;
  int *dir_nodes = nullptr;
  double *dir_vals = nullptr;
  double *lam = nullptr, *lamf = nullptr, *df = nullptr;

  // symbolic (device)
  int *node_dir = nullptr;     // [nv] index into the Dirichlet list, or -1
  int *node_isfrac = nullptr;  // [nv] 1 if the node lies on a fracture face
  int *cell_ff = nullptr;      // [6 nc] fracture-face id of each local face or -1
  int *ff_cells = nullptr;     // [2 nf] cells of each fracture face (-1: none)
  int *ff_lface = nullptr;     // [2 nf] local face index in that cell
  int *fc_index = nullptr;     // [nc] compact index of fracture cells or -1
  int *n2c_ptr = nullptr;      // [nv+1]
  int *n2c = nullptr;          // [8 nc]  cell*8 + local node
  int *n2f_ptr = nullptr;      // [nv+1]
  int *n2f = nullptr;          // [4 nf]  ff*4 + local node
  int *row_of_dof = nullptr;   // [nv + nf]
  int *dof_of_row = nullptr;   // [n_rows]
  int *rowptr = nullptr;       // [n_rows+1]
  int *col = nullptr;          // [nnz]
  int *diag_pos = nullptr;     // [n_rows]
  int *status = nullptr;       // device status word

  // numeric (device)
  double *Mc = nullptr;        // [45][nc]  packed upper triangle over (K, n0..n7), SoA
  double *Mfc = nullptr;       // [36][n_fc] per local face: (ss, sK, s n_t (4)) , SoA
  double *Mff = nullptr;       // [25][nf]  fracture matrices over (sigma, 4 nodes), SoA
  double *cvol = nullptr;      // [nc]
  double *ffarea = nullptr;    // [nf]
  double *val = nullptr;       // [nnz]
  // sliced-ELL copy (32-row slices, column-major inside a slice)
  int n_slices = 0;
  int64_t sell_nnz = 0;
  int sell_u = 0;              // loads in flight of the SELL row loop (0: not tuned yet)
  int *slice_ptr = nullptr;    // [n_slices+1] element offsets
  int *scol = nullptr;         // [sell_nnz]
  double *sval = nullptr;      // [sell_nnz]
  double *rhs = nullptr;       // [n_rows]
  double *dinv = nullptr;      // [n_rows]

  // solve (device)
  double *u = nullptr;         // [n_cv] full solution (nodes | ffaces | cells)
  double *kx = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr;   // [n_rows]
  double *partials = nullptr;  // [2 * n_tiles] (Krylov) / [kMaxRedBlocks] (transport)
  unsigned int *counter = nullptr;     // [n_sys + 1] arrival counters
  KrylovScalars *ks = nullptr;         // [n_sys]
  KrylovScalars *ks_host = nullptr;    // pinned mirror [n_sys]
  int *n_done = nullptr;               // systems converged (device)
  int *n_done_host = nullptr;          // pinned mirror
  int *amg_pin = nullptr;              // pinned, 4 ints: AMG setup read-backs
  Segments seg;
  cudaGraphExec_t pcg_graph = nullptr;
  int pcg_graph_chunk = 0;
  bool solved = false;
  bool last_mixed = false;
  Mixed mx;
  Amg amg;
  double *kz = nullptr;                // preconditioned residual (AMG)
  // BiCGStab: shadow residual r0^, s, s^ = M s, t = A s^, p^ = M p
  double *b_r0 = nullptr, *b_s = nullptr, *b_sh = nullptr, *b_t = nullptr, *b_ph = nullptr;
  cudaGraphExec_t bicg_graph = nullptr;
  cudaGraphExec_t pcg_graph_amg = nullptr;
  size_t amg_graph_nodes = 0;
  // Chebyshev preconditioner: coefficient table [2 kChebDegree per system],
  // work vectors, and the intervals [a, b] (host, per system)
  double *cheb_coef = nullptr;
  double *cw = nullptr, *cd = nullptr, *cy = nullptr;
  std::vector<double> cheb_bounds;
  cudaGraphExec_t pcg_graph_cheb = nullptr;
  size_t cheb_graph_nodes = 0;
  // GMRES: Arnoldi basis [m+1][n_rows], work vector, dot-product partials,
  // per-system state
  double *gm_V = nullptr, *gm_w = nullptr, *gm_part = nullptr;
  unsigned char *gm_state = nullptr;

  // transport (device)
  double *Fcn = nullptr;       // [8 nc]
  double *Fcf = nullptr;       // [6 nc]
  double *Fff = nullptr;       // [4 nf]
  bool have_flux = false;
  double *phi = nullptr;       // [n_cv]
  // upwind map in sliced ELL: slot i (rows sorted by inflow count inside
  // windows) holds control volume tperm[i]; slice s = 32 slots, entry u of
  // its lane r at tsp[s] + 32 u + r
  double *tdiag = nullptr;     // [n_cv + n_perf] by slot
  int *tperm = nullptr;        // [n_cv + n_perf]
  int *tsp = nullptr;          // [slices + 1]
  int *tcol = nullptr;         // [t_cap] (padding entries: own row, weight 0)
  double *tval = nullptr;      // [t_cap]
  int64_t t_cap = 0;
  double *cbuf = nullptr;      // [2 (n_cv + n_perf)]
  double *dts = nullptr;       // [2 n_sys]: per system dt_max, dt
  cudaGraphExec_t step_graph = nullptr;   // kStepChunk transport steps
  int64_t step_graph_cap = -1;
  int step_graph_rows = 0;
  int t_rows = 0;              // rows allocated for tdiag, tperm, tsp and each half of cbuf
  std::vector<double> dts_host;

  // timing events
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// allocation helpers (budget-checked)
void *sys_alloc_bytes(System *s, size_t bytes);
// device allocation from the context's pool (stream-ordered on its stream)
void *ctx_alloc(Ctx *c, size_t bytes);
void ctx_free(Ctx *c, void *p);
template <class T>
T *sys_alloc(System *s, size_t n) {
  return static_cast<T *>(sys_alloc_bytes(s, (n ? n : 1) * sizeof(T)));
}
void sys_free_all(System *s);

// Product of one row of a sliced-ELL matrix (32-row slices, column-major,
// see vag_sell.cu): one FMA per stored entry of the row, in CSR order, with
// U entries in flight (U is chosen per matrix size by the autotuner in
// vag_krylov.cu; the FMA sequence, hence the result, is the same for every
// U).  (A loop over the uniform slice width with eight in flight, padding
// included, measured 10-20 % slower on GB300.)
__device__ __forceinline__ float sell_val(__half v) { return __half2float(v); }
__device__ __forceinline__ float sell_val(float v) { return v; }
__device__ __forceinline__ double sell_val(double v) { return v; }
template <class T, int U = 4, class V = T>
__device__ __forceinline__ T sell_row(int row, const int *__restrict__ rowptr, const int *__restrict__ slice_ptr,
                                      const int *__restrict__ scol, const V *__restrict__ sval,
                                      const T *__restrict__ x) {
  const int len = rowptr[row + 1] - rowptr[row];
  const int base = slice_ptr[row >> 5] + (row & 31);
  T s = 0;
#pragma unroll(U)
  for (int k = 0; k < len; ++k) {
    const int idx = base + 32 * k;
    s = fma((T)sell_val(sval[idx]), x[scol[idx]], s);
  }
  return s;
}

// ----------------------------------------------------------- utilities ----
// Programmatic dependent launch (sm_90 and later): a kernel launched with
// launch_pdl may be scheduled while its predecessor in the stream finishes.
// It may read data that no kernel of the current sequence writes (matrix
// entries, index arrays) at once, and must call pdl_wait() before touching
// anything a predecessor produces; pdl_wait() returns when the predecessor
// has completed and its writes are visible.  pdl_trigger() (always after
// pdl_wait()) lets the next kernel be scheduled early.  Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                       Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess) fail(VAG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// Exclusive scan of n int32 values: out[0..n] (out[n] = total).  Returns the
// total (synchronises the stream).
int scan_exclusive(const int *in, int *out, int n, cudaStream_t st, bool want_total = true);
int read_status(System *s);
int grid_for(int64_t n, int block);
int num_sms();
// process-wide count of kernels this library has launched (graph launches
// count their kernel nodes)
void note_launches(unsigned long long n);
// while a stream capture is being recorded, launches are not counted (the
// graph launch counts its nodes instead)
void set_capturing(bool on);
unsigned long long launches_so_far();
// phase trace, active only with the environment variable VAG_TRACE set
// (labels must be string literals)
bool trace_enabled();
void trace_mark(cudaStream_t st, const char *label);
void trace_report(const char *call);

// General polyhedral descriptor (vag_mesh with cell_nodes == NULL) -> the
// padded per-shape numbering (vag_topo.h): device outputs cell_nodes
// [8 n_cells], ff_nodes [4 n_ff] and cell_shape [n_cells] (ids local to the
// mesh); *tri_ff is set when some fracture face is a triangle.  Returns the
// set of shapes seen (bit 1 << shape).  VAG_EMESH for a cell of none of the
// shapes, VAG_EINVAL for an offset or id out of range.
unsigned general_to_cells(Ctx *c, const vag_mesh &m, int mem, int32_t *cell_nodes, int32_t *ff_nodes,
                          int8_t *cell_shape, bool *tri_ff);

// ------------------------------------------------------------- phases -----
void symbolic_phase(System *s);
void numeric_phase(System *s);
double time_cell_local(System *s, int reps);   // mean ms of the local-matrix launches of one numeric phase
void pcg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
void bicgstab_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
void gmres_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
// y = A x (FP64 sliced ELL, tuned loads in flight), stream-ordered, capture-safe
void launch_spmv_plain(System *s, const double *x, double *y, cudaStream_t st);
// ks[sys].res2 = ||b - A x||^2 per system (x = s->kx)
void true_residual2(System *s, cudaStream_t st);
void amg_setup(System *s, bool f32, bool f16 = false, bool classical = false);
// classical coarsening of level L into C (vag_amg_rs.cu): fills L's P and R
// and C's matrix, diagonal inverse and system row starts; alloc gives the
// hierarchy's own memory
void rs_coarsen(System *s, AmgLevel &L, AmgLevel &C, const std::function<void *(size_t)> &alloc);
void amg_apply(System *s, const double *r, double *z, cudaStream_t st);
// z = V(r) on FP32 vectors with the FP32 hierarchy (the inner solve of the
// refinement loop); r and z must not be the hierarchy's own level-0 vectors
void amg_apply_f32(System *s, const float *r, float *z, cudaStream_t st);
// The FP64 V-cycle inside CG: amg_first_sweep_scale gives the finest level's
// l1 scaling, its first-sweep buffer t0 and omega (null for the FP32
// hierarchy or a hierarchy without coarse levels) so that the CG update can
// make the first sweep t0 = omega D_l1^-1 r; amg_apply_cg then runs the rest of
// the cycle and forms r.z (beta, rho) in its last sweep.
const double *amg_first_sweep_scale(System *s, double *&t0, double &omega);
bool amg_apply_cg(System *s, const double *r, double *z, cudaStream_t st);
// The same for the FP32 V-cycle of the CG inside refinement (inner scalars
// ks, n_done); unavailable (nullptr / false) with the FP16 finest level.
const float *amg_first_sweep_scale_f32(System *s, float *&t0, float &omega);
bool amg_apply_f32_cg(System *s, const float *r, float *z, cudaStream_t st, KrylovScalars *ks, int *n_done);
void amg_free(System *s);
// Chebyshev preconditioner (FP64): cheb_setup estimates each system's interval
// from Jacobi-CG Lanczos coefficients and fills the coefficient table;
// cheb_apply forms z = M r (in_iter: systems already done are skipped;
// w_ready: s->cw already holds D^-1 r; rz: the last step also sets beta and
// r.z in s->ks, as the r.z reduction of CG does).
void cheb_setup(System *s);
void cheb_apply(System *s, const double *r, double *z, cudaStream_t st, bool in_iter, bool w_ready, bool rz);
// m Jacobi-CG iterations from x = 0 on A x = v (v on the device, per system
// rows): alpha[sys*m + j], beta[sys*m + j] for j < steps[sys], the iterations
// that ran without breakdown.  Overwrites the Krylov work vectors.
void jacobi_cg_coefficients(System *s, const double *v, int m, std::vector<double> &alpha,
                            std::vector<double> &beta, std::vector<int> &steps);
// choose (once per context and matrix size class) the loads in flight of the
// sliced-ELL row loop by timing the candidates on this system's matrix;
// never call it while a stream capture is open
void tune_sell(System *s);
// measurement hooks: mean ms of one launch over `reps`
double time_spmv(System *s, int reps);
double time_smoother(System *s, int reps);
double time_transport_step(System *s, int reps);
double time_spmv32(System *s, int reps);
void mixed_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
// FP64 iterative refinement around FP32 CG preconditioned by the FP32 AMG
// V-cycle (VAG_MIXED / VAG_MIXED_F16 with VAG_PC_AMG and CG)
void mixed_amg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
void ensure_krylov_buffers(System *s);
// Krylov result in s->kx and per-system scalars in s->ks: scatter into u,
// recover the cells, compute the fluxes, fill the aggregate info.
void finish_solve(System *s, vag_solve_info *info, bool mixed);
void spmv_f64(System *s, const double *x, double *y);
void build_tiles(System *s);
void build_sell(System *s);
void sell_values(System *s);
void sell_values_scaled_f32(System *s, const double *scale, float *out);
void sell_values_f32(System *s, float *out);
void sell_values_scaled_f16(System *s, const double *scale, __half *out);
int64_t sell_structure(cudaStream_t st, int n, const int *rowptr, const int *col, int **slice_ptr_out,
                       int **scol_out, const std::function<void *(size_t)> &alloc);
void solve_infos(const System *s, vag_solve_info *infos);
void recover_cells_and_fluxes(System *s);
void transport_run(System *s, const vag_transport_opts *o, double *c_dev, vag_transport_info *info,
                   const double *phi_m, const double *phi_f, const double *cbar);

}  // namespace vag

struct vag_ctx {
  vag::Ctx c;
};
struct vag_system {
  vag::System s;
};
