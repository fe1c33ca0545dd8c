// Internal declarations of the VAG CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "vag.h"

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
};

constexpr int kMaxRowWidth = 160;   // unique columns of one eliminated row
constexpr int kMaxRedBlocks = 4096; // blocks of a reduction kernel

// ------------------------------------------------------------ context ------
struct Ctx {
  int device = 0;
  size_t budget = 0;
  size_t in_use = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string last_error;
};

// One device allocation owned by a system.
struct Alloc {
  void *ptr;
  size_t bytes;
};

// Krylov scalars kept on the device.
struct KrylovScalars {
  double rz, pq, alpha, beta, rr, bb, tol2, res2;
  int iter, maxit, done, breakdown;
};

struct System {
  Ctx *ctx = nullptr;
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
  int *cell_nodes = nullptr;
  int *ff_nodes = nullptr;
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
  double *rhs = nullptr;       // [n_rows]
  double *dinv = nullptr;      // [n_rows]

  // solve (device)
  double *u = nullptr;         // [n_cv] full solution (nodes | ffaces | cells)
  double *kx = nullptr, *kr = nullptr, *kp = nullptr, *kq = nullptr;   // [n_rows]
  double *partials = nullptr;  // [2 * kMaxRedBlocks]
  unsigned int *counter = nullptr;
  KrylovScalars *ks = nullptr;
  KrylovScalars *ks_host = nullptr;   // pinned mirror for polling
  cudaGraphExec_t pcg_graph = nullptr;
  int pcg_graph_chunk = 0;
  bool solved = false;

  // transport (device)
  double *Fcn = nullptr;       // [8 nc]
  double *Fcf = nullptr;       // [6 nc]
  double *Fff = nullptr;       // [4 nf]
  bool have_flux = false;
  double *phi = nullptr;       // [n_cv]
  double *tdiag = nullptr;     // [n_cv]
  int *trowptr = nullptr;      // [n_cv+1]
  int *tcol = nullptr;         // [nnz_t]
  double *tval = nullptr;      // [nnz_t]
  int64_t t_cap = 0;
  double *cbuf = nullptr;      // [2 n_cv]
  double *dts = nullptr;       // [4] dt_max, dt, ...

  // timing events
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// allocation helpers (budget-checked)
void *sys_alloc_bytes(System *s, size_t bytes);
template <class T>
T *sys_alloc(System *s, size_t n) {
  return static_cast<T *>(sys_alloc_bytes(s, (n ? n : 1) * sizeof(T)));
}
void sys_free_all(System *s);

// ----------------------------------------------------------- utilities ----
// Exclusive scan of n int32 values: out[0..n] (out[n] = total).  Returns the
// total (synchronises the stream).
int scan_exclusive(const int *in, int *out, int n, cudaStream_t st, bool want_total = true);
int read_status(System *s);
int grid_for(int64_t n, int block);
int num_sms();

// ------------------------------------------------------------- phases -----
void symbolic_phase(System *s);
void numeric_phase(System *s);
void pcg_solve(System *s, const vag_solve_opts *o, vag_solve_info *info);
void spmv_f64(System *s, const double *x, double *y);
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
