/*
 * vag.h -- C ABI of the GB300 implementation of the hybrid-dimensional Vertex
 * Approximate Gradient (VAG) Darcy solve and explicit upwind transport
 * (Xing, Masson, Lopez: "Parallel Vertex Approximate Gradient discretization
 * of hybrid dimensional Darcy flow and transport in discrete fracture
 * networks").
 *
 * One process drives one GPU.  Every array argument is a plain pointer plus
 * the sizes given in the structs; a `mem` argument says whether the pointers
 * are host (VAG_MEM_HOST) or device (VAG_MEM_DEVICE) addresses.  The caller
 * owns every array it passes; the library copies inputs in and writes outputs
 * out and keeps no caller pointer after a call returns.  Opaque handles are
 * owned by the library and released by the matching *_destroy call.
 *
 * Errors: every entry point returns a vag_status; VAG_OK is 0.  On an error
 * the outputs are left untouched (except VAG_ENOTCONVERGED, which writes the
 * last iterate and a filled info struct) and vag_last_error() describes the
 * cause.  No C++ exception crosses this boundary.  Device kernels never trap:
 * failed checks and exhausted waits set a status word that the host reads.
 *
 * Index base 0, indices int32.  Every global vector of unknowns or
 * concentrations is ordered [nodes | fracture faces | cells].
 *
 * Threading: a vag_ctx and the systems created from it are used by one host
 * thread at a time.  The server (vag_server_*) is internally synchronised.
 */
#ifndef VAG_H
#define VAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int vag_status;
enum {
  VAG_OK = 0,
  VAG_EINVAL = 1,          /* bad argument (null pointer, size, value)      */
  VAG_ENOMEM = 2,          /* device allocation failed                      */
  VAG_EBUDGET = 3,         /* the context's memory budget would be exceeded */
  VAG_ENOTCONVERGED = 4,   /* Krylov solve hit maxit above rtol             */
  VAG_EBREAKDOWN = 5,      /* p^T A p <= 0 (matrix not SPD) or NaN          */
  VAG_ETIMEOUT = 6,        /* a bounded wait expired                        */
  VAG_ECUDA = 7,           /* a CUDA runtime call failed                    */
  VAG_EMESH = 8            /* the mesh is not conforming / not supported    */
};

enum { VAG_MEM_HOST = 0, VAG_MEM_DEVICE = 1 };
/* Precision of vag_solve.
 * VAG_FP64: every operation in FP64.
 * VAG_MIXED: FP64 iterative refinement (residual b - A x, update and
 *   convergence test in FP64) around an FP32 inner Krylov solve: with
 *   VAG_PC_JACOBI, FP32 CG on D^-1/2 A D^-1/2; with VAG_PC_AMG, FP32 CG on A
 *   preconditioned by the FP32 copy of the AMG hierarchy (BiCGStab and GMRES
 *   with VAG_PC_AMG instead run FP64 iterations with the FP32 V-cycle).
 * VAG_MIXED_F16: VAG_MIXED with the AMG V-cycle's finest-level matrix stored
 *   in FP16 after symmetric diagonal scaling (D^-1/2 A D^-1/2, entries in
 *   [-1, 1]); VAG_PC_AMG only.
 * VAG_FP64_PC32: FP64 Krylov iterations preconditioned by the FP32 AMG
 *   V-cycle, no refinement; VAG_PC_AMG only. */
enum { VAG_FP64 = 0, VAG_MIXED = 1, VAG_MIXED_F16 = 2, VAG_FP64_PC32 = 3 };
/* Preconditioners: Jacobi D^-1; VAG_PC_CHEBYSHEV, four steps of Chebyshev
 * acceleration of Jacobi (a degree-3 polynomial in D^-1 A times D^-1) on
 * [b/100, b], b = 1.2 x the largest Ritz value of D^-1 A after ten Lanczos
 * (Jacobi-CG) steps from a pseudo-random vector, FP64 only; VAG_PC_AMG, the
 * library's aggregation AMG V-cycle (FP64, or FP32 under VAG_MIXED);
 * VAG_PC_AMG_RS, a classical (Ruge-Stueben-type) AMG V-cycle, the counterpart
 * of the classical AMG of the paper's solver experiments (Sec. 5.3): strength
 * on negative couplings (theta = 0.25), PMIS coarse/fine splitting with a
 * second pass, direct interpolation from at most four coarse neighbours,
 * Galerkin R A P with R = P^T, the same l1-Jacobi sweeps; FP64, FP32 under
 * VAG_MIXED or VAG_FP64_PC32 (not VAG_MIXED_F16).  Wherever VAG_PC_AMG is
 * accepted, VAG_PC_AMG_RS is too, except under VAG_MIXED_F16 (VAG_EINVAL). */
enum { VAG_PC_JACOBI = 0, VAG_PC_CHEBYSHEV = 1, VAG_PC_AMG = 2, VAG_PC_AMG_RS = 3 };
/* Krylov method: CG (the system is SPD), or one of the methods of the
 * paper's solver experiments (§5.3), both right-preconditioned: BiCGStab, or
 * restarted GMRES(30) (classical Gram-Schmidt applied twice, Givens
 * rotations; a system stops when its true residual meets rtol, at maxit
 * Arnoldi steps, or when a whole restart cycle no longer lowers it). */
enum { VAG_KRYLOV_CG = 0, VAG_KRYLOV_BICGSTAB = 1, VAG_KRYLOV_GMRES = 2 };

typedef struct vag_ctx vag_ctx;
typedef struct vag_system vag_system;

/*
 * Mesh (Sec. 3.1: a generalized polyhedral mesh conforming to the fracture
 * network), in one of two forms.
 *
 * Hexahedral fast path (cell_nodes != NULL):
 *   xyz        [3*n_nodes]  node coordinates, x y z interleaved.
 *   cell_nodes [8*n_cells]  node l of a cell sits at lattice offset
 *              (l&1, (l>>1)&1, (l>>2)&1): faces are {0,2,6,4} (-x),
 *              {1,3,7,5} (+x), {0,1,5,4} (-y), {2,3,7,6} (+y), {0,1,3,2} (-z),
 *              {4,5,7,6} (+z); faces need not be planar.
 *   ff_nodes   [4*n_ff]     the fracture faces F_Gamma, each a face of the
 *              mesh given by its four nodes in cyclic order.  A fracture face
 *              that is not a face of some cell is a VAG_EMESH error.
 *
 * General polyhedral descriptor (cell_nodes == NULL; ff_nodes ignored):
 *   n_faces, face_node_ptr [n_faces+1], face_node_idx: the nodes of face f,
 *              face_node_idx[face_node_ptr[f] .. face_node_ptr[f+1]), in
 *              cyclic order (consecutive nodes share an edge);
 *   cell_face_ptr [n_cells+1], cell_face_idx: the faces of cell K,
 *              cell_face_idx[cell_face_ptr[K] .. cell_face_ptr[K+1]);
 *   ff_face_ids [n_ff]: the fracture faces F_Gamma as face ids.
 *   The library recognises four cell shapes from their faces, whatever the
 *   order of the faces and the starting node of each face: hexahedra (six
 *   quadrilaterals forming a cube graph), tetrahedra (four triangles),
 *   triangular prisms (two triangles, three quadrilaterals) and pyramids
 *   (one quadrilateral, four triangles), in any mix.  Each cell is numbered
 *   canonically from its node ids (a hexahedron: node 0 = the smallest id,
 *   1, 2, 4 = its edge neighbours in increasing id), so on a lattice whose
 *   node ids grow with x, then y, then z a hexahedral mesh gets the lattice
 *   numbering and both forms give bitwise the same system; a mesh of
 *   hexahedra alone runs on the hexahedral kernels.  Fracture faces are
 *   triangles or quadrilaterals.  Any other cell or face is a VAG_EMESH
 *   error; an offset or id out of range is VAG_EINVAL.
 *
 * Cell centres x_K and face centres x_sigma are the isobarycentres of their
 * nodes (beta_{sigma,s} = 1/|V_sigma|).
 */
typedef struct {
  int32_t n_nodes;
  const double *xyz;
  int32_t n_cells;
  const int32_t *cell_nodes;
  int32_t n_ff;
  const int32_t *ff_nodes;
  int32_t n_faces;
  const int32_t *face_node_ptr;
  const int32_t *face_node_idx;
  const int32_t *cell_face_ptr;
  const int32_t *cell_face_idx;
  const int32_t *ff_face_ids;
} vag_mesh;

/*
 * Physical data of Eq. (modeleCont) and Eq. (varformVAG):
 *   lambda_m [6*n_cells] cellwise-constant SPD tensor Lambda_m as
 *            (xx, yy, zz, xy, xz, yz);
 *   lambda_f [n_ff]      isotropic tangential fracture permeability;
 *   d_f      [n_ff]      fracture aperture (width);
 *   mu                   viscosity (> 0).
 * Wells (Sec. 5.5, optional; n_perf = 0 for none): perforation p connects
 * fracture face well_ff[p] to a well through the Peaceman model, the
 * volume rate leaving the face into the well being
 *   q_p = well_wi[p] (u_sigma - well_pw[p]) - well_q[p],
 * so a producer has WI > 0 and its well pressure p_w, and an injector with
 * an imposed rate has WI = 0 and q > 0 (both terms may be combined).  The
 * pressure equation of the face gains q_p; in the transport a positive q_p
 * leaves the face with its concentration and a negative one enters it with
 * concentration well_cin[p].  Perforated faces are distinct fracture faces
 * of this mesh (0-based); every array has n_perf entries; WI >= 0.
 * vag_peaceman_wi gives the well index of a perforated fracture face.
 */
typedef struct {
  const double *lambda_m;
  const double *lambda_f;
  const double *d_f;
  double mu;
  int32_t n_perf;
  const int32_t *well_ff;
  const double *well_wi;
  const double *well_pw;
  const double *well_q;
  const double *well_cin;
} vag_props;

/*
 * Peaceman well index of a vertical well through a fracture face (Sec. 5.5):
 * the face expanded as a box dx x d_f x dz, the well's analytic radial
 * pressure imposed at the box corners and its rate at the box centre give
 *   WI = 2 pi dz Lambda_f / (mu log(r_0 / r_w)),  r_0 = D exp(-2 pi dz / C),
 *   C = 4/3 (dx dz / d_f + dx d_f / dz + dz d_f / dx),
 *   D = sqrt(dx^2 + d_f^2) / 2,
 * C being the cell diagonal of the VAG scheme on that box with unit
 * permeability.  Host arrays of n entries; every input > 0 and r_0 > r_w,
 * else VAG_EINVAL (wi_out untouched).  mu = 1 reproduces the paper's
 * expression, which has no viscosity.
 */
vag_status vag_peaceman_wi(int32_t n, const double *dx, const double *dz, const double *d_f,
                           const double *lambda_f, const double *r_w, double mu, double *wi_out);

/*
 * Dirichlet nodes V_D with pressure u_s = values[i] (Sec. 3.1; the paper's
 * V_ext).  Every other boundary node is a no-flow node.  Nodes must be
 * distinct.  At least one node must be given unless a well perforation with
 * WI > 0 fixes the pressure level (VAG_EINVAL otherwise).
 */
typedef struct {
  int32_t n_dir;
  const int32_t *nodes;
  const double *values;
} vag_dirichlet;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the device
 * memory all systems of this context may hold (0 = no cap).  The context owns
 * a non-blocking stream unless vag_ctx_set_stream() supplies one. */
vag_status vag_ctx_create(int device, size_t mem_budget_bytes, vag_ctx **out);
/* Release the context.  Systems created from it stay valid; the context's
 * resources are freed with the last of them.  No new system may be created
 * from a destroyed context. */
void vag_ctx_destroy(vag_ctx *ctx);
/* Use the caller's cudaStream_t (passed as void*); NULL restores the
 * context's own stream.  Every later call of this context runs on it. */
vag_status vag_ctx_set_stream(vag_ctx *ctx, void *cuda_stream);
/* Human-readable description of the last error on this context. */
const char *vag_last_error(const vag_ctx *ctx);
/* Device bytes currently held by the context's systems. */
size_t vag_ctx_bytes_in_use(const vag_ctx *ctx);
/* Number of CUDA kernels this library has launched in this process (kernels
 * inside a replayed CUDA graph count once per replay).  For instrumentation. */
unsigned long long vag_launch_count(void);

/* --------------------------------------------------------------- assembly */

/*
 * Build the VAG system of Sec. 3.1 and Sec. 4.2 on the device:
 *  - symbolic phase (once per mesh): fracture faces matched to cell faces,
 *    node->cell and node->fracture-face adjacency, the Krylov unknowns
 *    (V \ V_D) u F_Gamma and the CSR pattern of the cell-eliminated system;
 *  - numeric phase: the local matrices a_{K,nu}^{nu'} of Eq. (VAGFluxMatrix)
 *    on the 24 tetrahedra T_{K,sigma,e} of every cell, the fracture matrices
 *    a_{sigma,s}^{s'} of Eq. (VAGFluxFracture), and the Schur complement of
 *    Eq. (eqschur) (cell unknowns eliminated, A_cc diagonal) gathered row by
 *    row into CSR with the Dirichlet columns moved to the right-hand side.
 * Krylov rows are the non-Dirichlet nodes in increasing node id followed by
 * the fracture faces in input order.  All arithmetic is FP64.
 * mem: location of every pointer in mesh, props and bc.
 * Size limits (int32 indices): n_nodes + n_ff + n_cells < 2^31, 8 n_cells
 * and 4 n_ff < 2^31, and the eliminated system's stored entries, including
 * the sliced-ELL padding of 32-row slices, < 2^31; larger inputs are
 * VAG_EINVAL (the same limits hold for a batch's union).
 */
vag_status vag_assemble(vag_ctx *ctx, const vag_mesh *mesh, const vag_props *props,
                        const vag_dirichlet *bc, int mem, vag_system **out);
/*
 * Batch of independent realisations in one system handle: the n_sys meshes
 * are assembled as their disjoint union (node, cell and fracture-face ids of
 * system i are offset by the sizes of systems 0..i-1), so one symbolic phase,
 * one numeric phase, one Krylov loop and one transport loop serve the whole
 * batch.  Each system keeps its own CG scalars and convergence test and its
 * own CFL step, and its arithmetic is independent of the other systems: a
 * system gives bitwise the same results alone or in any batch.  meshes,
 * props, bcs: arrays of n_sys structs (per-system ids, 0-based); every system
 * must have the same mu.  Vectors of the batch (u_out, c_inout, phi_m, ...)
 * are the union's: [all nodes | all fracture faces | all cells], each block
 * ordered by system; vag_system_get_batch gives the offsets.
 */
vag_status vag_assemble_batch(vag_ctx *ctx, int32_t n_sys, const vag_mesh *meshes, const vag_props *props,
                              const vag_dirichlet *bcs, int mem, vag_system **out);
/* Layout of a batch: n_sys, and (arrays of n_sys+1, any may be NULL) the first
 * node, fracture face, cell and Krylov row of each system.  A single system is
 * a batch of one. */
vag_status vag_system_get_batch(const vag_system *sys, int32_t *n_sys, int32_t *node_start, int32_t *ff_start,
                                int32_t *cell_start, int32_t *row_start);

/* Re-run the numeric phase with new properties (and wells) on the same mesh.
 * On a batch, props' arrays (and the wells' fracture-face ids) cover the
 * union. */
vag_status vag_update_props(vag_system *sys, const vag_props *props, int mem);
void vag_system_destroy(vag_system *sys);

typedef struct {
  int32_t n_nodes, n_cells, n_ff, n_dir;
  int32_t n_rows;          /* Krylov unknowns: non-Dirichlet nodes + fracture faces */
  int64_t nnz;             /* nonzeros of the eliminated system                   */
  int32_t n_frac_cells;    /* cells with at least one fracture face               */
  int32_t n_cv;            /* control volumes = n_nodes + n_ff + n_cells          */
  int64_t nnz_transport;   /* off-diagonal entries of the upwind transport map    */
  size_t device_bytes;     /* device memory held by this system                   */
} vag_system_info;
vag_status vag_system_get_info(const vag_system *sys, vag_system_info *info);

/* ------------------------------------------------------------------ solve */

typedef struct {
  int precision;     /* VAG_FP64, VAG_MIXED, VAG_MIXED_F16, VAG_FP64_PC32   */
  int precond;       /* VAG_PC_JACOBI, VAG_PC_CHEBYSHEV (VAG_FP64 only;
                        VAG_EINVAL otherwise), VAG_PC_AMG, VAG_PC_AMG_RS     */
  double rtol;       /* stop at ||b - A x||_2 <= rtol ||b||_2 (> 0)           */
  int32_t maxit;     /* Krylov iteration cap (total over refinements)          */
  int mem;           /* location of u_out                                     */
  int32_t krylov;    /* VAG_KRYLOV_CG (0, the default), VAG_KRYLOV_BICGSTAB
                        or VAG_KRYLOV_GMRES (FP64 iterations; with VAG_MIXED
                        only for an AMG preconditioner, whose V-cycle then
                        runs on the FP32 hierarchy); iterations counts
                        Arnoldi steps for GMRES                            */
  double inner_rtol; /* VAG_MIXED(_F16) with an AMG preconditioner and CG:
                        smallest relative tolerance of an inner FP32 solve
                        (each refinement step solves to max(inner_rtol,
                        0.3 x the reduction still needed), at most 0.1);
                        0 = 1e-6                                           */
} vag_solve_opts;

typedef struct {
  int32_t iterations;    /* Krylov iterations (inner iterations for MIXED)     */
  int32_t outer;         /* refinement steps (MIXED), else 1                   */
  double rel_residual;   /* final ||b - A x|| / ||b|| recomputed in FP64       */
  double ms_setup;       /* preconditioner setup, device time                   */
  double ms_solve;       /* Krylov loop + cell recovery, device time            */
  vag_status status;
} vag_solve_info;

/*
 * Solve the eliminated system by preconditioned conjugate gradients (the
 * matrix is symmetric positive definite: Galerkin form, Dirichlet rows
 * removed; opts->krylov selects BiCGStab or GMRES(30) instead), then recover
 * the cell unknowns by Eq. (eqschurcell) and keep the full solution on the
 * device for vag_transport.  u_out (optional, may be
 * NULL): [n_nodes + n_ff + n_cells] in the [nodes | ffaces | cells] order, the
 * Dirichlet values echoed at Dirichlet nodes.
 */
vag_status vag_solve(vag_system *sys, const vag_solve_opts *opts, double *u_out,
                     vag_solve_info *info);

/* Per-system results of the last vag_solve of a batch: infos [n_sys]
 * (ms_setup and ms_solve are 0; vag_solve reports the batch's times). */
vag_status vag_solve_get_infos(const vag_system *sys, vag_solve_info *infos);

/* y = A x on the Krylov rows of the eliminated system (FP64).  x, y: [n_rows].
 * With VAG_MEM_DEVICE the call is stream-ordered on the context stream and
 * returns without waiting; with VAG_MEM_HOST it returns after y is written. */
vag_status vag_spmv(vag_system *sys, const double *x, double *y, int mem);

/* -------------------------------------------------------------- transport */

typedef struct {
  const double *phi_m;   /* [n_cells] matrix porosity                          */
  const double *phi_f;   /* [n_ff] fracture porosity                           */
  const double *cbar;    /* [n_dir] Dirichlet concentration, aligned with bc   */
  double omega;          /* control-volume fraction alpha = omega/|V_K| (Sec.
                            3.2.1); 0 <= omega < 1, typically 0.5             */
  double cfl;            /* > 0: dt = cfl * the CFL bound of Eq. (eq_CFL)     */
  double dt;             /* used when cfl <= 0                                */
  int32_t n_steps;       /* explicit Euler steps to take (>= 0)               */
  int mem;               /* location of phi_m, phi_f, cbar and c_inout        */
} vag_transport_opts;

typedef struct {
  double dt_max;         /* the CFL bound min(dt_M, dt_F, dt_V) (a batch: the
                            smallest over its systems)                        */
  double dt;             /* the step used (a batch: the smallest)             */
  int32_t steps;
  double ms;             /* device time of the steps                          */
} vag_transport_info;

/*
 * Explicit first-order upwind transport (Sec. 3.2, Eq. darcyfluxH) driven by
 * the fluxes of the last vag_solve (or of vag_set_fluxes).  Porous volumes
 * follow Sec. 3.2.1 with alpha_{K,s} = omega/|V_K| on nodes of K outside
 * V_D u V_Gamma (omega/8 on a hexahedron) and alpha_{sigma,s} =
 * omega/|V_sigma| on nodes of sigma outside V_D.  Well perforations (Sec.
 * 5.5) add their rates: a producer's outflow leaves its fracture face with
 * the face's concentration, an injector's inflow enters at its well_cin.
 * c_inout: [n_nodes + n_ff + n_cells]; on entry c^0, on exit c^{n_steps}.  The
 * Dirichlet entries are set to cbar before the first step (c^0_s = cbar_s).
 */
vag_status vag_transport(vag_system *sys, const vag_transport_opts *opts, double *c_inout,
                         vag_transport_info *info);

/* The same operation under the name of the problem statement's transport
 * step (Eq. tracero1own applied n_steps times): *dt_used (may be NULL)
 * receives the step used (a batch: its smallest); info may be NULL. */
vag_status vag_transport_step(vag_system *sys, const vag_transport_opts *opts, double *c_inout, double *dt_used,
                              vag_transport_info *info);

/* Per-system CFL bound and step of the last vag_transport: [n_sys] each (a
 * system with no outflow anywhere has bound +inf and step 0 under cfl > 0). */
vag_status vag_transport_get_dts(const vag_system *sys, double *dt_max, double *dt);

/* ----------------------------------------------------- inspection / tests */

/* Copy out the eliminated system: rowptr [n_rows+1], col [nnz] (row indices),
 * val [nnz], rhs [n_rows], row_dof [n_rows] (global DOF of each row: node id,
 * or n_nodes + fracture-face index).  Any pointer may be NULL. */
vag_status vag_export_system(const vag_system *sys, int32_t *rowptr, int32_t *col, double *val,
                             double *rhs, int32_t *row_dof, int mem);
/* Fluxes of Eq. (VAGFluxMatrix) / Eq. (VAGFluxFracture) in the library's
 * layout: F_cell_nodes [8*n_cells] (F_{K,s}, s in the cell's node-slot
 * order, see vag_export_cells; 0 in unused slots), F_cell_faces
 * [6*n_cells] (F_{K,sigma} on the cell's faces in the local face order of
 * its shape, the hexahedral fast path's being that of vag_mesh; 0 where
 * the face is not a fracture face or does not exist), F_frac [4*n_ff]
 * (F_{sigma,s}, s in the order of vag_export_cells' ff_nodes; 0 in a
 * triangle's fourth slot). */
/* The numbering the kernels run on: cell_nodes [8*n_cells] (the node slots
 * of each cell in its shape's local order, -1 in unused slots), shape
 * [n_cells] (VAG_SHAPE_*), ff_nodes [4*n_ff] (each fracture face's nodes in
 * cyclic order, -1 in a triangle's fourth slot).  For the hexahedral fast
 * path these are the caller's arrays; for the general descriptor the
 * canonical numbering described at vag_mesh.  Any pointer may be NULL. */
/* Local numbering of the shapes (faces in local face order, each cyclic):
 *   VAG_SHAPE_HEX     node l at offset (l&1, (l>>1)&1, (l>>2)&1); faces
 *                     {0,2,6,4} {1,3,7,5} {0,1,5,4} {2,3,7,6} {0,1,3,2} {4,5,7,6}
 *   VAG_SHAPE_TET     faces {1,2,3} {0,3,2} {0,1,3} {0,2,1} (face l opposite node l)
 *   VAG_SHAPE_PRISM   0 1 2 bottom, 3+i above i; faces {0,1,2} {3,4,5} {0,1,4,3}
 *                     {1,2,5,4} {2,0,3,5}
 *   VAG_SHAPE_PYRAMID 0 1 2 3 base, 4 apex; faces {0,1,2,3} {0,1,4} {1,2,4}
 *                     {2,3,4} {3,0,4} */
enum { VAG_SHAPE_HEX = 0, VAG_SHAPE_TET = 1, VAG_SHAPE_PRISM = 2, VAG_SHAPE_PYRAMID = 3 };
vag_status vag_export_cells(const vag_system *sys, int32_t *cell_nodes, int8_t *shape, int32_t *ff_nodes, int mem);
vag_status vag_export_fluxes(const vag_system *sys, double *F_cell_nodes, double *F_cell_faces,
                             double *F_frac, int mem);
/* Rates q_p of the well perforations (n_perf entries, in the order given in
 * vag_props) from the last vag_solve: positive = leaving the fracture face
 * into the well (production).  Zero before the first solve. */
vag_status vag_export_well_rates(const vag_system *sys, double *q_out, int mem);

/* Replace the fluxes (same layout) used by the next vag_transport. */
vag_status vag_set_fluxes(vag_system *sys, const double *F_cell_nodes, const double *F_cell_faces,
                          const double *F_frac, int mem);
/* Porous volumes phi_mu [n_cv] of the last vag_transport (0 at Dirichlet nodes). */
vag_status vag_export_porous_volumes(const vag_system *sys, double *phi, int mem);

/* ------------------------------------------------------------ measurement */

/* Hot kernels that vag_kernel_time can time. */
enum {
  VAG_KERNEL_SPMV = 0,            /* q = A p, FP64 sliced ELL (the CG product)      */
  VAG_KERNEL_SMOOTH = 1,          /* one l1-Jacobi sweep on the finest level of the
                                     last AMG hierarchy (FP64, or FP32 after a
                                     mixed-precision AMG solve)                    */
  VAG_KERNEL_TRANSPORT_STEP = 2,  /* one explicit upwind step c' = d c + W c          */
  VAG_KERNEL_SPMV32 = 3,          /* q = A p and p.q in FP32, sliced ELL (the inner
                                     CG product of a VAG_MIXED AMG solve)          */
  VAG_KERNEL_CELL_LOCAL = 4       /* the local VAG matrices of every cell (one
                                     launch per cell shape present; the time is
                                     that of all of them)                          */
};

/*
 * Measurement hook (the paper has no counterpart): time `reps` back-to-back
 * launches of one hot kernel on this system's own data with CUDA events on the
 * context's stream and return the mean duration of a launch in *ms_per_launch.
 * VAG_KERNEL_SMOOTH needs the AMG hierarchy of a previous vag_solve with
 * VAG_PC_AMG or VAG_PC_AMG_RS (VAG_MIXED_F16's FP16 finest level excepted);
 * VAG_KERNEL_SPMV32 needs a previous VAG_MIXED or VAG_MIXED_F16 solve with
 * an AMG preconditioner and CG; VAG_KERNEL_CELL_LOCAL rewrites the system's local
 * matrices with the same values; VAG_KERNEL_TRANSPORT_STEP needs the upwind map of a
 * previous vag_transport; VAG_EINVAL otherwise, or for reps < 1.  The kernels
 * run on the system's Krylov and transport work vectors, whose contents are
 * overwritten (the solution and the concentrations already returned are not
 * touched).  Synchronises the stream.
 */
vag_status vag_kernel_time(vag_system *sys, int kernel, int32_t reps, double *ms_per_launch);

/* ---------------------------------------------------------------- server */

/*
 * Request server with continuous batching (the paper has no counterpart: its
 * runs are single MPI jobs).  `slots` worker threads each own a context
 * (stream and memory pool) on `device`.  A free slot takes the oldest queued
 * request together with every queued request of identical solver settings
 * (precision, preconditioner, rtol, maxit, n_steps, omega, cfl, mu) whose
 * estimated device memory still fits mem_budget_bytes, runs them as one batch
 * (vag_assemble_batch, vag_solve, vag_transport) and completes them.
 * Requests that arrive while batches run are admitted as slots and budget
 * free up; batches of different slots overlap on the GPU.  A request's
 * results are bitwise the same as when it is solved alone.
 */
typedef struct vag_server vag_server;

typedef struct {
  int device;
  size_t mem_budget_bytes;   /* admission budget for batches in flight (0 = none) */
  int32_t slots;             /* concurrent batches (<= 0: 2)                      */
  int32_t max_batch;         /* requests per batch (<= 0: 64)                     */
} vag_server_opts;

typedef struct {
  vag_mesh mesh;             /* host pointers; everything is copied at submit     */
  vag_props props;
  vag_dirichlet bc;
  const double *phi_m, *phi_f, *cbar;   /* transport data (when n_steps > 0)      */
  const double *c0;          /* optional [n_cv] initial concentration (NULL: cbar
                                on Dirichlet nodes, 0 elsewhere)                 */
  double omega, cfl;
  int32_t n_steps;
  int precision, precond;
  double rtol;
  int32_t maxit;
  double *u_out;             /* host [n_cv] or NULL: pressures ([nodes|ffaces|cells]) */
  double *c_out;             /* host [n_cv] or NULL: c after n_steps; both must stay
                                valid until vag_server_wait returns VAG_OK      */
} vag_request;

typedef struct {
  vag_status status;         /* of the request's batch (VAG_ETIMEOUT: cancelled by
                                vag_server_destroy before it ran)                 */
  vag_solve_info solve;      /* this request's system                            */
  vag_transport_info transport; /* dt_max and dt of this request's system        */
  double latency_ms;         /* submit -> results written                        */
  double queue_ms;           /* submit -> start of its batch                     */
  int32_t batch_size;
} vag_result;

typedef struct {
  uint64_t submitted, completed, rejected, in_queue, in_flight;
  double p50_ms, p99_ms;     /* latency over completed requests                   */
  double solves_per_s;       /* completed / (last completion - first submit)     */
  size_t bytes_reserved, peak_bytes;   /* admission estimates                     */
} vag_server_stats;

vag_status vag_server_create(const vag_server_opts *opts, vag_server **out);
/* Non-blocking.  VAG_EBUDGET if the request alone exceeds the budget (it
 * could never be admitted); VAG_EINVAL for malformed requests. */
vag_status vag_server_submit(vag_server *srv, const vag_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: no limit) for a ticket; VAG_ETIMEOUT when it is
 * not done yet (the ticket stays valid).  After VAG_OK the ticket is released. */
vag_status vag_server_wait(vag_server *srv, uint64_t ticket, int32_t timeout_ms, vag_result *out);
vag_status vag_server_get_stats(vag_server *srv, vag_server_stats *stats);
const char *vag_server_last_error(const vag_server *srv);
/* Cancels queued requests, finishes the batches in flight, joins the slots. */
void vag_server_destroy(vag_server *srv);

/* ------------------------------------------------- allocation-free variant */

/* Largest matrix (rows) vag_spmv_dot_noalloc accepts: its scratch holds one
 * partial sum per 32 rows in a fixed 1 MiB device array. */
#define VAG_NOALLOC_MAX_ROWS (1 << 22)

/*
 * y = A x and *xdoty = x . y for a CSR matrix the caller owns, allocating
 * nothing -- for callers that cannot call cudaMalloc where they need the
 * product (inside their own stream capture, allocation-free serving threads,
 * memory fully reserved by another runtime).  The paper has no counterpart:
 * this is the library's SpMV with the fused dot of its CG iteration, with the
 * block partial sums kept in a fixed file-scope device array (1 MiB plus a
 * counter) that every GPU which loads the library holds until the process
 * exits.
 *   n_rows  rows and columns, 0 <= n_rows <= VAG_NOALLOC_MAX_ROWS (else
 *           VAG_EINVAL, nothing launched);
 *   rowptr [n_rows+1], col [nnz] (int32), val [nnz], x [n_rows], y [n_rows],
 *           xdoty [1]: device pointers owned by the caller; y must not
 *           overlap x (VAG_EINVAL), rowptr, col or val;
 *   stream  cudaStream_t (void*), NULL = the legacy default stream.
 * Stream-ordered: returns without waiting.  VAG_ECUDA if a CUDA call fails.
 * The first call on a device looks up the scratch address (no allocation);
 * make it before any stream capture that includes a call.  The address is
 * kept for the life of the process: after cudaDeviceReset on a device, do not
 * call this entry point on that device again in the same process.  All calls
 * on a device share the scratch: calls whose kernels overlap on the GPU race
 * and must be ordered (same stream, or events).
 */
vag_status vag_spmv_dot_noalloc(int32_t n_rows, const int32_t *rowptr, const int32_t *col, const double *val,
                                const double *x, double *y, double *xdoty, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VAG_H */
