"""CPU oracle for the hybrid-dimensional VAG Darcy solve and upwind transport.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: it exists so that tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` can check the CUDA path against a plain, slow,
obviously-correct FP64 restatement of the paper's scheme.  It shares no code
with the CUDA path; both read the same seeded inputs from ``vag_inputs``.

What it computes, in the paper's order and notation:

* Sec. 3.1 (generalized polyhedral mesh): cell centre x_K, face centres
  x_sigma = sum_s beta_{sigma,s} x_s, the tetrahedral sub-mesh T_{K,sigma,e}.
* Sec. 3.1, Eq. (varformVAG): the Galerkin P1 system on that sub-mesh, with the
  face-centre values of non-fracture faces given by I_sigma and the fracture
  term integrated on the triangles (x_sigma, e) of every fracture face.
* Eq. (VAGFluxMatrix), Eq. (VAGFluxFracture): the transmissivities
  a_{K,nu}^{nu'} and a_{sigma,s}^{s'} and the fluxes F_{K,nu}, F_{sigma,s}.
* Sec. 4.2, Eq. (eqschur) and Eq. (eqschurcell): cell elimination and cell
  recovery (the solve itself is a sparse direct solve of the full system).
* Sec. 3.2: control volumes, Eq. (eq_CFL) and the explicit upwind step with
  the two-point fluxes of Eq. (darcyfluxH).

Readings of points the paper leaves open (shared with the CUDA path only as
prose, never as code):

* beta_{sigma,s} = 1 / |V_sigma| and x_K = isobarycentre of the cell's nodes;
* Lambda_m cellwise constant (full SPD 3x3), Lambda_f, d_f constant per
  fracture face, mu a scalar;
* the Dirichlet node set V_D plays the role of V_ext; other boundary nodes are
  no-flow nodes with a conservation equation and a control volume;
* alpha_{K,s} = omega / |V_K| for s in V_K minus (V_D union V_Gamma), and
  alpha_{sigma,s} = omega / |V_sigma| for s in V_sigma minus V_D;
* the CFL step is computed once from the fluxes.

Floating point: float64 throughout.  DOF order of every global vector:
[nodes | fracture faces | cells].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

CHUNK = 32768  # cells per vectorised batch (memory only; arithmetic unchanged)


# ----------------------------------------------------------------------------
# P1 element matrices
# ----------------------------------------------------------------------------

def tet_p1_stiffness(v, lam):
    """P1 stiffness on tetrahedra: S_ij = |T| grad(l_i)^T Lam grad(l_j).

    v: [B, 4, 3] vertices, lam: [B, 3, 3].  Barycentric gradients are the rows
    of J^{-1}, J = [v1 - v0, v2 - v0, v3 - v0] (columns), and
    grad(l_0) = -(grad(l_1) + grad(l_2) + grad(l_3)).
    Returns (S [B, 4, 4], volume [B]).
    """
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    vol = np.abs(np.linalg.det(J)) / 6.0
    Ginv = np.linalg.inv(J)                         # rows: grad l1, l2, l3
    G = np.concatenate([-Ginv.sum(axis=1, keepdims=True), Ginv], axis=1)  # [B,4,3]
    S = vol[:, None, None] * np.einsum("bia,bac,bjc->bij", G, lam, G)
    return S, vol


def tri_p1_stiffness(v, coef):
    """P1 stiffness of the tangential Laplacian on triangles embedded in 3-D:
    S_ij = |T| coef grad_tau(l_i) . grad_tau(l_j).

    v: [B, 3, 3] vertices, coef: [B].  The tangential gradients of l_1, l_2
    are the rows of the pseudo-inverse of J = [v1 - v0, v2 - v0] (3x2).
    Returns (S [B, 3, 3], area [B]).
    """
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]], axis=2)   # [B,3,2]
    JtJ = np.einsum("bka,bkc->bac", J, J)
    area = 0.5 * np.sqrt(np.linalg.det(JtJ))
    P = np.einsum("bac,bkc->bak", np.linalg.inv(JtJ), J)           # [B,2,3]
    G = np.concatenate([-P.sum(axis=1, keepdims=True), P], axis=1)  # [B,3,3]
    S = (area * coef)[:, None, None] * np.einsum("bia,bja->bij", G, G)
    return S, area


def sym6_to_3x3(l6):
    """(xx, yy, zz, xy, xz, yz) -> 3x3."""
    L = np.empty(l6.shape[:-1] + (3, 3))
    L[..., 0, 0] = l6[..., 0]; L[..., 1, 1] = l6[..., 1]; L[..., 2, 2] = l6[..., 2]
    L[..., 0, 1] = L[..., 1, 0] = l6[..., 3]
    L[..., 0, 2] = L[..., 2, 0] = l6[..., 4]
    L[..., 1, 2] = L[..., 2, 1] = l6[..., 5]
    return L


# ----------------------------------------------------------------------------
# mesh bookkeeping (Sec. 3.1)
# ----------------------------------------------------------------------------

class Mesh:
    """Cells -> faces -> nodes with the sets the paper names: V_K, F_Gamma,K,
    V_sigma, x_K, x_sigma (beta = 1/|V_sigma|).

    ``pb.faces`` [n_faces, q_max] lists each face's nodes in cyclic order,
    padded at the end with -1 where a face has fewer than q_max nodes;
    ``pb.cell_faces`` [n_cells, f_max] is padded the same way.  Cells are
    grouped by the node counts of their faces (in ``cell_faces`` order), so
    every group has one |V_K| and one face layout; ``groups`` lists
    (cells, V_K [B, |V_K|] sorted, face ids [B, n_F], face sizes)."""

    def __init__(self, pb):
        self.xyz = pb.xyz
        self.faces = pb.faces
        self.cell_faces = pb.cell_faces
        self.nv = pb.n_nodes
        self.nc = pb.cell_faces.shape[0]
        self.nF = pb.faces.shape[0]
        self.ff = pb.ff_faces
        self.nf = self.ff.shape[0]
        fvalid = self.faces >= 0
        self.fq = fvalid.sum(axis=1)                          # |V_sigma| of every face
        if np.any(fvalid[:, 1:] & ~fvalid[:, :-1]):
            raise ValueError("face padding must come after the nodes")
        # face id -> fracture-face index (or -1)
        self.face_ff = -np.ones(self.nF, np.int64)
        self.face_ff[self.ff] = np.arange(self.nf)
        if np.all(fvalid):
            self.xS = self.xyz[self.faces].mean(axis=1)       # every face centre
        else:
            f0 = np.where(fvalid, self.faces, 0)
            self.xS = (self.xyz[f0] * fvalid[..., None]).sum(axis=1) / self.fq[:, None]
        # cells grouped by the sizes of their faces
        cf = self.cell_faces
        sizes = np.where(cf >= 0, self.fq[np.where(cf >= 0, cf, 0)], 0)
        sig, gid = np.unique(sizes, axis=0, return_inverse=True)
        self.group_of = gid.reshape(-1)
        self.groups = []
        self.xK = np.zeros((self.nc, 3))
        for g in range(sig.shape[0]):
            cells = np.nonzero(self.group_of == g)[0]
            cols = np.nonzero(sig[g] > 0)[0]
            fids = cf[cells][:, cols]
            fsz = sig[g][cols]
            allnodes = np.sort(np.concatenate([self.faces[fids[:, j]][:, :fsz[j]] for j in range(cols.size)],
                                              axis=1), axis=1)
            keep = np.ones(allnodes.shape, bool)
            keep[:, 1:] = allnodes[:, 1:] != allnodes[:, :-1]
            cnt = keep.sum(axis=1)
            if not np.all(cnt == cnt[0]):
                raise ValueError("cells with the same face sizes but different node counts")
            VK = allnodes[keep].reshape(cells.size, cnt[0])
            self.xK[cells] = self.xyz[VK].mean(axis=1)
            self.groups.append((cells, VK, fids, fsz))
        self.VK = self.groups[0][1] if len(self.groups) == 1 else None
        self.VG = np.zeros(self.nv, bool)                   # V_Gamma
        if self.nf:
            fn = self.faces[self.ff]
            self.VG[np.unique(fn[fn >= 0])] = True


# ----------------------------------------------------------------------------
# local matrices
# ----------------------------------------------------------------------------

def cell_local_matrices(pb, mesh=None, cells=None):
    """Per-cell VAG matrix over the local unknowns (K, V_K, F_Gamma,K):
    M[i, j] = int_K Lambda_m / mu grad(eta_i) . grad(eta_j)  (Eq. VAGFluxMatrix),
    integrated exactly on the tetrahedra T_{K,sigma,e} = conv(x_K, x_sigma, e).

    Returns dict(dofs [B, L] global DOF ids (-1 = unused slot), M [B, L, L],
    vol [B]); local slot 0 is the cell, 1..|V_K| the sorted nodes, then the
    fracture faces of K in the order of its faces.
    """
    m = mesh or Mesh(pb)
    if cells is None:
        cells = np.arange(m.nc)
    cells = np.asarray(cells)
    g = np.unique(m.group_of[cells])
    if g.size != 1:
        raise ValueError("cells of one face layout per call (Mesh.groups)")
    gcells, gVK, gfids, fsz = m.groups[int(g[0])]
    row = np.searchsorted(gcells, cells)
    nv, nf = m.nv, m.nf
    nVK = gVK.shape[1]
    nFK = fsz.size
    L = 1 + nVK + nFK
    B = cells.shape[0]
    dofs = -np.ones((B, L), np.int64)
    dofs[:, 0] = nv + nf + cells
    dofs[:, 1:1 + nVK] = gVK[row]
    cf = gfids[row]                               # [B, nFK]
    cff = m.face_ff[cf]                           # fracture index or -1
    slot_of_face = np.full(cf.shape, -1)
    isff = cff >= 0
    rank = np.cumsum(isff, axis=1) - 1
    slot_of_face[isff] = 1 + nVK + rank[isff]
    rows = np.nonzero(isff)
    dofs[rows[0], slot_of_face[isff]] = nv + cff[isff]
    M = np.zeros((B, L, L))
    vol = np.zeros(B)
    lam = sym6_to_3x3(pb.lambda_m[cells]) / pb.mu
    xK = m.xK[cells]
    VKc = gVK[row]
    bidx = np.arange(B)
    for f in range(nFK):
        fid = cf[:, f]
        q = int(fsz[f])
        fnodes = m.faces[fid][:, :q]              # [B, q] cyclic
        xs = m.xS[fid]
        for e in range(q):
            a = fnodes[:, e]
            b = fnodes[:, (e + 1) % q]
            v = np.stack([xK, xs, m.xyz[a], m.xyz[b]], axis=1)
            S, tv = tet_p1_stiffness(v, lam)
            vol += tv
            W = np.zeros((B, 4, L))
            W[:, 0, 0] = 1.0
            # vertex x_sigma: the fracture-face unknown, or I_sigma on nodes
            ff_here = isff[:, f]
            W[bidx[ff_here], 1, slot_of_face[ff_here, f]] = 1.0
            for t in range(q):
                pos = 1 + np.sum(VKc < fnodes[:, t:t + 1], axis=1)
                W[bidx[~ff_here], 1, pos[~ff_here]] += 1.0 / q
            pa = 1 + np.sum(VKc < a[:, None], axis=1)
            pbb = 1 + np.sum(VKc < b[:, None], axis=1)
            W[bidx, 2, pa] = 1.0
            W[bidx, 3, pbb] = 1.0
            M += np.matmul(np.matmul(W.transpose(0, 2, 1), S), W)   # W^T S W
    return dict(cells=cells, dofs=dofs, M=M, vol=vol)


def fracture_local_matrices(pb, mesh=None):
    """Per-fracture-face matrix over (sigma, V_sigma):
    M[i, j] = int_sigma d_f Lambda_f / mu grad_tau(eta_i) . grad_tau(eta_j)
    (Eq. VAGFluxFracture) on the triangles (x_sigma, e).
    Returns dict(dofs [nf, 1+Q], M [nf, 1+Q, 1+Q], area [nf]) with Q the
    largest |V_sigma|; a face with fewer nodes has dof -1 and zero rows and
    columns in its unused slots."""
    m = mesh or Mesh(pb)
    nv, nf = m.nv, m.nf
    fn = m.faces[m.ff]                            # [nf, Q] cyclic, -1 padded
    Q = fn.shape[1]
    qf = m.fq[m.ff]
    xs = m.xS[m.ff]
    coef = pb.d_f * pb.lambda_f / pb.mu
    M = np.zeros((nf, 1 + Q, 1 + Q))
    area = np.zeros(nf)
    for q in np.unique(qf):
        sel = np.nonzero(qf == q)[0]
        for e in range(q):
            a = fn[sel, e]; b = fn[sel, (e + 1) % q]
            v = np.stack([xs[sel], m.xyz[a], m.xyz[b]], axis=1)
            S, ar = tri_p1_stiffness(v, coef[sel])
            area[sel] += ar
            idx = [0, 1 + e, 1 + (e + 1) % q]
            for i in range(3):
                for j in range(3):
                    M[sel, idx[i], idx[j]] += S[:, i, j]
    dofs = np.concatenate([(nv + np.arange(nf))[:, None], fn], axis=1)
    return dict(dofs=dofs, M=M, area=area)


def _all_cell_matrices(pb, mesh):
    out = []
    for cells, _, _, _ in mesh.groups:
        for s in range(0, cells.size, CHUNK):
            out.append(cell_local_matrices(pb, mesh, cells[s:s + CHUNK]))
    return out


# ----------------------------------------------------------------------------
# global system, elimination, solve (Sec. 3.1 and Sec. 4.2)
# ----------------------------------------------------------------------------

def assemble_full(pb, mesh=None, cellmats=None, fracmats=None):
    """Full Galerkin matrix over X_D, ordered [nodes | ffaces | cells]."""
    m = mesh or Mesh(pb)
    n = m.nv + m.nf + m.nc
    cellmats = cellmats if cellmats is not None else _all_cell_matrices(pb, m)
    fracmats = fracmats if fracmats is not None else fracture_local_matrices(pb, m)
    rows, cols, vals = [], [], []
    for cm in cellmats:
        d = cm["dofs"]; M = cm["M"]
        L = d.shape[1]
        R = np.repeat(d[:, :, None], L, axis=2)
        C = np.repeat(d[:, None, :], L, axis=1)
        ok = (R >= 0) & (C >= 0)
        rows.append(R[ok]); cols.append(C[ok]); vals.append(M[ok])
    if m.nf:
        d = fracmats["dofs"]; M = fracmats["M"]
        L = d.shape[1]
        R = np.repeat(d[:, :, None], L, axis=2)
        C = np.repeat(d[:, None, :], L, axis=1)
        ok = (R >= 0) & (C >= 0)
        rows.append(R[ok]); cols.append(C[ok]); vals.append(M[ok])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def peaceman_wi(dx, dz, d_f, lam_f, r_w, mu=1.0):
    """Sec. 5.5: well index of a vertical well of radius r_w through a
    fracture face seen as a box dx x d_f x dz (dx the face's horizontal
    edge, dz its height): WI = 2 pi dz Lambda_f / (mu log(r_0 / r_w)) with
    r_0 = D exp(-2 pi dz / C), C = 4/3 (dx dz/d_f + dx d_f/dz + dz d_f/dx),
    D = sqrt(dx^2 + d_f^2) / 2.  (C is the cell diagonal of the VAG scheme
    on that box with unit permeability; the paper's expression has mu = 1.)"""
    dx, dz, d_f, lam_f, r_w = (np.asarray(a, np.float64) for a in (dx, dz, d_f, lam_f, r_w))
    C = 4.0 / 3.0 * (dx * dz / d_f + dx * d_f / dz + dz * d_f / dx)
    D = 0.5 * np.sqrt(dx ** 2 + d_f ** 2)
    r0 = D * np.exp(-2.0 * np.pi * dz / C)
    return 2.0 * np.pi * dz * lam_f / (mu * np.log(r0 / r_w))


def well_terms(pb):
    """Peaceman wells of ``pb.wells`` (per perforation: fracture face ff,
    WI, p_w, imposed rate q, injected concentration c_in).  The rate leaving
    face sigma into the well, q_p = WI (u_sigma - p_w) - q, enters the face's
    conservation equation: WI goes to its diagonal and WI p_w + q to its
    right-hand side.  Returns (d, g) over the full DOFs, or (None, None)."""
    w = getattr(pb, "wells", None)
    if not w:
        return None, None
    n = pb.n_nodes + pb.n_ff + pb.n_cells
    dof = pb.n_nodes + np.asarray(w["ff"], np.int64)
    d = np.zeros(n); g = np.zeros(n)
    np.add.at(d, dof, w["wi"])
    np.add.at(g, dof, np.asarray(w["wi"]) * np.asarray(w["pw"]) + np.asarray(w["q"]))
    return d, g


def well_rates(pb, u):
    """q_p = WI (u_sigma - p_w) - q for every perforation."""
    w = pb.wells
    return np.asarray(w["wi"]) * (u[pb.n_nodes + np.asarray(w["ff"], np.int64)] - np.asarray(w["pw"])) \
        - np.asarray(w["q"])


def split_dofs(pb):
    nv, nf, nc = pb.n_nodes, pb.n_ff, pb.n_cells
    isdir = np.zeros(nv + nf + nc, bool)
    isdir[pb.dir_nodes] = True
    R = np.nonzero(~isdir[:nv + nf])[0]          # (V \ V_D) u F_Gamma, in order
    C = nv + nf + np.arange(nc)
    D = np.asarray(pb.dir_nodes, np.int64)
    return R, C, D


def schur_system(pb, A=None, mesh=None, g=None):
    """Eq. (eqschur): eliminate the cell unknowns (A_cc is diagonal).
    Rows/columns: the non-Dirichlet nodes in increasing id, then the fracture
    faces; g: an optional source over the full DOFs (the wells).  Returns
    (S csr, b, R)."""
    A = A if A is not None else assemble_full(pb, mesh)
    R, C, D = split_dofs(pb)
    uD = pb.dir_values
    A_RR = A[R][:, R]; A_RC = A[R][:, C]; A_CR = A[C][:, R]
    A_CC = A[C][:, C].diagonal()
    b_R = -(A[R][:, D] @ uD)
    b_C = -(A[C][:, D] @ uD)
    if g is not None:
        b_R = b_R + g[R]
        b_C = b_C + g[C]
    S = (A_RR - A_RC @ sp.diags(1.0 / A_CC) @ A_CR).tocsr()
    b = b_R - A_RC @ (b_C / A_CC)
    S.sort_indices()
    return S, b, R


def solve_full(pb, A=None, mesh=None, g=None):
    """Direct sparse solve of the full Galerkin system with the Dirichlet
    values substituted (and an optional source g over the full DOFs).
    Returns u over [nodes | ffaces | cells]."""
    A = A if A is not None else assemble_full(pb, mesh)
    n = A.shape[0]
    isdir = np.zeros(n, bool); isdir[pb.dir_nodes] = True
    U = np.nonzero(~isdir)[0]
    u = np.zeros(n)
    u[pb.dir_nodes] = pb.dir_values
    rhs = -(A[U][:, pb.dir_nodes] @ pb.dir_values)
    if g is not None:
        rhs = rhs + g[U]
    u[U] = spla.spsolve(A[U][:, U].tocsc(), rhs)
    return u


def solve_schur_direct(pb, A=None, mesh=None, g=None):
    """Solve Eq. (eqschur) directly, then recover the cells by Eq. (eqschurcell)."""
    A = A if A is not None else assemble_full(pb, mesh)
    S, b, R = schur_system(pb, A, g=g)
    n = A.shape[0]
    u = np.zeros(n)
    u[pb.dir_nodes] = pb.dir_values
    u[R] = spla.spsolve(S.tocsc(), b)
    return recover_cells(pb, A, u)


def recover_cells(pb, A, u):
    """Eq. (eqschurcell): U_c = A_cc^{-1}(b_c - A_cv U_v - A_cf U_f), where the
    Dirichlet columns of A_cv sit in b_c."""
    _, C, _ = split_dofs(pb)
    nonc = np.arange(pb.n_nodes + pb.n_ff)
    Acn = A[C][:, nonc]
    u = u.copy()
    u[C] = -(Acn @ u[nonc]) / A[C][:, C].diagonal()
    return u


def pcg_jacobi(A, b, rtol=1e-14, maxit=100000, x0=None):
    """Textbook Jacobi-preconditioned CG (used only where a direct solve is too
    large).  Stops at ||r|| <= rtol ||b|| or when ||r|| stops decreasing for 50
    iterations."""
    d = A.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    z = r / d
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    best = np.inf; stall = 0
    for it in range(maxit):
        nr = np.linalg.norm(r)
        if nr <= rtol * nb:
            break
        if nr < best:
            best = nr; stall = 0
        else:
            stall += 1
            if stall > 50:
                break
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


# ----------------------------------------------------------------------------
# fluxes (Eq. VAGFluxMatrix, Eq. VAGFluxFracture)
# ----------------------------------------------------------------------------

def cell_fluxes(cm, u):
    """F_{K,nu} = sum_{nu'} a_{K,nu}^{nu'} (u_K - u_{nu'}) with
    a_{K,nu}^{nu'} = M[nu, nu'] over nu, nu' in V_K u F_Gamma,K.
    Returns F [B, L-1] aligned with cm['dofs'][:, 1:] (0 where unused)."""
    d = cm["dofs"]; M = cm["M"]
    a = M[:, 1:, 1:]
    valid = d[:, 1:] >= 0
    uK = u[d[:, 0]]
    un = np.where(valid, u[np.where(valid, d[:, 1:], 0)], 0.0)
    diff = np.where(valid, uK[:, None] - un, 0.0)
    F = np.einsum("bij,bj->bi", a, diff)
    return np.where(valid, F, 0.0)


def fracture_fluxes(fm, u):
    """F_{sigma,s} = sum_{s'} a_{sigma,s}^{s'} (u_sigma - u_{s'})."""
    d = fm["dofs"]; M = fm["M"]
    a = M[:, 1:, 1:]
    valid = d[:, 1:] >= 0
    diff = np.where(valid, u[d[:, 0]][:, None] - u[np.where(valid, d[:, 1:], 0)], 0.0)
    return np.einsum("bij,bj->bi", a, diff)


# ----------------------------------------------------------------------------
# transport (Sec. 3.2)
# ----------------------------------------------------------------------------

class Transport:
    """Control volumes, CFL step and the explicit upwind scheme.

    Edges: (K, nu) for nu in V_K u F_Gamma,K carrying F_{K,nu}, and
    (sigma, s) for s in V_sigma carrying F_{sigma,s}.  Global CV ids follow
    the [nodes | ffaces | cells] order.
    """

    def __init__(self, pb, cellmats, fracmats, F_cell, F_frac, omega=0.5, mesh=None, well_rates=None):
        m = mesh or Mesh(pb)
        nv, nf, nc = m.nv, m.nf, m.nc
        self.n = nv + nf + nc
        # well perforations (Sec. 5.5): rate q_p leaving face sigma into the
        # well; a negative rate enters the face at the injected concentration
        w = getattr(pb, "wells", None)
        if w:
            self.w_cv = nv + np.asarray(w["ff"], np.int64)
            self.w_F = np.asarray(well_rates, np.float64)
            self.w_cin = np.asarray(w["cin"], np.float64)
        else:
            self.w_cv = np.zeros(0, np.int64); self.w_F = np.zeros(0); self.w_cin = np.zeros(0)
        isdir = np.zeros(nv, bool); isdir[pb.dir_nodes] = True
        self.isdir = isdir
        self.dir_nodes = pb.dir_nodes
        self.cbar = pb.cbar
        # edges
        src, dst, flx = [], [], []
        vol = np.zeros(nc)
        for cm, F in zip(cellmats, F_cell):
            d = cm["dofs"]
            K = np.repeat(d[:, :1], d.shape[1] - 1, axis=1)
            ok = d[:, 1:] >= 0
            src.append(K[ok]); dst.append(d[:, 1:][ok]); flx.append(F[ok])
            vol[cm["cells"]] = cm["vol"]
        if nf:
            d = fracmats["dofs"]
            S = np.repeat(d[:, :1], d.shape[1] - 1, axis=1)
            ok = d[:, 1:] >= 0
            src.append(S[ok]); dst.append(d[:, 1:][ok]); flx.append(F_frac[ok])
        self.src = np.concatenate(src); self.dst = np.concatenate(dst); self.F = np.concatenate(flx)
        # porous volumes (Sec. 3.2.1)
        phi = np.zeros(self.n)
        pv_cell = vol * pb.phi_m
        for cells, VK, _, _ in m.groups:
            nVK = VK.shape[1]
            elig = ~(isdir[VK] | m.VG[VK])                  # s in V_K \ (V_D u V_Gamma)
            aK = omega / nVK
            phi[nv + nf + cells] = (1.0 - aK * elig.sum(axis=1)) * pv_cell[cells]
            np.add.at(phi, VK[elig], np.repeat(aK * pv_cell[cells][:, None], nVK, axis=1)[elig])
        if nf:
            fn = m.faces[m.ff]
            valid = fn >= 0
            q = m.fq[m.ff]
            eligf = valid & ~isdir[np.where(valid, fn, 0)]
            af = omega / q
            pv_ff = pb.d_f * fracmats["area"] * pb.phi_f
            phi[nv:nv + nf] = (1.0 - af * eligf.sum(axis=1)) * pv_ff
            np.add.at(phi, fn[eligf], np.repeat((af * pv_ff)[:, None], fn.shape[1], axis=1)[eligf])
        phi[pb.dir_nodes] = 0.0
        self.phi = phi
        self.vol = vol

    def outflow(self):
        """Per CV: sum of the fluxes leaving it (the denominators of Eq. eq_CFL)."""
        out = np.zeros(self.n)
        np.add.at(out, self.src, np.maximum(self.F, 0.0))
        np.add.at(out, self.dst, np.maximum(-self.F, 0.0))
        np.add.at(out, self.w_cv, np.maximum(self.w_F, 0.0))
        return out

    def cfl_dt(self):
        """min over cells, fracture faces and non-Dirichlet nodes of
        phi_mu / (outgoing flux), Eq. (eq_CFL)."""
        out = self.outflow()
        active = np.ones(self.n, bool)
        active[self.dir_nodes] = False
        with np.errstate(divide="ignore"):
            r = np.where(out[active] > 0, self.phi[active] / out[active], np.inf)
        return float(np.min(r))

    def _well_H(self, c):
        """Upwind well terms: q c_sigma for production, q c_in for injection."""
        return np.where(self.w_F > 0.0, c[self.w_cv] * self.w_F, self.w_cin * self.w_F)

    def step(self, c, dt):
        """One explicit Euler step with the upwind fluxes of Eq. (darcyfluxH):
        H = c_src F^+ + c_dst F^-; the source CV of each edge loses H, the
        destination gains it; a well takes H = q c_sigma (q > 0) or q c_in
        (q < 0) from its face; Dirichlet nodes are reset to cbar."""
        H = c[self.src] * np.maximum(self.F, 0.0) + c[self.dst] * np.minimum(self.F, 0.0)
        net = np.zeros(self.n)
        np.add.at(net, self.src, -H)
        np.add.at(net, self.dst, H)
        np.add.at(net, self.w_cv, -self._well_H(c))
        cn = c.copy()
        act = np.ones(self.n, bool); act[self.dir_nodes] = False
        cn[act] = c[act] + dt / self.phi[act] * net[act]
        cn[self.dir_nodes] = self.cbar
        return cn

    def boundary_inflow(self, c):
        """Net upwind flux entering the non-Dirichlet CVs through edges that
        touch a Dirichlet node, and through the wells (the only terms that do
        not cancel in the total mass)."""
        H = c[self.src] * np.maximum(self.F, 0.0) + c[self.dst] * np.minimum(self.F, 0.0)
        dd = self.isdir_full(self.dst)
        ds = self.isdir_full(self.src)
        return float(np.sum(-H[dd & ~ds]) + np.sum(H[ds & ~dd]) - np.sum(self._well_H(c)))

    def isdir_full(self, ids):
        out = np.zeros(ids.shape, bool)
        nd = ids < self.isdir.shape[0]
        out[nd] = self.isdir[ids[nd]]
        return out


# ----------------------------------------------------------------------------
# the whole path in one call
# ----------------------------------------------------------------------------

class DarcyTransport:
    """Assemble, solve, recover, fluxes, control volumes and CFL step."""

    def __init__(self, pb, omega=0.5, solver="auto", rtol=1e-14):
        self.pb = pb
        self.mesh = Mesh(pb)
        self.cellmats = _all_cell_matrices(pb, self.mesh)
        self.fracmats = fracture_local_matrices(pb, self.mesh)
        self.A = assemble_full(pb, self.mesh, self.cellmats, self.fracmats)
        wd, g = well_terms(pb)
        Aw = self.A if wd is None else (self.A + sp.diags(wd)).tocsr()   # the system with the wells
        if solver == "auto":
            solver = "direct" if self.A.shape[0] <= 30000 else "schur_pcg"
        self.solver = solver
        if solver == "direct":
            self.u = solve_full(pb, Aw, g=g)
        elif solver == "schur_direct":
            self.u = solve_schur_direct(pb, Aw, g=g)
        elif solver == "schur_pcg":
            S, b, R = schur_system(pb, Aw, g=g)
            x, self.iters = pcg_jacobi(S, b, rtol=rtol)
            u = np.zeros(self.A.shape[0]); u[pb.dir_nodes] = pb.dir_values; u[R] = x
            self.u = recover_cells(pb, Aw, u)
        else:
            raise ValueError(solver)
        self.F_cell = [cell_fluxes(cm, self.u) for cm in self.cellmats]
        self.F_frac = fracture_fluxes(self.fracmats, self.u) if pb.n_ff else np.zeros((0, 4))
        self.q_well = well_rates(pb, self.u) if wd is not None else np.zeros(0)
        self.tr = Transport(pb, self.cellmats, self.fracmats, self.F_cell, self.F_frac,
                            omega=omega, mesh=self.mesh, well_rates=self.q_well)

    def run_transport(self, n_steps, cfl=0.9, c=None):
        dt = cfl * self.tr.cfl_dt()
        c = self.pb.c0() if c is None else c
        for _ in range(n_steps):
            c = self.tr.step(c, dt)
        return c, dt

    def run_to_time(self, T, c=None):
        """Sec. 4.3 time stepping: dt = the CFL maximum, N = ceil(T / dt), the
        last step shortened to reach T exactly."""
        dt = self.tr.cfl_dt()
        N = int(np.ceil(T / dt))
        c = self.pb.c0() if c is None else c
        for n in range(N):
            h = dt if n < N - 1 else T - (N - 1) * dt
            c = self.tr.step(c, h)
        return c, dt, N


def stationary_concentration(tr: Transport):
    """Steady state of the upwind scheme of Sec. 3.2: the concentrations for
    which every non-Dirichlet control volume has zero net upwind flux (the
    limit of the explicit iteration, independent of phi and dt), with the
    Dirichlet nodes held at cbar.  Sparse direct solve."""
    n = tr.n
    Fp = np.maximum(tr.F, 0.0); Fm = np.minimum(tr.F, 0.0)
    wp = tr.w_F > 0.0
    r = np.concatenate([tr.src, tr.src, tr.dst, tr.dst, tr.w_cv[wp]])
    c = np.concatenate([tr.src, tr.dst, tr.src, tr.dst, tr.w_cv[wp]])
    v = np.concatenate([-Fp, -Fm, Fp, Fm, -tr.w_F[wp]])
    B = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    inj = np.zeros(n)                                      # injection: -q c_in enters the face
    np.add.at(inj, tr.w_cv[~wp], -tr.w_F[~wp] * tr.w_cin[~wp])
    isd = np.zeros(n, bool); isd[tr.dir_nodes] = True
    U = np.nonzero(~isd)[0]
    cfull = np.zeros(n)
    cfull[tr.dir_nodes] = tr.cbar
    rhs = -(B[U][:, tr.dir_nodes] @ tr.cbar) - inj[U]
    cfull[U] = spla.spsolve(B[U][:, U].tocsc(), rhs)
    return cfull
