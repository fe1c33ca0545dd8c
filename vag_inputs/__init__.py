"""Seeded synthetic inputs for the hybrid-dimensional VAG Darcy + transport path.

This module only *describes problems*: node coordinates, hexahedral cell
connectivity, the unique faces of the mesh, which faces carry a fracture,
permeabilities, apertures, porosities and boundary data.  It holds none of the
scheme's arithmetic (no gradients, no transmissivities, no fluxes), so both the
CUDA path and the CPU oracle can consume the same inputs without sharing any
of the method.

Mesh conventions (Sec. 3.1 of the paper: generalized polyhedral meshes
conforming to the fracture network):

* ``xyz``        float64 [n_nodes, 3]
* ``cell_nodes`` int32   [n_cells, 8]   hexahedron, node ``l`` sits at the
  lattice offset ``(l & 1, (l >> 1) & 1, (l >> 2) & 1)`` of the cell (the
  tetrahedral, prismatic and pyramidal generators list their own node
  counts, -1-padded to 8 where shapes mix).
* ``faces``      int32   [n_faces, 4]   every face of the mesh once, nodes in
  cyclic order (consecutive entries share an edge); a triangle has -1 in
  its last slot (a tetrahedral mesh has [n_faces, 3]).
* ``cell_faces`` int32   [n_cells, 6]   face ids of each cell, -1 after the
  last face of a cell with fewer than six.
* ``ff_faces``   int32   [n_ff]         ids (into ``faces``) of the fracture
  faces, sorted; ``ff_nodes = faces[ff_faces]``.
* ``lambda_m``   float64 [n_cells, 6]   symmetric matrix permeability tensor
  (xx, yy, zz, xy, xz, yz).
* ``lambda_f``, ``d_f`` float64 [n_ff]  isotropic tangential fracture
  permeability and aperture.
* ``dir_nodes`` int32 [n_dir] (sorted), ``dir_values`` float64 [n_dir]:
  Dirichlet pressure; every other boundary node is a no-flow node.
* ``phi_m`` [n_cells], ``phi_f`` [n_ff]: porosities; ``cbar`` [n_dir]: the
  Dirichlet concentrations.
* ``wells`` (optional, ``well_arrays``): per perforation the fracture face
  ``ff``, well index ``wi``, well pressure ``pw``, imposed rate ``q`` and
  injected concentration ``cin``; ``meta["well_geometry"]`` holds what the
  Peaceman index is computed from.

All random draws come from ``numpy.random.default_rng(seed)`` in a fixed order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Problem", "hex_lattice", "axis_fracture_faces", "build_problem",
    "config_plain16", "config_scale64", "config_mixed128", "random_dfn_problem",
    "one_fracture_problem", "four_fracture_problem", "batch_problems", "tet_problem", "prism_problem",
    "pyramid_problem", "well_problem", "well_arrays", "config_tet54", "config_prism55",
]


@dataclass
class Problem:
    dims: Tuple[int, int, int]
    xyz: np.ndarray
    cell_nodes: np.ndarray
    faces: np.ndarray
    cell_faces: np.ndarray
    ff_faces: np.ndarray
    ff_nodes: np.ndarray
    ff_frac: np.ndarray
    lambda_m: np.ndarray
    lambda_f: np.ndarray
    d_f: np.ndarray
    mu: float
    dir_nodes: np.ndarray
    dir_values: np.ndarray
    phi_m: np.ndarray
    phi_f: np.ndarray
    cbar: np.ndarray
    meta: dict = field(default_factory=dict)
    wells: Optional[dict] = None

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cell_nodes.shape[0])

    @property
    def n_ff(self) -> int:
        return int(self.ff_faces.shape[0])

    def c0(self) -> np.ndarray:
        """Initial concentration in the [nodes | ffaces | cells] order: the
        Dirichlet value on Dirichlet nodes, zero elsewhere."""
        c = np.zeros(self.n_nodes + self.n_ff + self.n_cells)
        c[self.dir_nodes] = self.cbar
        return c


# ----------------------------------------------------------------------------
# structured hexahedral lattice (topologically Cartesian)
# ----------------------------------------------------------------------------

def _nid(dims, i, j, k):
    nx, ny, nz = dims
    return i + (nx + 1) * (j + (ny + 1) * k)


def hex_lattice(dims):
    """Connectivity of an nx*ny*nz hexahedral lattice.

    Returns (cell_nodes, faces, cell_faces, face_axis, face_ijk) where face ids
    are grouped as x-normal, y-normal, z-normal lattice faces.
    """
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i = i.ravel(); j = j.ravel(); k = k.ravel()
    cell_nodes = np.stack([
        _nid(dims, i + (l & 1), j + ((l >> 1) & 1), k + ((l >> 2) & 1)) for l in range(8)
    ], axis=1).astype(np.int32)

    # x-normal faces at (i, j, k), i in 0..nx, j < ny, k < nz
    kx, jx, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx + 1), indexing="ij")
    ix = ix.ravel(); jx = jx.ravel(); kx = kx.ravel()
    fx = np.stack([_nid(dims, ix, jx, kx), _nid(dims, ix, jx + 1, kx),
                   _nid(dims, ix, jx + 1, kx + 1), _nid(dims, ix, jx, kx + 1)], axis=1)
    ky, jy, iy = np.meshgrid(np.arange(nz), np.arange(ny + 1), np.arange(nx), indexing="ij")
    iy = iy.ravel(); jy = jy.ravel(); ky = ky.ravel()
    fy = np.stack([_nid(dims, iy, jy, ky), _nid(dims, iy + 1, jy, ky),
                   _nid(dims, iy + 1, jy, ky + 1), _nid(dims, iy, jy, ky + 1)], axis=1)
    kz, jz, iz = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    iz = iz.ravel(); jz = jz.ravel(); kz = kz.ravel()
    fz = np.stack([_nid(dims, iz, jz, kz), _nid(dims, iz + 1, jz, kz),
                   _nid(dims, iz + 1, jz + 1, kz), _nid(dims, iz, jz + 1, kz)], axis=1)
    faces = np.concatenate([fx, fy, fz]).astype(np.int32)
    nfx = fx.shape[0]; nfy = fy.shape[0]

    def xf(ii, jj, kk):
        return ii + (nx + 1) * (jj + ny * kk)

    def yf(ii, jj, kk):
        return nfx + ii + nx * (jj + (ny + 1) * kk)

    def zf(ii, jj, kk):
        return nfx + nfy + ii + nx * (jj + ny * kk)

    cell_faces = np.stack([xf(i, j, k), xf(i + 1, j, k), yf(i, j, k), yf(i, j + 1, k),
                           zf(i, j, k), zf(i, j, k + 1)], axis=1).astype(np.int32)
    face_axis = np.concatenate([np.zeros(nfx), np.ones(nfy), 2 * np.ones(fz.shape[0])]).astype(np.int8)
    face_ijk = np.concatenate([np.stack([ix, jx, kx], 1), np.stack([iy, jy, ky], 1),
                               np.stack([iz, jz, kz], 1)]).astype(np.int64)
    return cell_nodes, faces, cell_faces, face_axis, face_ijk


def axis_fracture_faces(dims, axis, plane, lo_a, hi_a, lo_b, hi_b):
    """Face ids of an axis-aligned rectangle lying on lattice node plane
    ``plane`` normal to ``axis``; (lo_a, hi_a) x (lo_b, hi_b) are cell-index
    ranges in the two other axes, in increasing axis order."""
    nx, ny, nz = dims
    nfx = (nx + 1) * ny * nz
    nfy = nx * (ny + 1) * nz
    a = np.arange(lo_a, hi_a)
    b = np.arange(lo_b, hi_b)
    A, B = np.meshgrid(a, b, indexing="ij")
    A = A.ravel(); B = B.ravel()
    if axis == 0:
        ids = plane + (nx + 1) * (A + ny * B)
    elif axis == 1:
        ids = nfx + A + nx * (plane + (ny + 1) * B)
    else:
        ids = nfx + nfy + A + nx * (B + ny * plane)
    return ids.astype(np.int64)


def _lattice_xyz(dims):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel() / nx, j.ravel() / ny, k.ravel() / nz], axis=1).astype(np.float64)


def _jitter(dims, xyz, faces, ff_faces, face_axis, amp, rng):
    """Perturb interior nodes uniformly by +-amp*h per coordinate, keeping each
    fracture face planar: a node on a fracture plane keeps that plane's normal
    coordinate."""
    nx, ny, nz = dims
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    d = rng.uniform(-amp, amp, size=xyz.shape) * h[None, :]
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    boundary = ((i == 0) | (i == nx) | (j == 0) | (j == ny) | (k == 0) | (k == nz)).ravel()
    d[boundary] = 0.0
    for ax in range(3):
        sel = ff_faces[face_axis[ff_faces] == ax]
        if sel.size:
            frozen = np.unique(faces[sel].ravel())
            d[frozen, ax] = 0.0
    return xyz + d


def _lognormal_aniso(n_cells, rng, log10_std=1.0, aniso=10.0):
    """Cellwise tensor k_K (I + (aniso-1) a a^T), log10 k_K ~ N(0, std), one
    seeded unit axis a for the whole field."""
    logk = rng.normal(0.0, log10_std, size=n_cells)
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    k = 10.0 ** logk
    t = aniso - 1.0
    lam = np.empty((n_cells, 6))
    lam[:, 0] = k * (1 + t * a[0] * a[0])
    lam[:, 1] = k * (1 + t * a[1] * a[1])
    lam[:, 2] = k * (1 + t * a[2] * a[2])
    lam[:, 3] = k * t * a[0] * a[1]
    lam[:, 4] = k * t * a[0] * a[2]
    lam[:, 5] = k * t * a[1] * a[2]
    return lam


def build_problem(dims, fractures: Sequence[Tuple], *, jitter=0.0, seed=0,
                  lam_m="identity", ratio=1e4, d_f=1e-2, phi_m=0.2, phi_f=0.4,
                  xyz=None, frac_lambda: Optional[Sequence[float]] = None,
                  frac_df: Optional[Sequence[float]] = None,
                  dirichlet="x", meta=None) -> Problem:
    """Assemble a Problem on a hexahedral lattice.

    ``fractures``: list of (axis, plane, lo_a, hi_a, lo_b, hi_b) rectangles, or
    lists of raw face ids (for meshes whose fracture is not axis-aligned).
    Overlapping rectangles on one plane merge; each face is one fracture face.
    ``dirichlet="x"``: p = 1 - x on the x = 0 and x = 1 faces (inflow c = 1 on
    x = 0), no-flow elsewhere.
    """
    rng = np.random.default_rng(seed)
    cell_nodes, faces, cell_faces, face_axis, _ = hex_lattice(dims)
    ids, owner = [], []
    for f_idx, fr in enumerate(fractures):
        if isinstance(fr, np.ndarray):
            fid = fr.astype(np.int64)
        else:
            fid = axis_fracture_faces(dims, *fr)
        ids.append(fid)
        owner.append(np.full(fid.shape, f_idx))
    if ids:
        allid = np.concatenate(ids)
        allown = np.concatenate(owner)
        ff_faces, first = np.unique(allid, return_index=True)
        ff_frac = allown[first].astype(np.int32)
    else:
        ff_faces = np.zeros(0, np.int64)
        ff_frac = np.zeros(0, np.int32)
    ff_faces = ff_faces.astype(np.int32)
    if xyz is None:
        xyz = _lattice_xyz(dims)
        if jitter > 0:
            xyz = _jitter(dims, xyz, faces, ff_faces, face_axis, jitter, rng)
    n_cells = cell_nodes.shape[0]
    if isinstance(lam_m, np.ndarray):
        lam = lam_m
        med = 1.0
    elif lam_m == "identity":
        lam = np.zeros((n_cells, 6)); lam[:, :3] = 1.0
        med = 1.0
    elif lam_m == "lognormal":
        lam = _lognormal_aniso(n_cells, rng)
        med = 1.0   # median of k_K: log10 mean 0
    else:
        raise ValueError(lam_m)
    nff = ff_faces.shape[0]
    if frac_lambda is not None:
        lam_f = np.asarray(frac_lambda, np.float64)[ff_frac]
    else:
        lam_f = np.full(nff, ratio * med)
    if frac_df is not None:
        dff = np.asarray(frac_df, np.float64)[ff_frac]
    else:
        dff = np.full(nff, d_f)
    if dirichlet == "x":
        nx, ny, nz = dims
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        i = i.ravel()
        left = np.nonzero(i == 0)[0]; right = np.nonzero(i == nx)[0]
        dir_nodes = np.concatenate([left, right])
        order = np.argsort(dir_nodes)
        dir_nodes = dir_nodes[order].astype(np.int32)
        dir_values = (1.0 - xyz[dir_nodes, 0])
        cbar = np.where(np.isin(dir_nodes, left), 1.0, 0.0)
    else:
        dir_nodes, dir_values, cbar = dirichlet
        dir_nodes = np.asarray(dir_nodes, np.int32)
    return Problem(
        dims=tuple(dims), xyz=np.ascontiguousarray(xyz, np.float64),
        cell_nodes=cell_nodes, faces=faces, cell_faces=cell_faces,
        ff_faces=ff_faces, ff_nodes=np.ascontiguousarray(faces[ff_faces]).astype(np.int32),
        ff_frac=ff_frac, lambda_m=np.ascontiguousarray(lam, np.float64),
        lambda_f=lam_f, d_f=dff, mu=1.0,
        dir_nodes=dir_nodes, dir_values=np.asarray(dir_values, np.float64),
        phi_m=np.full(n_cells, float(phi_m)), phi_f=np.full(nff, float(phi_f)),
        cbar=np.asarray(cbar, np.float64), meta=dict(meta or {}))


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def config_plain16(n=16) -> Problem:
    """Unit cube, n^3 hex cells, one fracture on the node plane x = 0.5,
    Lambda_m = I, d_f = 1e-2, Lambda_f = 1e4 (K_f d_f = 1e2), p = 1 - x on
    x = 0/1, porosities 0.2 / 0.4, inflow c = 1 on x = 0."""
    dims = (n, n, n)
    return build_problem(dims, [(0, n // 2, 0, n, 0, n)], ratio=1e4,
                         meta={"name": f"plain{n}", "seed": None})


def config_scale64(n=64, seed=1234) -> Problem:
    """n^3 jittered (+-20% h) hex mesh with four fractures x=.5, y=.5, z=.5 and
    x=.25 restricted to y<.5; lognormal (log10 std 1) matrix permeability with
    10:1 anisotropy along a seeded axis; fracture/matrix ratio 1e4."""
    h = n // 2
    fr = [(0, h, 0, n, 0, n), (1, h, 0, n, 0, n), (2, h, 0, n, 0, n), (0, n // 4, 0, h, 0, n)]
    return build_problem((n, n, n), fr, jitter=0.2, seed=seed, lam_m="lognormal",
                         ratio=1e4, meta={"name": f"scale{n}", "seed": seed})


def random_rectangles(n, n_frac, rng):
    """Seeded axis-aligned rectangles snapped to lattice lines: normal axis
    uniform in {x, y, z}, interior node plane uniform, side lengths U(0.1, 0.6),
    placed uniformly so that the rectangle fits in the unit square."""
    out = []
    for _ in range(n_frac):
        axis = int(rng.integers(0, 3))
        plane = int(rng.integers(1, n))
        la = max(1, int(round(rng.uniform(0.1, 0.6) * n)))
        lb = max(1, int(round(rng.uniform(0.1, 0.6) * n)))
        a0 = int(rng.integers(0, n - la + 1))
        b0 = int(rng.integers(0, n - lb + 1))
        out.append((axis, plane, a0, a0 + la, b0, b0 + lb))
    return out


def random_dfn_problem(n, n_frac, ratio, seed, jitter=0.2) -> Problem:
    rng = np.random.default_rng(seed)
    fr = random_rectangles(n, n_frac, rng)
    sub = int(rng.integers(0, 2**31 - 1))
    return build_problem((n, n, n), fr, jitter=jitter, seed=sub, lam_m="lognormal",
                         ratio=ratio, meta={"name": f"dfn{n}_{n_frac}", "seed": seed,
                                            "ratio": ratio})


def config_mixed128(n=128, ratio=1e4, seed=4321) -> Problem:
    """128^3 jittered mesh with a DFN of 50 seeded axis-aligned rectangles."""
    return random_dfn_problem(n, 50, ratio, seed)


def batch_params(count, seed=99, n_lo=16, n_hi=48):
    """(n, number of rectangles, ratio, seed) of each realisation of a batch."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        nf = int(rng.integers(1, 21))
        ratio = float(10.0 ** rng.uniform(2.0, 6.0))
        s = int(rng.integers(0, 2**31 - 1))
        out.append((n, nf, ratio, s))
    return out


def batch_problems(count, seed=99, n_lo=16, n_hi=48):
    """Independent realisations: n ~ U{n_lo..n_hi}, 1-20 rectangles,
    fracture/matrix ratio log-uniform in [1e2, 1e6], lognormal matrix K."""
    return [random_dfn_problem(*p) for p in batch_params(count, seed, n_lo, n_hi)]


# ----------------------------------------------------------------------------
# meshes of the two analytical test cases (Sec. 5.1 and 5.2), extruded in z
# ----------------------------------------------------------------------------

def _line_intersections(xa0, xa1, yb0, yb1):
    """Nodes of a topologically Cartesian grid whose i-lines run from
    (xa0[i], 0) to (xa1[i], 1) and whose j-lines run from (0, yb0[j]) to
    (1, yb1[j]).  Returns X, Y of shape [nj, ni]."""
    XA0 = xa0[None, :]; XA1 = xa1[None, :]
    YB0 = yb0[:, None]; YB1 = yb1[:, None]
    # point on i-line: x = XA0 + s (XA1 - XA0), y = s
    # point on j-line: y = YB0 + x (YB1 - YB0)
    # s = YB0 + (XA0 + s dX) dY  ->  s (1 - dX dY) = YB0 + XA0 dY
    dX = XA1 - XA0; dY = YB1 - YB0
    s = (YB0 + XA0 * dY) / (1.0 - dX * dY)
    return XA0 + s * dX, s


def _extrude(X, Y, dz):
    nj, ni = X.shape
    xyz = np.zeros((2, nj, ni, 3))
    xyz[:, :, :, 0] = X[None]
    xyz[:, :, :, 1] = Y[None]
    xyz[1, :, :, 2] = dz
    return xyz.reshape(-1, 3)


def one_fracture_problem(nx, tan_theta=0.5, lam_f=20.0, d_f=0.01):
    """Sec. 5.1: unit square, fracture from (0, 1/4) to (1, 1/4 + tan(theta)),
    Lambda_m = 1, phi_m = phi_f = 1, p = 1 - x on x = 0 and x = 1, y walls and
    z walls no-flow; c = 1 enters on the whole x = 0 side.  The grid's j-lines
    follow the fracture (it lies on the j = nx/2 line), the i-lines are
    x = i / nx, one cell layer of thickness 1/nx in z."""
    ny = nx
    jf = nx // 2
    xa = np.arange(nx + 1) / nx
    yl = 0.25; yr = 0.25 + tan_theta
    jj = np.arange(ny + 1)
    yb0 = np.where(jj <= jf, yl * jj / jf, yl + (1 - yl) * (jj - jf) / (ny - jf))
    yb1 = np.where(jj <= jf, yr * jj / jf, yr + (1 - yr) * (jj - jf) / (ny - jf))
    X, Y = _line_intersections(xa, xa, yb0, yb1)
    dims = (nx, ny, 1)
    xyz = _extrude(X, Y, 1.0 / nx)
    ff = axis_fracture_faces(dims, 1, jf, 0, nx, 0, 1)
    nnodes = xyz.shape[0]
    i = np.arange(nnodes) % (nx + 1)
    left = np.nonzero(i == 0)[0]; right = np.nonzero(i == nx)[0]
    dn = np.sort(np.concatenate([left, right]))
    dv = 1.0 - xyz[dn, 0]
    cb = np.where(np.isin(dn, left), 1.0, 0.0)
    return build_problem(dims, [ff], xyz=xyz, frac_lambda=[lam_f], frac_df=[d_f],
                         phi_m=1.0, phi_f=1.0, dirichlet=(dn, dv, cb),
                         meta={"name": f"onefrac{nx}", "tan_theta": tan_theta,
                               "lam_f": lam_f, "d_f": d_f, "jf": jf})


def four_fracture_problem(nx, tan1=5.0 / 8.0, tan2=0.25, lam_f1=200.0, lam_f3=400.0, d_f=0.01):
    """Sec. 5.2: fractures along the line (0, 1/4)-(1, 1/4 + tan1) (Gamma_1,
    Gamma_2) and the line (3/4, 0)-(3/4 - tan2, 1) (Gamma_3, Gamma_4), crossing
    at x_0.  Grid lines follow both fracture lines; p = 1 - x on x = 0, x = 1
    and at the two fracture tips on y = 0 and y = 1; other walls no-flow.
    Dirichlet concentration 1 at the tip of Gamma_1 on x = 0 and at the tip of
    Gamma_4 on y = 1, zero on every other Dirichlet node."""
    ny = nx
    jf = int(round(0.5625 * ny))
    i_f = int(round(0.625 * nx))
    ii = np.arange(nx + 1)
    xb, xt = 0.75, 0.75 - tan2
    xa0 = np.where(ii <= i_f, xb * ii / i_f, xb + (1 - xb) * (ii - i_f) / (nx - i_f))
    xa1 = np.where(ii <= i_f, xt * ii / i_f, xt + (1 - xt) * (ii - i_f) / (nx - i_f))
    jj = np.arange(ny + 1)
    yl, yr = 0.25, 0.25 + tan1
    yb0 = np.where(jj <= jf, yl * jj / jf, yl + (1 - yl) * (jj - jf) / (ny - jf))
    yb1 = np.where(jj <= jf, yr * jj / jf, yr + (1 - yr) * (jj - jf) / (ny - jf))
    X, Y = _line_intersections(xa0, xa1, yb0, yb1)
    dims = (nx, ny, 1)
    xyz = _extrude(X, Y, 1.0 / nx)
    f1 = axis_fracture_faces(dims, 1, jf, 0, i_f, 0, 1)
    f2 = axis_fracture_faces(dims, 1, jf, i_f, nx, 0, 1)
    f3 = axis_fracture_faces(dims, 0, i_f, 0, jf, 0, 1)
    f4 = axis_fracture_faces(dims, 0, i_f, jf, ny, 0, 1)
    nnodes = xyz.shape[0]
    i = np.arange(nnodes) % (nx + 1)
    j = (np.arange(nnodes) // (nx + 1)) % (ny + 1)
    left = np.nonzero(i == 0)[0]; right = np.nonzero(i == nx)[0]
    tip_bot = np.nonzero((i == i_f) & (j == 0))[0]
    tip_top = np.nonzero((i == i_f) & (j == ny))[0]
    dn = np.unique(np.concatenate([left, right, tip_bot, tip_top]))
    dv = 1.0 - xyz[dn, 0]
    tip1 = left[(j[left] == jf)]
    cb = np.where(np.isin(dn, tip1) | np.isin(dn, tip_top), 1.0, 0.0)
    return build_problem(dims, [f1, f2, f3, f4], xyz=xyz,
                         frac_lambda=[lam_f1, lam_f1, lam_f3, lam_f3],
                         frac_df=[d_f] * 4, phi_m=1.0, phi_f=1.0,
                         dirichlet=(dn, dv, cb),
                         meta={"name": f"fourfrac{nx}", "tan1": tan1, "tan2": tan2,
                               "lam_f1": lam_f1, "lam_f3": lam_f3, "d_f": d_f,
                               "jf": jf, "if": i_f})


# ----------------------------------------------------------------------------
# tetrahedral meshes (Sec. 3.1 admits any polyhedral cells)
# ----------------------------------------------------------------------------

def tet_problem(dims, fractures: Sequence[Tuple] = (), *, jitter=0.0, seed=0, lam_m="identity", ratio=1e4,
                d_f=1e-2, phi_m=0.2, phi_f=0.4, meta=None) -> Problem:
    """A conforming tetrahedral mesh of the unit box: every cell of an
    nx*ny*nz hexahedral lattice cut into the six tetrahedra around its
    diagonal from lattice offset (0,0,0) to (1,1,1) (one per order of the
    three axes), so neighbouring cells cut their shared square the same way.
    ``faces`` are the unique triangles [n_faces, 3], ``cell_faces``
    [n_cells, 4], ``cell_nodes`` [n_cells, 4].  ``fractures``: axis-aligned
    rectangles (axis, plane, lo_a, hi_a, lo_b, hi_b) on lattice node planes,
    as for the hexahedral lattice; their fracture faces are the triangles
    lying in them.  Interior nodes are jittered by U(-jitter h, jitter h) per
    coordinate with fracture-normal coordinates frozen; p = 1 - x on x = 0 and
    x = 1 (inflow c = 1 on x = 0), no-flow elsewhere."""
    import itertools
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    hex_nodes, _, _, _, _ = hex_lattice(dims)
    tets = []
    for perm in itertools.permutations((1, 2, 4)):
        loc = [0, perm[0], perm[0] | perm[1], 7]
        tets.append(hex_nodes[:, loc])
    cell_nodes = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)   # the 6 tets of a hex stay together
    n_cells = cell_nodes.shape[0]
    tri = np.concatenate([cell_nodes[:, [1, 2, 3]], cell_nodes[:, [0, 2, 3]], cell_nodes[:, [0, 1, 3]],
                          cell_nodes[:, [0, 1, 2]]])
    key = np.sort(tri, axis=1).astype(np.int64)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    if nn < (1 << 21):   # one int64 per triangle: the same order as the rows, much faster
        code = (key[:, 0] << 42) | (key[:, 1] << 21) | key[:, 2]
        ucode, inv = np.unique(code, return_inverse=True)
        faces = np.stack([ucode >> 42, (ucode >> 21) & ((1 << 21) - 1), ucode & ((1 << 21) - 1)], axis=1)
    else:
        faces, inv = np.unique(key, axis=0, return_inverse=True)
    faces = faces.astype(np.int32)
    cell_faces = inv.reshape(4, n_cells).T.astype(np.int32)
    # lattice index of every node
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    ids, owner = [], []
    frozen = np.zeros((ijk.shape[0], 3), bool)
    # the triangles lying on a lattice plane of each axis, with their nodes' lattice indices
    on_plane = {}
    if len(fractures):
        fi = ijk[faces]                                          # [n_faces, 3 nodes, 3 axes]
        for ax in range(3):
            sel = np.nonzero((fi[:, 0, ax] == fi[:, 1, ax]) & (fi[:, 0, ax] == fi[:, 2, ax]))[0]
            on_plane[ax] = (sel, fi[sel])
    for f_idx, (axis, plane, lo_a, hi_a, lo_b, hi_b) in enumerate(fractures):
        oa, ob = [a for a in range(3) if a != axis]
        sel, fs = on_plane[axis]
        on = fs[:, 0, axis] == plane
        ina = np.all((fs[:, :, oa] >= lo_a) & (fs[:, :, oa] <= hi_a), axis=1)
        inb = np.all((fs[:, :, ob] >= lo_b) & (fs[:, :, ob] <= hi_b), axis=1)
        fid = sel[np.nonzero(on & ina & inb)[0]]
        ids.append(fid)
        owner.append(np.full(fid.shape, f_idx))
        frozen[np.unique(faces[fid].ravel()), axis] = True
    if ids:
        allid = np.concatenate(ids)
        allown = np.concatenate(owner)
        ff_faces, first = np.unique(allid, return_index=True)
        ff_frac = allown[first].astype(np.int32)
    else:
        ff_faces = np.zeros(0, np.int64)
        ff_frac = np.zeros(0, np.int32)
    ff_faces = ff_faces.astype(np.int32)
    xyz = _lattice_xyz(dims)
    if jitter > 0:
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        d = rng.uniform(-jitter, jitter, size=xyz.shape) * h[None, :]
        boundary = ((ijk[:, 0] == 0) | (ijk[:, 0] == nx) | (ijk[:, 1] == 0) | (ijk[:, 1] == ny) |
                    (ijk[:, 2] == 0) | (ijk[:, 2] == nz))
        d[boundary] = 0.0
        d[frozen] = 0.0
        xyz = xyz + d
    if isinstance(lam_m, np.ndarray):
        lam = lam_m
    elif lam_m == "identity":
        lam = np.zeros((n_cells, 6)); lam[:, :3] = 1.0
    elif lam_m == "lognormal":
        lam = _lognormal_aniso(n_cells, rng)
    else:
        raise ValueError(lam_m)
    nff = ff_faces.shape[0]
    left = np.nonzero(ijk[:, 0] == 0)[0]
    right = np.nonzero(ijk[:, 0] == nx)[0]
    dir_nodes = np.sort(np.concatenate([left, right])).astype(np.int32)
    dir_values = 1.0 - xyz[dir_nodes, 0]
    cbar = np.where(np.isin(dir_nodes, left), 1.0, 0.0)
    return Problem(
        dims=tuple(dims), xyz=np.ascontiguousarray(xyz, np.float64), cell_nodes=cell_nodes, faces=faces,
        cell_faces=cell_faces, ff_faces=ff_faces, ff_nodes=np.ascontiguousarray(faces[ff_faces]).astype(np.int32),
        ff_frac=ff_frac, lambda_m=np.ascontiguousarray(lam, np.float64), lambda_f=np.full(nff, float(ratio)),
        d_f=np.full(nff, float(d_f)), mu=1.0, dir_nodes=dir_nodes, dir_values=np.asarray(dir_values, np.float64),
        phi_m=np.full(n_cells, float(phi_m)), phi_f=np.full(nff, float(phi_f)), cbar=np.asarray(cbar, np.float64),
        meta=dict(meta or {}, name=f"tet{nx}x{ny}x{nz}", seed=seed))


# ----------------------------------------------------------------------------
# extruded triangular meshes: prisms (the mesh type of Sec. 5.5), optionally
# mixed with hexahedral columns
# ----------------------------------------------------------------------------

# local faces, cyclic (the library's tables list the same faces)
_PRISM_FACES = [(0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)]
_HEX_FACES = [(0, 2, 6, 4), (1, 3, 7, 5), (0, 1, 5, 4), (2, 3, 7, 6), (0, 1, 3, 2), (4, 5, 7, 6)]


def _faces_of_cells(cell_nodes, kinds, tables):
    """Unique faces (padded [n_faces, 4], -1 after the nodes, each in the
    cyclic order of its first cell) and the padded cell -> face table
    [n_cells, 6] of cells given as -1-padded node rows; cell K uses the
    local faces tables[kinds[K]]."""
    cells_l, slot_l, rows_l = [], [], []
    for k, table in enumerate(tables):
        C = np.nonzero(kinds == k)[0]
        for f, lf in enumerate(table):
            r = -np.ones((C.size, 4), np.int64)
            r[:, :len(lf)] = cell_nodes[C][:, list(lf)]
            cells_l.append(C); slot_l.append(np.full(C.size, f)); rows_l.append(r)
    cell = np.concatenate(cells_l); slot = np.concatenate(slot_l); rows = np.concatenate(rows_l)
    order = np.lexsort((slot, cell))              # by cell, then local face
    cell, slot, rows = cell[order], slot[order], rows[order]
    key = np.sort(rows, axis=1)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    faces = rows[first].astype(np.int32)
    cell_faces = -np.ones((cell_nodes.shape[0], 6), np.int32)
    cell_faces[cell, slot] = inv.ravel()
    return faces, cell_faces


def prism_problem(nxy, nz, fractures: Sequence[Tuple] = (), *, split="all", jitter=0.0, seed=0,
                  lam_m="identity", ratio=1e4, d_f=1e-2, phi_m=0.2, phi_f=0.4, dirichlet="x",
                  lengths=(1.0, 1.0, 1.0), meta=None) -> Problem:
    """The tensor product of a triangular mesh of the rectangle with a
    uniform vertical mesh of nz layers, as in Sec. 5.5: the nx*ny lattice
    squares are cut into the triangles (00, 10, 11) and (00, 11, 01) and
    each triangle times each layer is a prism (nodes: the bottom triangle,
    then the nodes above it).  ``split``: "all" (prisms only), "half"
    (columns with i < nx/2 are cut, the others stay hexahedra) or "checker"
    (columns with i + j even are cut) for meshes that mix both shapes.
    ``cell_nodes`` is [n_cells, 8] with -1 after a prism's 6 nodes, ``faces``
    [n_faces, 4] with -1 after a triangle's 3 nodes, ``cell_faces``
    [n_cells, 6] with -1 after a prism's 5 faces.

    ``fractures``: vertical rectangles made of lattice faces, each
    ("x", i, j0, j1, k0, k1) on the plane of node column i for squares
    j0 <= j < j1 and layers k0 <= k < k1, ("y", j, i0, i1, k0, k1), or
    ("d", d, i0, i1, k0, k1) on the diagonals (i, i - d) -> (i + 1, i + 1 - d)
    of cut squares i0 <= i < i1.  Interior nodes are jittered by
    U(-jitter h, jitter h) per coordinate with the coordinates normal to a
    fracture plane frozen.  ``dirichlet="x"``: p = 1 - x/Lx on the x = 0 and
    x = Lx node planes (inflow c = 1 at x = 0); None: no Dirichlet nodes
    (wells fix the pressure).  ``lengths``: the box (Lx, Ly, Lz)."""
    rng = np.random.default_rng(seed)
    nx, ny = nxy
    dims = (nx, ny, nz)
    cut = np.zeros((nx, ny), bool)
    for i in range(nx):
        for j in range(ny):
            cut[i, j] = split == "all" or (split == "half" and i < nx // 2) or (split == "checker" and (i + j) % 2 == 0)
    # columns in (k, j, i) order; a cut column holds two prisms, the others a hexahedron
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kk, jj, ii = kk.ravel(), jj.ravel(), ii.ravel()
    iscut = cut[ii, jj]
    per = np.where(iscut, 2, 1)
    start = np.concatenate([[0], np.cumsum(per)[:-1]])
    n_cells = int(per.sum())
    up = (nx + 1) * (ny + 1)
    n00, n10 = _nid(dims, ii, jj, kk), _nid(dims, ii + 1, jj, kk)
    n01, n11 = _nid(dims, ii, jj + 1, kk), _nid(dims, ii + 1, jj + 1, kk)
    cell_nodes = -np.ones((n_cells, 8), np.int64)
    kinds = np.zeros(n_cells, np.int64)
    c = np.nonzero(iscut)[0]
    for t, tri in enumerate(((n00, n10, n11), (n00, n11, n01))):
        rows = start[c] + t
        bot = np.stack([v[c] for v in tri], axis=1)
        cell_nodes[rows, :6] = np.concatenate([bot, bot + up], axis=1)
        kinds[rows] = 0
    h = np.nonzero(~iscut)[0]
    bot = np.stack([n00[h], n10[h], n01[h], n11[h]], axis=1)
    cell_nodes[start[h]] = np.concatenate([bot, bot + up], axis=1)
    kinds[start[h]] = 1
    faces, cell_faces = _faces_of_cells(cell_nodes, kinds, [_PRISM_FACES, _HEX_FACES])
    cell_nodes = cell_nodes.astype(np.int32)
    k3, j3, i3 = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ijk = np.stack([i3.ravel(), j3.ravel(), k3.ravel()], axis=1)
    # fracture faces: vertical quadrilaterals over listed edges of the 2-D mesh
    up2 = (nx + 1) * (ny + 1)

    def n2(i, j):
        return np.asarray(i, np.int64) + (nx + 1) * np.asarray(j, np.int64)

    fkeys, fown, fz = [], [], []
    for f_idx, spec in enumerate(fractures):
        kind = spec[0]
        if kind == "e":                  # ("e", edges [m, 2] of 2-D node ids, k0, k1)
            _, e2, k0, k1 = spec
            a, b = np.asarray(e2, np.int64)[:, 0], np.asarray(e2, np.int64)[:, 1]
            frz = (0, 1)
        else:
            _, plane, a0, a1, k0, k1 = spec
            t = np.arange(a0, a1)
            if kind == "x":
                a, b, frz = n2(plane, t), n2(plane, t + 1), (0,)
            elif kind == "y":
                a, b, frz = n2(t, plane), n2(t + 1, plane), (1,)
            elif kind == "d":
                t = t[(t - plane >= 0) & (t + 1 - plane <= ny)]
                a, b, frz = n2(t, t - plane), n2(t + 1, t + 1 - plane), (0, 1)
            else:
                raise ValueError(kind)
        e = np.minimum(a, b) * up2 + np.maximum(a, b)
        for k in range(k0, k1):
            fkeys.append(e * nz + k)
            fown.append(np.full(e.shape, f_idx))
            fz.append((np.stack([a, b], 1), k, frz))
    quad = faces[:, 3] >= 0
    f64 = np.where(faces >= 0, faces, 0).astype(np.int64)
    f2 = np.sort(f64 % up2, axis=1)                                # 2-D nodes of each face
    fk = f64 // up2                                                # layers of each face
    # a vertical quadrilateral: two 2-D nodes, each twice, on layers k and k + 1
    vertical = (quad & (f2[:, 0] == f2[:, 1]) & (f2[:, 2] == f2[:, 3]) & (f2[:, 1] != f2[:, 2]) &
                (fk.min(axis=1) + 1 == fk.max(axis=1)))
    lo2, hi2 = f2[:, 0], f2[:, 2]
    face_key = np.where(vertical, (lo2 * up2 + hi2) * nz + fk.min(axis=1), -1)
    frozen = np.zeros((ijk.shape[0], 3), bool)
    if fkeys:
        K_ = np.concatenate(fkeys)
        O_ = np.concatenate(fown)
        order = np.lexsort((O_, K_))
        K_, O_ = K_[order], O_[order]
        keep = np.ones(K_.size, bool)
        keep[1:] = K_[1:] != K_[:-1]
        K_, O_ = K_[keep], O_[keep]                                # each face once, its first fracture
        pos = np.searchsorted(K_, face_key)
        pos = np.minimum(pos, K_.size - 1)
        hit = vertical & (K_[pos] == face_key)
        ff_faces = np.nonzero(hit)[0]
        ff_frac = O_[pos[ff_faces]].astype(np.int32)
        for (e2, k, frz) in fz:
            nodes = np.concatenate([e2.ravel() + k * up2, e2.ravel() + (k + 1) * up2])
            for ax in frz:
                frozen[nodes, ax] = True
        # freeze only nodes of faces that exist as fracture faces
        used = np.zeros(ijk.shape[0], bool)
        used[faces[ff_faces].ravel()] = True
        frozen &= used[:, None]
    else:
        ff_faces = np.zeros(0, np.int64)
        ff_frac = np.zeros(0, np.int32)
    ff_faces = ff_faces.astype(np.int32)
    L = np.asarray(lengths, np.float64)
    xyz = _lattice_xyz(dims) * L[None, :]
    if jitter > 0:
        h = L / np.array([nx, ny, nz])
        d = rng.uniform(-jitter, jitter, size=xyz.shape) * h[None, :]
        boundary = ((ijk[:, 0] == 0) | (ijk[:, 0] == nx) | (ijk[:, 1] == 0) | (ijk[:, 1] == ny) |
                    (ijk[:, 2] == 0) | (ijk[:, 2] == nz))
        d[boundary] = 0.0
        d[frozen] = 0.0
        xyz = xyz + d
    if isinstance(lam_m, np.ndarray):
        lam = lam_m
    elif lam_m == "identity":
        lam = np.zeros((n_cells, 6)); lam[:, :3] = 1.0
    elif lam_m == "lognormal":
        lam = _lognormal_aniso(n_cells, rng)
    else:
        raise ValueError(lam_m)
    nff = ff_faces.shape[0]
    if dirichlet == "x":
        left = np.nonzero(ijk[:, 0] == 0)[0]
        right = np.nonzero(ijk[:, 0] == nx)[0]
        dir_nodes = np.sort(np.concatenate([left, right])).astype(np.int32)
        dir_values = 1.0 - xyz[dir_nodes, 0] / L[0]
        cbar = np.where(np.isin(dir_nodes, left), 1.0, 0.0)
    elif dirichlet is None:
        dir_nodes = np.zeros(0, np.int32); dir_values = np.zeros(0); cbar = np.zeros(0)
    else:
        raise ValueError(dirichlet)
    return Problem(
        dims=tuple(dims), xyz=np.ascontiguousarray(xyz, np.float64), cell_nodes=cell_nodes, faces=faces,
        cell_faces=cell_faces, ff_faces=ff_faces, ff_nodes=np.ascontiguousarray(faces[ff_faces]).astype(np.int32),
        ff_frac=ff_frac, lambda_m=np.ascontiguousarray(lam, np.float64), lambda_f=np.full(nff, float(ratio)),
        d_f=np.full(nff, float(d_f)), mu=1.0, dir_nodes=dir_nodes, dir_values=np.asarray(dir_values, np.float64),
        phi_m=np.full(n_cells, float(phi_m)), phi_f=np.full(nff, float(phi_f)), cbar=np.asarray(cbar, np.float64),
        meta=dict(meta or {}, name=f"prism{nx}x{ny}x{nz}_{split}", seed=seed))


def pyramid_problem(dims, fractures: Sequence[Tuple] = (), *, jitter=0.0, seed=0, lam_m="identity", ratio=1e4,
                    d_f=1e-2, phi_m=0.2, phi_f=0.4, meta=None) -> Problem:
    """Every cell of an nx*ny*nz hexahedral lattice cut into six pyramids,
    one on each of its faces, with a common apex at an added node in the
    middle of the cell (node ids after the lattice nodes).  Neighbouring
    cells share the square between them as the base of two pyramids, so the
    mesh is conforming.  ``fractures`` as for ``build_problem`` (their faces
    are lattice squares, i.e. pyramid bases).  Lattice nodes are jittered as
    in ``build_problem``; the apexes sit at the mean of their cell's eight
    corners plus U(-jitter h/4, jitter h/4).  p = 1 - x on x = 0 and x = 1
    (inflow c = 1 at x = 0), no-flow elsewhere."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    hex_nodes, hfaces, hcell_faces, face_axis, _ = hex_lattice(dims)
    nlat = (nx + 1) * (ny + 1) * (nz + 1)
    ids, owner = [], []
    for f_idx, fr in enumerate(fractures):
        fid = axis_fracture_faces(dims, *fr)
        ids.append(fid)
        owner.append(np.full(fid.shape, f_idx))
    if ids:
        allid = np.concatenate(ids)
        allown = np.concatenate(owner)
        ff_lat, first = np.unique(allid, return_index=True)
        ff_frac = allown[first].astype(np.int32)
    else:
        ff_lat = np.zeros(0, np.int64)
        ff_frac = np.zeros(0, np.int32)
    xyz = _lattice_xyz(dims)
    if jitter > 0:
        xyz = _jitter(dims, xyz, hfaces, ff_lat, face_axis, jitter, rng)
    n_hex = hex_nodes.shape[0]
    apex = nlat + np.arange(n_hex)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    xa = xyz[hex_nodes].mean(axis=1)
    if jitter > 0:
        xa = xa + rng.uniform(-jitter / 4, jitter / 4, size=xa.shape) * h[None, :]
    xyz = np.concatenate([xyz, xa])
    # cells: pyramid (base = lattice face in cyclic order, apex) for each hex face
    n_cells = 6 * n_hex
    cell_nodes = -np.ones((n_cells, 8), np.int64)
    cell_nodes[:, :4] = hfaces[hcell_faces].reshape(n_cells, 4)     # six pyramids per cube, in face order
    cell_nodes[:, 4] = np.repeat(apex, 6)
    PYR = [(0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)]
    faces, cell_faces = _faces_of_cells(cell_nodes, np.zeros(n_cells, np.int64), [PYR])
    cell_nodes = cell_nodes.astype(np.int32)
    # fracture faces: the lattice squares among the new faces
    key = {tuple(sorted(f[f >= 0].tolist())): i for i, f in enumerate(faces)}
    ff_faces = np.array([key[tuple(sorted(hfaces[f].tolist()))] for f in ff_lat], np.int64)
    order = np.argsort(ff_faces)
    ff_faces = ff_faces[order].astype(np.int32)
    ff_frac = ff_frac[order]
    if isinstance(lam_m, np.ndarray):
        lam = lam_m
    elif lam_m == "identity":
        lam = np.zeros((n_cells, 6)); lam[:, :3] = 1.0
    elif lam_m == "lognormal":
        lam = _lognormal_aniso(n_cells, rng)
    else:
        raise ValueError(lam_m)
    nff = ff_faces.shape[0]
    k3, j3, i3 = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ii = i3.ravel()
    left = np.nonzero(ii == 0)[0]
    right = np.nonzero(ii == nx)[0]
    dir_nodes = np.sort(np.concatenate([left, right])).astype(np.int32)
    dir_values = 1.0 - xyz[dir_nodes, 0]
    cbar = np.where(np.isin(dir_nodes, left), 1.0, 0.0)
    return Problem(
        dims=tuple(dims), xyz=np.ascontiguousarray(xyz, np.float64), cell_nodes=cell_nodes, faces=faces,
        cell_faces=cell_faces, ff_faces=ff_faces, ff_nodes=np.ascontiguousarray(faces[ff_faces]).astype(np.int32),
        ff_frac=ff_frac, lambda_m=np.ascontiguousarray(lam, np.float64), lambda_f=np.full(nff, float(ratio)),
        d_f=np.full(nff, float(d_f)), mu=1.0, dir_nodes=dir_nodes, dir_values=np.asarray(dir_values, np.float64),
        phi_m=np.full(n_cells, float(phi_m)), phi_f=np.full(nff, float(phi_f)), cbar=np.asarray(cbar, np.float64),
        meta=dict(meta or {}, name=f"pyramid{nx}x{ny}x{nz}", seed=seed))


def _place_wells(pb, nxy, nz, specs, k0, k1, lam_f, d_f, r_w, q_inj):
    """Wells at fracture edges of an extruded mesh: specs lists (kind, 2-D
    node a, 2-D node b) with a -> b an edge of the triangular mesh carrying
    a fracture; each well perforates that edge's fracture faces in layers
    k0 <= k < k1.  Fills meta["well_geometry"] and meta["wells"]."""
    nx, ny = nxy
    up2 = (nx + 1) * (ny + 1)
    fn = np.sort(pb.ff_nodes.astype(np.int64), axis=1)         # vertical quads: [a, b, a', b'] sorted
    f2 = np.sort(fn % up2, axis=1)
    fkey = (f2[:, 0] * up2 + f2[:, 2]) * nz + (fn // up2).min(axis=1)
    order = np.argsort(fkey)
    ff, well, dx, dz = [], [], [], []
    wells = []
    for w, (kind, a, b) in enumerate(specs):
        e = min(a, b) * up2 + max(a, b)
        want = e * nz + np.arange(k0, k1)
        pos = np.searchsorted(fkey[order], want)
        pos = np.minimum(pos, fkey.size - 1)
        hit = fkey[order][pos] == want
        perf = order[pos[hit]]
        if not perf.size:
            raise ValueError(f"well {w}: no fracture face on its edge")
        for i in perf:
            p = pb.xyz[pb.ff_nodes[i]]
            bot = np.argsort(p[:, 2])[:2]
            dx.append(float(np.linalg.norm(p[bot[0], :2] - p[bot[1], :2])))
            dz.append(float(p[:, 2].max() - p[:, 2].min()))
            ff.append(int(i))
            well.append(w)
        wells.append(dict(kind=kind, pw=0.0, rate=q_inj if kind == "injector" else 0.0,
                          cin=1.0 if kind == "injector" else 0.0))
    pb.meta["well_geometry"] = dict(ff=np.array(ff, np.int32), well=np.array(well, np.int32), dx=np.array(dx),
                                    dz=np.array(dz), d_f=np.full(len(ff), float(d_f)),
                                    lam_f=np.full(len(ff), float(lam_f)), r_w=np.full(len(ff), float(r_w)))
    pb.meta["wells"] = wells


def well_problem(nxy=(12, 8), nz=6, *, split="all", lengths=(600.0, 400.0, 60.0), jitter=0.15, seed=0,
                 lam_m=1e-15, lam_f=1e-11, d_f=1.0, phi=0.1, mu=1e-3, r_w=0.1, q_inj=0.16, dirichlet=None,
                 meta=None) -> Problem:
    """A prism mesh with vertical fractures and vertical wells in the manner
    of Sec. 5.5: isotropic Lambda_m and Lambda_f, aperture d_f, porosity phi
    in both media, viscosity mu, no Dirichlet node (the producers fix the
    pressure level).  Three fractures: the planes of node column i = nx/3
    and of node row j = ny/2 (partly) and a diagonal.  Each well is vertical
    at the middle of one fracture edge of the triangular mesh and perforates
    the fracture faces of that edge in the central half of the layers: the
    injector (total rate q_inj, concentration 1, split evenly over its
    perforations) on the first fracture, two producers (p_w = 0) on the
    others.  ``meta["well_geometry"]`` gives per perforation the face, its
    well, dx (the face's horizontal edge), dz (its height), d_f, Lambda_f and
    r_w, and ``meta["wells"]`` the wells; ``well_arrays`` turns them into the
    per-perforation arrays once the well indices are known."""
    nx, ny = nxy
    i_f, j_f = nx // 3, ny // 2
    fr = [("x", i_f, 0, ny, 0, nz), ("y", j_f, i_f, nx, 0, nz), ("d", 0, 0, min(nx, ny) // 2, 0, nz)]
    pb = prism_problem(nxy, nz, fr, split=split, jitter=jitter, seed=seed, ratio=lam_f, d_f=d_f, phi_m=phi,
                       phi_f=phi, dirichlet=dirichlet, lengths=lengths, meta=meta)
    lam = np.zeros((pb.n_cells, 6)); lam[:, :3] = lam_m
    pb.lambda_m = lam
    pb.mu = float(mu)

    def n2(i, j):
        return i + (nx + 1) * j
    specs = [("injector", n2(i_f, ny // 4), n2(i_f, ny // 4 + 1)),
             ("producer", n2(nx - 2, j_f), n2(nx - 1, j_f)),
             ("producer", n2(1, 1), n2(2, 2))]
    _place_wells(pb, nxy, nz, specs, nz // 4, nz - nz // 4, lam_f, d_f, r_w, q_inj)
    pb.meta["name"] = f"wells{nx}x{ny}x{nz}_{split}"
    return pb


def config_prism55(nxy=(695, 372), nz=24, n_frac=600, seed=5505, jitter=0.15) -> Problem:
    """The complex fracture network of Sec. 5.5 at its size, synthetic: the
    domain 5888.75 x 3157.5 x 250 m, the tensor product of a triangular mesh
    (nxy squares cut in two: 517 080 triangles) with 24 uniform layers
    (12.4 M prisms, 6.5 M nodes); n_frac vertical fractures through the whole
    height, each a run of U{10..60} consecutive mesh edges along a lattice
    line or a cut diagonal (about 21 000 edges, 5.1e5 fracture faces);
    Lambda_f = 1e-11, Lambda_m = 1e-15 m^2, phi = 0.1, d_f = 1 m, mu = 1e-3;
    one injector (5e6 m^3 a year, c = 1) and two producers (p_w = 0), each at
    the middle of a fracture edge nearest to (0.2, 0.5), (0.8, 0.25) and
    (0.8, 0.75) of the plan, perforating the 12 central layers; no Dirichlet
    node."""
    rng = np.random.default_rng(seed)
    nx, ny = nxy
    L = (5888.75, 3157.5, 250.0)

    def n2(i, j):
        return np.asarray(i, np.int64) + (nx + 1) * np.asarray(j, np.int64)
    edges = []
    for _ in range(n_frac):
        kind = int(rng.integers(0, 3))
        m = int(rng.integers(10, 61))
        i0 = int(rng.integers(0, nx - m)) if kind != 1 else int(rng.integers(0, nx))
        j0 = int(rng.integers(0, ny - m)) if kind != 0 else int(rng.integers(0, ny))
        t = np.arange(m)
        if kind == 0:        # along x
            a, b = n2(i0 + t, j0), n2(i0 + t + 1, j0)
        elif kind == 1:      # along y
            a, b = n2(i0, j0 + t), n2(i0, j0 + t + 1)
        else:                # along the cut diagonal
            a, b = n2(i0 + t, j0 + t), n2(i0 + t + 1, j0 + t + 1)
        edges.append(("e", np.stack([a, b], 1), 0, nz))
    pb = prism_problem(nxy, nz, edges, split="all", jitter=jitter, seed=seed + 1, ratio=1e-11, d_f=1.0,
                       phi_m=0.1, phi_f=0.1, dirichlet=None, lengths=L)
    lam = np.zeros((pb.n_cells, 6)); lam[:, :3] = 1e-15
    pb.lambda_m = lam
    pb.mu = 1e-3
    # well edges: the fracture edge (bottom layer) whose midpoint is nearest each target
    up2 = (nx + 1) * (ny + 1)
    fn = pb.ff_nodes.astype(np.int64)
    bottom = fn[(fn // up2).max(axis=1) == 1]
    e2 = np.sort(np.sort(bottom % up2, axis=1)[:, [0, 2]], axis=1)
    xy = np.stack([(e2 % (nx + 1)) / nx * L[0], (e2 // (nx + 1)) / ny * L[1]], axis=-1).mean(axis=1)
    specs = []
    for kind, (tx, ty) in (("injector", (0.2, 0.5)), ("producer", (0.8, 0.25)), ("producer", (0.8, 0.75))):
        i = int(np.argmin(np.hypot(xy[:, 0] - tx * L[0], xy[:, 1] - ty * L[1])))
        specs.append((kind, int(e2[i, 0]), int(e2[i, 1])))
    _place_wells(pb, nxy, nz, specs, 6, 18, 1e-11, 1.0, 0.1, 5.0e6 / (365.0 * 86400.0))
    pb.meta["name"] = f"prism55_{nx}x{ny}x{nz}"
    pb.meta["seed"] = seed
    return pb


def config_tet54(n=100, n_frac=30, seed=5404) -> Problem:
    """The tetrahedral test case of Sec. 5.4 at its size, synthetic: n^3
    lattice cubes cut into six tetrahedra each (6.0 M cells, 1.03 M nodes at
    n = 100) with a DFN of n_frac seeded lattice rectangles (about 7e4
    fracture triangles); the physics of Sec. 5.3: Lambda_m = 1, Lambda_f = 20,
    phi_m = phi_f = 1, mu = 1, d_f = 1e-2."""
    rng = np.random.default_rng(seed)
    fr = random_rectangles(n, n_frac, rng)
    sub = int(rng.integers(0, 2**31 - 1))
    return tet_problem((n, n, n), fr, jitter=0.2, seed=sub, lam_m="identity", ratio=20.0, d_f=1e-2,
                       phi_m=1.0, phi_f=1.0, meta={"name": f"tet54_{n}", "seed": seed})


def well_arrays(pb, wi):
    """Per-perforation arrays (ff, wi, pw, q, cin) of ``pb.meta["wells"]``
    given the Peaceman well index of every perforation: a producer keeps
    its WI and p_w; an injector has WI = 0 and its rate split evenly over
    its perforations."""
    g = pb.meta["well_geometry"]
    wells = pb.meta["wells"]
    n = g["ff"].size
    out = dict(ff=g["ff"].copy(), wi=np.zeros(n), pw=np.zeros(n), q=np.zeros(n), cin=np.zeros(n))
    for w, spec in enumerate(wells):
        sel = g["well"] == w
        if spec["kind"] == "producer":
            out["wi"][sel] = np.asarray(wi)[sel]
            out["pw"][sel] = spec["pw"]
        else:
            out["q"][sel] = spec["rate"] / sel.sum()
            out["cin"][sel] = spec["cin"]
    return out
