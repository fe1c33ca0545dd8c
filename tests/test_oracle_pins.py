"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an exactness property of the scheme, an invariant of the
discrete equations or a brute-force computation.  CPU only.
"""
import os

import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


# --------------------------------------------------------------------------
# element matrices
# --------------------------------------------------------------------------

def test_p1_reference_tet_golden():
    v = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], float)
    S, vol = vo.tet_p1_stiffness(v, np.eye(3)[None])
    assert vol[0] == pytest.approx(1 / 6)
    np.testing.assert_allclose(6 * S[0], _golden("p1_reference_tet.txt"), atol=1e-14)


def test_p1_reference_triangle_golden():
    v = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]]], float)
    S, area = vo.tri_p1_stiffness(v, np.array([1.0]))
    assert area[0] == pytest.approx(0.5)
    np.testing.assert_allclose(2 * S[0], _golden("p1_reference_triangle.txt"), atol=1e-14)


def test_tet_energy_of_affine_field():
    """u^T S u = |T| g^T Lam g for u = g.x at the vertices, S 1 = 0."""
    rng = np.random.default_rng(0)
    v = rng.normal(size=(50, 4, 3))
    A = rng.normal(size=(50, 3, 3))
    lam = np.einsum("bij,bkj->bik", A, A) + 0.1 * np.eye(3)
    S, vol = vo.tet_p1_stiffness(v, lam)
    g = rng.normal(size=(50, 3))
    u = np.einsum("bia,ba->bi", v, g)
    e = np.einsum("bi,bij,bj->b", u, S, u)
    np.testing.assert_allclose(e, vol * np.einsum("ba,bac,bc->b", g, lam, g), rtol=1e-10)
    assert np.abs(S.sum(axis=2)).max() < 1e-10 * np.abs(S).max()


def test_tri_energy_of_affine_field():
    rng = np.random.default_rng(1)
    v = rng.normal(size=(40, 3, 3))
    coef = rng.uniform(0.5, 2.0, size=40)
    S, area = vo.tri_p1_stiffness(v, coef)
    g = rng.normal(size=(40, 3))
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    gt = g - np.sum(g * n, axis=1, keepdims=True) * n          # tangential part
    u = np.einsum("bia,ba->bi", v, g)
    e = np.einsum("bi,bij,bj->b", u, S, u)
    np.testing.assert_allclose(e, coef * area * np.sum(gt * gt, axis=1), rtol=1e-10)
    # area against Heron-free cross-product formula
    np.testing.assert_allclose(area, 0.5 * np.linalg.norm(
        np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1), rtol=1e-12)


# --------------------------------------------------------------------------
# single-cell fluxes: closed forms on the unit cube
# --------------------------------------------------------------------------

def _unit_cube(frac=False, lam6=None, mu=1.0, df=1.0, lamf=1.0):
    fr = [(0, 1, 0, 1, 0, 1)] if frac else []
    pb = vi.build_problem((1, 1, 1), fr, frac_lambda=[lamf] if frac else None,
                          frac_df=[df] if frac else None)
    if lam6 is not None:
        pb.lambda_m[:] = lam6
    pb.mu = mu
    return pb


FACE_NORMALS = {0: np.array([-1.0, 0, 0]), 1: np.array([1.0, 0, 0]), 2: np.array([0, -1.0, 0]),
                3: np.array([0, 1.0, 0]), 4: np.array([0, 0, -1.0]), 5: np.array([0, 0, 1.0])}


@pytest.mark.parametrize("frac", [False, True])
def test_unit_cube_cell_fluxes_closed_form(frac):
    """Affine u = g.x on the unit cube with constant Lambda: by the divergence
    theorem F_{K,s} = -sum_{faces f containing s} (Lambda g / mu . n_f) int_f eta_s,
    with int_f eta_s = 1/4 on a face whose centre is interpolated (I_sigma) and
    1/6 on a fracture face; F_{K,sigma} = -(Lambda g / mu . n_sigma) / 3."""
    lam6 = np.array([2.0, 1.5, 0.7, 0.3, -0.2, 0.1])
    mu = 1.7
    pb = _unit_cube(frac, lam6, mu)
    m = vo.Mesh(pb)
    cm = vo.cell_local_matrices(pb, m)
    g = np.array([0.7, -1.3, 0.4])
    n = pb.n_nodes + pb.n_ff + pb.n_cells
    u = np.zeros(n)
    u[:pb.n_nodes] = pb.xyz @ g
    u[pb.n_nodes:pb.n_nodes + pb.n_ff] = m.xS[pb.ff_faces] @ g
    u[pb.n_nodes + pb.n_ff:] = m.xK @ g
    F = vo.cell_fluxes(cm, u)[0]
    flux = vo.sym6_to_3x3(lam6) @ g / mu
    dofs = cm["dofs"][0, 1:]
    for slot, d in enumerate(dofs):
        if d < 0:
            continue
        if d < pb.n_nodes:
            expect = 0.0
            for f in range(6):
                fid = pb.cell_faces[0, f]
                if d in pb.faces[fid]:
                    w = (1 / 6) if (frac and fid == pb.ff_faces[0]) else 0.25
                    expect -= flux @ FACE_NORMALS[f] * w
        else:
            expect = -(flux @ FACE_NORMALS[1]) / 3.0
        assert F[slot] == pytest.approx(expect, abs=1e-13)


def test_unit_square_fracture_fluxes_closed_form():
    """F_{sigma,s} = -(d_f Lambda_f / mu) sum_{edges e containing s}
    (grad_tau u . n_e) |e| / 2 for affine u on a unit-square fracture face."""
    pb = _unit_cube(True, mu=0.5, df=0.02, lamf=30.0)
    m = vo.Mesh(pb)
    fm = vo.fracture_local_matrices(pb, m)
    g = np.array([0.9, -0.6, 1.1])
    n = pb.n_nodes + pb.n_ff + pb.n_cells
    u = np.zeros(n)
    u[:pb.n_nodes] = pb.xyz @ g
    u[pb.n_nodes] = m.xS[pb.ff_faces[0]] @ g
    F = vo.fracture_fluxes(fm, u)[0]
    coef = 0.02 * 30.0 / 0.5
    # face on x = 1: tangential coordinates (y, z); edge normals in that plane
    for t, s in enumerate(pb.ff_nodes[0]):
        y, z = pb.xyz[s, 1], pb.xyz[s, 2]
        ny = np.array([0, -1.0, 0]) if y == 0 else np.array([0, 1.0, 0])
        nz = np.array([0, 0, -1.0]) if z == 0 else np.array([0, 0, 1.0])
        expect = -coef * (g @ ny + g @ nz) * 0.5
        assert F[t] == pytest.approx(expect, abs=1e-13)
    assert fm["area"][0] == pytest.approx(1.0)


def test_cell_matrix_rigid_motion_invariance():
    """Rotating the mesh and the tensor together leaves the local matrix."""
    pb = _unit_cube(True, np.array([2.0, 1.5, 0.7, 0.3, -0.2, 0.1]))
    M0 = vo.cell_local_matrices(pb)["M"][0]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    pb.xyz = pb.xyz @ R.T + np.array([3.0, -1.0, 2.0])
    L = R @ vo.sym6_to_3x3(pb.lambda_m[0]) @ R.T
    pb.lambda_m[0] = [L[0, 0], L[1, 1], L[2, 2], L[0, 1], L[0, 2], L[1, 2]]
    M1 = vo.cell_local_matrices(pb)["M"][0]
    np.testing.assert_allclose(M1, M0, atol=1e-13)


# --------------------------------------------------------------------------
# global system
# --------------------------------------------------------------------------

def _scale_small(n=6, seed=3, lam="lognormal"):
    h = n // 2
    fr = [(0, h, 0, n, 0, n), (1, h, 0, n, 0, n), (2, h, 0, n, 0, n), (0, max(1, n // 4), 0, h, 0, n)]
    return vi.build_problem((n, n, n), fr, jitter=0.2, seed=seed, lam_m=lam, ratio=1e4)


def test_global_matrix_symmetric_zero_rowsum():
    pb = _scale_small()
    A = vo.assemble_full(pb)
    scale = abs(A).max()
    assert abs(A - A.T).max() <= 1e-14 * scale
    assert np.abs(np.asarray(A.sum(axis=1))).max() <= 1e-13 * scale


def test_global_matrix_invariant_under_renumbering():
    """Relabelling the nodes and reordering the cells permutes the assembled
    system and nothing else: the scheme depends on the mesh, not on its
    numbering (V_K is kept sorted by node id, so the local slots move)."""
    import dataclasses
    pb = _scale_small(n=4, seed=5)
    A = vo.assemble_full(pb).tocsr()
    rng = np.random.default_rng(11)
    pn = rng.permutation(pb.n_nodes)          # new id of node i
    pc = rng.permutation(pb.n_cells)          # old cell at new position k
    q = dataclasses.replace(pb)
    xyz = np.empty_like(pb.xyz)
    xyz[pn] = pb.xyz
    q.xyz = xyz
    q.faces = pn[pb.faces]
    q.cell_nodes = pn[pb.cell_nodes][pc]
    q.cell_faces = pb.cell_faces[pc]
    q.lambda_m = pb.lambda_m[pc]
    q.phi_m = pb.phi_m[pc]
    q.ff_nodes = pn[pb.ff_nodes]
    q.dir_nodes = pn[pb.dir_nodes]
    B = vo.assemble_full(q).tocsr()
    nv, nf, nc = pb.n_nodes, pb.n_ff, pb.n_cells
    inv_pc = np.empty(nc, np.int64)
    inv_pc[pc] = np.arange(nc)
    new_of_old = np.concatenate([pn, nv + np.arange(nf), nv + nf + inv_pc])
    Bp = B[new_of_old][:, new_of_old]
    assert abs(Bp - A).max() <= 1e-13 * abs(A).max()
    u = vo.solve_full(pb, A)
    v = vo.solve_full(q, B)
    assert np.abs(v[new_of_old] - u).max() <= 1e-11 * np.abs(u).max()


def test_zero_flux_at_constant_pressure():
    pb = _scale_small()
    m = vo.Mesh(pb)
    cm = vo.cell_local_matrices(pb, m)
    fm = vo.fracture_local_matrices(pb, m)
    u = np.full(pb.n_nodes + pb.n_ff + pb.n_cells, 3.25)
    s = np.abs(cm["M"]).max()
    assert np.abs(vo.cell_fluxes(cm, u)).max() <= 1e-13 * s
    assert np.abs(vo.fracture_fluxes(fm, u)).max() <= 1e-13 * np.abs(fm["M"]).max()


def test_affine_exact_config1_boundary_conditions():
    """p = 1 - x with no-flow walls parallel to grad p and a fracture normal to
    it, on a jittered mesh: the scheme reproduces p at every node, fracture
    face and cell (Sec. 3.1 exactness of the P1 Galerkin form on affine
    functions)."""
    n = 6
    pb = vi.build_problem((n, n, n), [(0, n // 2, 0, n, 0, n)], jitter=0.2, seed=5, ratio=1e4)
    m = vo.Mesh(pb)
    u = vo.solve_full(pb)
    ex = np.concatenate([1 - pb.xyz[:, 0], 1 - m.xS[pb.ff_faces, 0], 1 - m.xK[:, 0]])
    assert np.abs(u - ex).max() < 1e-11


def test_affine_exact_all_dirichlet_anisotropic():
    """Any affine p, constant anisotropic Lambda_m, fracture planes spanning the
    domain with Dirichlet boundary everywhere: exact."""
    n = 5
    fr = [(0, 3, 0, n, 0, n), (1, 2, 0, n, 0, n), (2, 2, 0, n, 0, n)]
    g = np.array([-1.0, 0.35, 0.2])
    base = vi.build_problem((n, n, n), fr, jitter=0.2, seed=11)
    x = base.xyz
    bnd = np.nonzero(np.any((x == 0) | (x == 1), axis=1))[0].astype(np.int32)
    vals = 0.5 + x[bnd] @ g
    pb = vi.build_problem((n, n, n), fr, jitter=0.2, seed=11, ratio=300.0,
                          dirichlet=(bnd, vals, np.zeros(bnd.size)))
    pb.lambda_m[:] = [2.0, 1.0, 0.5, 0.4, 0.1, -0.2]
    m = vo.Mesh(pb)
    u = vo.solve_full(pb)
    ex = np.concatenate([0.5 + pb.xyz @ g, 0.5 + m.xS[pb.ff_faces] @ g, 0.5 + m.xK @ g])
    assert np.abs(u - ex).max() < 1e-11


def test_schur_elimination_equals_full_dense_solve():
    """Eq. (eqschur) + Eq. (eqschurcell) against a dense solve of the full
    X_D system on a tiny heterogeneous mesh."""
    pb = _scale_small(n=3, seed=8)
    A = vo.assemble_full(pb)
    Ad = A.toarray()
    n = Ad.shape[0]
    isd = np.zeros(n, bool); isd[pb.dir_nodes] = True
    U = ~isd
    u = np.zeros(n); u[pb.dir_nodes] = pb.dir_values
    u[U] = np.linalg.solve(Ad[np.ix_(U, U)], -Ad[np.ix_(U, isd)] @ pb.dir_values)
    u2 = vo.solve_schur_direct(pb, A)
    assert np.abs(u2 - u).max() < 1e-10
    S, b, R = vo.schur_system(pb, A)
    Sd = S.toarray()
    assert np.abs(Sd - Sd.T).max() <= 1e-13 * np.abs(Sd).max()
    assert np.all(np.linalg.eigvalsh(0.5 * (Sd + Sd.T)) > 0)


def test_conservation_equations_hold():
    """The discrete conservation laws of Sec. 3.1: the fluxes of the solution
    sum to zero on every cell, fracture face and non-Dirichlet node."""
    pb = _scale_small(n=5, seed=4)
    dt = vo.DarcyTransport(pb)
    tr = dt.tr
    net = np.zeros(tr.n)
    np.add.at(net, tr.src, tr.F)
    np.add.at(net, tr.dst, -tr.F)
    net[pb.dir_nodes] = 0
    assert np.abs(net).max() <= 1e-9 * np.abs(tr.F).max()


# --------------------------------------------------------------------------
# transport invariants
# --------------------------------------------------------------------------

def test_transport_mass_balance_and_max_principle():
    pb = _scale_small(n=5, seed=6)
    dt = vo.DarcyTransport(pb)
    tr = dt.tr
    h = 0.9 * tr.cfl_dt()
    act = np.ones(tr.n, bool); act[pb.dir_nodes] = False
    c = pb.c0()
    for _ in range(40):
        mass0 = np.sum(tr.phi[act] * c[act])
        inflow = tr.boundary_inflow(c)
        cn = tr.step(c, h)
        mass1 = np.sum(tr.phi[act] * cn[act])
        assert abs(mass1 - mass0 - h * inflow) <= 1e-12 * max(1.0, np.sum(tr.phi))
        assert cn.min() >= -1e-14 and cn.max() <= 1 + 1e-14
        c = cn
    assert c[act].max() > 0.05          # the front moved in


def test_transport_constant_state_preserved():
    pb = _scale_small(n=5, seed=7)
    pb.cbar[:] = 1.0
    dt = vo.DarcyTransport(pb)
    c = np.ones(dt.tr.n)
    h = 0.9 * dt.tr.cfl_dt()
    for _ in range(20):
        c = dt.tr.step(c, h)
    assert np.abs(c - 1).max() < 1e-9


def test_cfl_step_is_sharp_enough():
    """At the CFL step the scheme is monotone: every update weight is in [0, 1]
    (diagonal coefficient 1 - dt/phi * outflow >= 0), and at a step 5x larger
    some weight turns negative."""
    pb = _scale_small(n=4, seed=2)
    tr = vo.DarcyTransport(pb).tr
    act = np.ones(tr.n, bool); act[pb.dir_nodes] = False
    out = tr.outflow()
    d = tr.cfl_dt()
    assert np.min(1 - d / tr.phi[act] * out[act]) >= -1e-12
    assert np.min(1 - 5 * d / tr.phi[act] * out[act]) < 0
