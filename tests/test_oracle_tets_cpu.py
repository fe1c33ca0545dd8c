"""The oracle on tetrahedral meshes (Sec. 3.1 admits any polyhedral cell; a
tetrahedron is its own sub-mesh of 12 tetrahedra T_{K,sigma,e}).  Pins that
do not depend on the cell shape: an affine pressure is reproduced exactly
with a fracture plane normal to its gradient, constant pressure has no flux,
the Galerkin matrix is symmetric with zero row sums, the cells tile the box,
the conservation equations hold, and the explicit transport conserves mass
and keeps 0 <= c <= 1 at CFL 0.9.  CPU only."""
import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo


@pytest.fixture(scope="module")
def tet():
    pb = vi.tet_problem((5, 4, 4), [(0, 2, 0, 4, 0, 4), (1, 2, 0, 2, 0, 4)], jitter=0.2, seed=3,
                        lam_m="lognormal", ratio=1e3)
    return pb, vo.DarcyTransport(pb)


def test_tet_mesh_shape():
    pb = vi.tet_problem((3, 2, 2), [(0, 1, 0, 2, 0, 2)])
    assert pb.n_cells == 6 * 12 and pb.faces.shape[1] == 3 and pb.cell_faces.shape == (72, 4)
    # every interior triangle is shared by two tetrahedra, boundary ones by one
    cnt = np.bincount(pb.cell_faces.ravel(), minlength=pb.faces.shape[0])
    assert set(np.unique(cnt)) == {1, 2}
    assert pb.n_ff == 2 * 2 * 2   # the fracture square of 2x2 lattice faces, two triangles each


def test_affine_pressure_is_exact_on_tets():
    """p = 1 - x with a fracture on x = 1/2 (normal to the gradient), constant
    tensor: the P1 scheme on the sub-mesh reproduces it at every node,
    fracture face and cell."""
    pb = vi.tet_problem((4, 3, 3), [(0, 2, 0, 3, 0, 3)], jitter=0.2, seed=1)
    d = vo.DarcyTransport(pb)
    m = d.mesh
    ex = np.concatenate([1 - pb.xyz[:, 0], 1 - m.xS[pb.ff_faces, 0], 1 - m.xK[:, 0]])
    assert np.abs(d.u - ex).max() <= 1e-12


def test_tet_galerkin_structure_and_volume(tet):
    pb, d = tet
    A = d.A
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    assert np.abs(np.asarray(A.sum(axis=1)).ravel()).max() <= 1e-12 * abs(A).max()
    assert sum(cm["vol"].sum() for cm in d.cellmats) == pytest.approx(1.0, rel=1e-13)
    u1 = np.ones(A.shape[0])
    F = [vo.cell_fluxes(cm, u1) for cm in d.cellmats]
    assert max(np.abs(f).max() for f in F) <= 1e-13 * abs(A).max()


def test_tet_conservation_equations(tet):
    """Residual of the full system at the non-Dirichlet rows (the
    conservation equations of the cells, fracture faces and free nodes)."""
    pb, d = tet
    r = d.A @ d.u
    free = np.ones(r.shape[0], bool)
    free[pb.dir_nodes] = False
    assert np.abs(r[free]).max() <= 1e-10 * np.abs(d.A).max()


def test_tet_transport_mass_and_max_principle(tet):
    pb, d = tet
    tr = d.tr
    dt = 0.9 * tr.cfl_dt()
    act = np.ones(tr.n, bool)
    act[pb.dir_nodes] = False
    c = pb.c0()
    for _ in range(30):
        m0 = float(np.sum(tr.phi[act] * c[act]))
        gain = dt * tr.boundary_inflow(c)
        c = tr.step(c, dt)
        m1 = float(np.sum(tr.phi[act] * c[act]))
        assert abs(m1 - (m0 + gain)) <= 1e-12 * max(m1, 1e-300) + 1e-15
    assert c.min() >= -1e-12 and c.max() <= 1 + 1e-12
    # matrix pore volume phi_m |Omega| plus phi_f d_f times the fracture areas
    # (the plane x = 2/5 over the unit square, 1.0; y = 1/2 for x < 2/5, 0.4)
    assert tr.phi.sum() == pytest.approx(0.2 * 1.0 + 0.4 * 0.01 * (1.0 + 0.4), rel=1e-12)
