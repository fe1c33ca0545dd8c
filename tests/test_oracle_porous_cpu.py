"""Pins of the oracle's control volumes (Sec. 3.2.1) and of its iterative solver.

Control volumes.  Sec. 3.2.1 partitions every cell K into omega_K and pieces
omega_{K,s} for its nodes outside V_ext u V_Gamma, and every fracture face
sigma into omega_sigma and pieces omega_{sigma,s} for its nodes outside
V_ext; a fracture node collects only fracture pieces, a matrix node only
matrix pieces, so the two rocktypes never mix.  With the library's fractions
alpha_{K,s} = omega/8 and alpha_{sigma,s} = omega/4 on a uniform lattice,
every porous volume is a count of cells or faces times a fixed number.  The
values below are worked out by hand on a 4^3 unit-cube lattice (h = 1/4) with
a fracture on the half plane x = 1/2, y < 1/2, Dirichlet nodes on x = 0 and
x = 1, phi_m = 0.2, phi_f = 0.4, d_f = 0.01:
  one cell:              phi_m h^3        = 0.2 / 64   = 3.125e-3
  one fracture face:     phi_f d_f h^2    = 0.004 / 16 = 2.5e-4.

Solver.  The oracle's Jacobi-CG (used above 30 000 unknowns) must give the
sparse direct solution on a case of that size.  CPU only.
"""
import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo

H3 = 0.2 / 64.0           # pore volume of one cell
A2 = 0.4 * 0.01 / 16.0    # pore volume of one fracture face


def _half_plane_problem():
    n = 4
    return vi.build_problem((n, n, n), [(0, 2, 0, 2, 0, n)], ratio=1e2, phi_m=0.2, phi_f=0.4, d_f=0.01)


def _porous(pb, omega):
    dt = vo.DarcyTransport(pb)
    tr = vo.Transport(pb, dt.cellmats, dt.fracmats, dt.F_cell, dt.F_frac, omega=omega, mesh=dt.mesh)
    return tr.phi


def _node(i, j, k, n=4):
    return i + (n + 1) * (j + (n + 1) * k)


def _cell(pb, i, j, k, n=4):
    return pb.n_nodes + pb.n_ff + i + n * (j + n * k)


# (node (i, j, k), porous volume at omega = 1/2, why)
NODE_CASES = [
    ((1, 2, 2), 8 * (0.5 / 8) * H3, "interior matrix node: 8 cells give omega/8 each"),
    ((2, 3, 2), 8 * (0.5 / 8) * H3, "matrix node on the fracture plane but off the fracture"),
    ((1, 0, 2), 4 * (0.5 / 8) * H3, "matrix node on the no-flow wall y = 0: 4 cells"),
    ((1, 0, 0), 2 * (0.5 / 8) * H3, "matrix node on the edge y = z = 0: 2 cells"),
    ((2, 1, 2), 4 * (0.5 / 4) * A2, "fracture node inside the fracture: 4 faces give omega/4, no matrix share"),
    ((2, 2, 2), 2 * (0.5 / 4) * A2, "fracture node on the fracture tip y = 1/2: 2 faces, no matrix share"),
    ((2, 1, 0), 2 * (0.5 / 4) * A2, "fracture node on the wall z = 0: 2 faces"),
    ((2, 0, 0), 1 * (0.5 / 4) * A2, "fracture node on the edge y = z = 0: 1 face"),
    ((0, 2, 2), 0.0, "Dirichlet node"),
    ((4, 1, 1), 0.0, "Dirichlet node"),
]

# (cell (i, j, k), porous volume at omega = 1/2): the cell keeps 1 - omega/8
# per node outside V_ext u V_Gamma
CELL_CASES = [
    ((0, 2, 2), (1 - 4 * 0.5 / 8) * H3),   # 4 Dirichlet nodes on x = 0, 4 matrix nodes
    ((1, 0, 1), (1 - 4 * 0.5 / 8) * H3),   # 4 of its nodes lie on the fracture
    ((1, 2, 1), (1 - 6 * 0.5 / 8) * H3),   # 2 nodes on the fracture tip
    ((1, 3, 1), (1 - 8 * 0.5 / 8) * H3),   # no Dirichlet, no fracture node
    ((2, 1, 1), (1 - 4 * 0.5 / 8) * H3),   # the other side of the fracture
    ((3, 1, 1), (1 - 4 * 0.5 / 8) * H3),   # 4 Dirichlet nodes on x = 1
]


def test_porous_volumes_closed_form_per_class():
    pb = _half_plane_problem()
    assert pb.n_ff == 8
    phi = _porous(pb, 0.5)
    for (ijk, expect, why) in NODE_CASES:
        assert phi[_node(*ijk)] == pytest.approx(expect, rel=1e-12, abs=1e-18), (ijk, why)
    for (ijk, expect) in CELL_CASES:
        assert phi[_cell(pb, *ijk)] == pytest.approx(expect, rel=1e-12), ijk
    # every fracture face: its four nodes are off V_ext, each takes omega/4
    ffv = phi[pb.n_nodes:pb.n_nodes + pb.n_ff]
    np.testing.assert_allclose(ffv, (1 - 4 * 0.5 / 4) * A2, rtol=1e-12)
    # nothing is created or lost: total = phi_m |Omega| + phi_f d_f |Gamma|
    assert phi.sum() == pytest.approx(0.2 * 1.0 + 0.4 * 0.01 * 0.5, rel=1e-12)


@pytest.mark.parametrize("omega", [0.0, 0.25, 0.9])
def test_porous_volumes_omega_sweep(omega):
    """At omega = 0 nodes hold nothing and cells / faces keep their whole pore
    volume; every volume is affine in omega with the slopes of the counts."""
    pb = _half_plane_problem()
    phi = _porous(pb, omega)
    for (ijk, expect, why) in NODE_CASES:
        assert phi[_node(*ijk)] == pytest.approx(expect * omega / 0.5, rel=1e-12, abs=1e-18), (ijk, why)
    slopes = {(0, 2, 2): 4, (1, 0, 1): 4, (1, 2, 1): 6, (1, 3, 1): 8}
    for ijk, cnt in slopes.items():
        assert phi[_cell(pb, *ijk)] == pytest.approx((1 - cnt * omega / 8) * H3, rel=1e-12), ijk
    np.testing.assert_allclose(phi[pb.n_nodes:pb.n_nodes + pb.n_ff], (1 - omega) * A2, rtol=1e-12)


def test_total_pore_volume_on_a_jittered_mesh():
    """Jittered 8^3 lattice with the benchmark's four fractures (three full
    planes and the half plane x = 1/4, y < 1/2): the cells still tile the unit
    cube and the fractures still cover area 3.5 (fracture-normal coordinates
    are frozen and the half plane's tip lies on the frozen plane y = 1/2), so
    the porous volumes add up to phi_m + phi_f d_f 3.5 whatever omega is."""
    pb = vi.config_scale64(8)
    pb.phi_m[:] = 0.2
    pb.phi_f[:] = 0.4
    for omega in (0.0, 0.5, 0.9):
        phi = _porous(pb, omega)
        assert phi.sum() == pytest.approx(0.2 + 0.4 * 0.01 * 3.5, rel=1e-12), omega
        assert np.all(phi[pb.dir_nodes] == 0.0)
        if omega > 0:
            assert np.all(np.delete(phi, pb.dir_nodes) > 0.0)


def test_jacobi_cg_equals_direct_solve():
    """The oracle switches to its Jacobi-CG above 30 000 unknowns; on the
    128 x 128 one-fracture mesh of Sec. 5.1 (49 794 unknowns, the case behind
    the golden L1 errors) it must give the sparse direct solution."""
    pb = vi.one_fracture_problem(128)
    d = vo.DarcyTransport(pb, solver="direct")
    c = vo.DarcyTransport(pb, solver="schur_pcg")
    assert d.A.shape[0] > 30000
    assert np.linalg.norm(c.u - d.u) / np.linalg.norm(d.u) <= 1e-11
