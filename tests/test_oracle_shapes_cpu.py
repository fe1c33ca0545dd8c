"""The oracle on prisms (the extruded triangular meshes of Sec. 5.5), on
prisms mixed with hexahedra and on pyramids: the pins of the tetrahedral
case, which hold for any polyhedral cell of Sec. 3.1 (sub-mesh of the
tetrahedra T_{K,sigma,e}, one per edge of each face).  An affine pressure is
reproduced exactly when the fracture planes are normal to its gradient; the
Galerkin matrix is symmetric with zero row sums; the cells tile the box;
the conservation equations hold; the transport conserves mass and stays in
[0, 1]; the pore volume is phi_m |Omega| + phi_f d_f |Gamma|.  CPU only."""
import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo


def _mesh(kind, fr_x_only=False):
    if kind == "pyramid":
        return vi.pyramid_problem((3, 2, 2), [(0, 1, 0, 2, 0, 2)] + ([] if fr_x_only else [(1, 1, 0, 2, 0, 2)]),
                                  jitter=0.2, seed=2, lam_m="identity" if fr_x_only else "lognormal", ratio=1e3)
    split = {"prism": "all", "prism_half": "half", "prism_checker": "checker"}[kind]
    fr = [("x", 2, 0, 3, 0, 3)] + ([] if fr_x_only else [("d", 0, 0, 2, 0, 3), ("y", 1, 2, 4, 0, 2)])
    return vi.prism_problem((4, 3), 3, fr, split=split, jitter=0.2, seed=1,
                            lam_m="identity" if fr_x_only else "lognormal", ratio=1e3)


KINDS = ["prism", "prism_half", "prism_checker", "pyramid"]


@pytest.mark.parametrize("kind", KINDS)
def test_affine_pressure_is_exact(kind):
    pb = _mesh(kind, fr_x_only=True)
    d = vo.DarcyTransport(pb)
    m = d.mesh
    ex = np.concatenate([1 - pb.xyz[:, 0], 1 - m.xS[pb.ff_faces, 0], 1 - m.xK[:, 0]])
    assert np.abs(d.u - ex).max() <= 1e-12


@pytest.mark.parametrize("kind", KINDS)
def test_structure_volume_conservation_transport(kind):
    pb = _mesh(kind)
    d = vo.DarcyTransport(pb)
    A = d.A
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    assert np.abs(np.asarray(A.sum(axis=1)).ravel()).max() <= 1e-12 * abs(A).max()
    assert sum(cm["vol"].sum() for cm in d.cellmats) == pytest.approx(1.0, rel=1e-13)
    r = A @ d.u
    free = np.ones(r.shape[0], bool)
    free[pb.dir_nodes] = False
    assert np.abs(r[free]).max() <= 1e-10 * np.abs(A).max()
    # the fracture area from the fracture matrices equals the sum of the
    # fracture faces' own triangle areas
    fa = d.fracmats["area"]
    xyz = pb.xyz
    area = 0.0
    for f in pb.ff_faces:
        nodes = [v for v in pb.faces[f] if v >= 0]
        c = xyz[nodes].mean(axis=0)
        for t in range(len(nodes)):
            a, b = xyz[nodes[t]] - c, xyz[nodes[(t + 1) % len(nodes)]] - c
            area += 0.5 * np.linalg.norm(np.cross(a, b))
    assert fa.sum() == pytest.approx(area, rel=1e-13)
    tr = d.tr
    assert tr.phi.sum() == pytest.approx(0.2 + 0.4 * 0.01 * area, rel=1e-12)
    dt = 0.9 * tr.cfl_dt()
    act = np.ones(tr.n, bool)
    act[pb.dir_nodes] = False
    c = pb.c0()
    for _ in range(25):
        m0 = float(np.sum(tr.phi[act] * c[act]))
        gain = dt * tr.boundary_inflow(c)
        c = tr.step(c, dt)
        m1 = float(np.sum(tr.phi[act] * c[act]))
        assert abs(m1 - (m0 + gain)) <= 1e-12 * max(m1, 1e-300) + 1e-15
    assert c.min() >= -1e-12 and c.max() <= 1 + 1e-12


def test_mixed_mesh_groups_match_the_pure_meshes():
    """On a mesh of prism columns and hexahedral columns, every cell's local
    matrix equals the one the same cell gets in a mesh of its own shape
    alone (the local matrices depend on the cell only)."""
    mix = vi.prism_problem((4, 2), 2, [], split="half", jitter=0.0)
    allp = vi.prism_problem((4, 2), 2, [], split="all", jitter=0.0)
    m1, m2 = vo.Mesh(mix), vo.Mesh(allp)
    assert len(m1.groups) == 2
    for cells, VK, _, _ in m1.groups:
        cm = vo.cell_local_matrices(mix, m1, cells)
        if VK.shape[1] == 6:   # prisms: find the same node set in the all-prism mesh
            key2 = {tuple(v): i for i, v in enumerate(m2.groups[0][1].tolist())}
            other = np.array([m2.groups[0][0][key2[tuple(v)]] for v in VK.tolist()])
            cm2 = vo.cell_local_matrices(allp, m2, other)
            assert np.allclose(cm["M"], cm2["M"], rtol=0, atol=1e-14 * np.abs(cm["M"]).max())
        else:                  # hexahedra: boxes hx x hy x hz with the closed-form cell diagonal
            hx, hy, hz = 1 / 4, 1 / 2, 1 / 2
            C = 4 / 3 * (hx * hy / hz + hx * hz / hy + hy * hz / hx)
            assert np.allclose(cm["M"][:, 0, 0], C, rtol=1e-13)
