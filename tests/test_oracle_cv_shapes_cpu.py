"""Pins of the oracle's control volumes on every cell shape, and of its CFL
step, against values computed here from the definitions (CPU only).

Control volumes (Sec. 3.2.1, reading 8): a cell K gives alpha_{K,s} =
omega/|V_K| of its pore volume to each node s in V_K outside V_D u V_Gamma
and keeps the rest; a fracture face sigma gives alpha_{sigma,s} =
omega/|V_sigma| of its pore volume to each node s in V_sigma outside V_D.
On undistorted meshes every cell of one shape has the same volume (h^3/6 for
the tetrahedra of a Kuhn-cut cube and for the six pyramids of a cube, half
the box for a prism) and every fracture face the same area (h^2/2 for a
triangle, h^2 for a square), so each porous volume is a count of the cells
and faces around a node times those numbers.  The counts come from the raw
mesh arrays, in plain loops.

CFL step (Eq. eq_CFL): with cbar = 0 the explicit step is a linear map
c' = M c whose diagonal entry for control volume mu is 1 - dt/phi_mu times
the flux leaving mu; at dt = CFL x the bound, the smallest diagonal entry over
the non-Dirichlet volumes is exactly 1 - CFL, no entry of M is negative, and
the outflow behind the bound is, volume by volume, the one the step applies.
The columns of M are taken from the step itself applied to unit vectors.
"""
import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo


def _meshes():
    return {
        "tet": (vi.tet_problem((3, 3, 3), [(0, 1, 0, 3, 0, 3), (1, 2, 0, 2, 0, 3)]), 1.0 / 27 / 6, 1.0 / 9 / 2),
        "prism": (vi.prism_problem((3, 3), 3, [("x", 1, 0, 3, 0, 3), ("y", 2, 0, 2, 0, 2)]), 1.0 / 27 / 2,
                  1.0 / 9),
        "pyramid": (vi.pyramid_problem((2, 2, 2), [(0, 1, 0, 2, 0, 2)]), 1.0 / 8 / 6, 1.0 / 4),
    }


def _expected_porous(pb, vol, area, omega):
    """Porous volumes [nodes | fracture faces | cells] from the definition."""
    nv, nf, nc = pb.n_nodes, pb.n_ff, pb.n_cells
    isdir = np.zeros(nv, bool)
    isdir[pb.dir_nodes] = True
    ffn = [[int(v) for v in pb.faces[f] if v >= 0] for f in pb.ff_faces]
    frac_node = np.zeros(nv, bool)
    for nodes in ffn:
        frac_node[nodes] = True
    phi = np.zeros(nv + nf + nc)
    for K in range(nc):
        VK = sorted({int(v) for v in pb.cell_nodes[K] if v >= 0})
        pv = pb.phi_m[K] * vol
        give = [s for s in VK if not isdir[s] and not frac_node[s]]
        for s in give:
            phi[s] += omega / len(VK) * pv
        phi[nv + nf + K] = (1.0 - omega / len(VK) * len(give)) * pv
    for i, nodes in enumerate(ffn):
        pv = pb.phi_f[i] * pb.d_f[i] * area
        give = [s for s in nodes if not isdir[s]]
        for s in give:
            phi[s] += omega / len(nodes) * pv
        phi[nv + i] = (1.0 - omega / len(nodes) * len(give)) * pv
    return phi


@pytest.mark.parametrize("kind", ["tet", "prism", "pyramid"])
@pytest.mark.parametrize("omega", [0.5, 0.8])
def test_porous_volumes_per_shape(kind, omega):
    pb, vol, area = _meshes()[kind]
    assert pb.n_ff > 0 and len(pb.dir_nodes) > 0
    d = vo.DarcyTransport(pb)
    tr = vo.Transport(pb, d.cellmats, d.fracmats, d.F_cell, d.F_frac, omega=omega, mesh=d.mesh)
    expect = _expected_porous(pb, vol, area, omega)
    np.testing.assert_allclose(tr.phi, expect, rtol=1e-12, atol=1e-18)


def _step_matrix(tr, dt):
    n = tr.n
    M = np.zeros((n, n))
    for mu in range(n):
        e = np.zeros(n)
        e[mu] = 1.0
        M[:, mu] = tr.step(e, dt)
    return M


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_cfl_step_is_exactly_the_bound(kind):
    if kind == "hex":
        pb = vi.build_problem((4, 4, 3), [(0, 2, 0, 4, 0, 3)], jitter=0.2, seed=3, lam_m="lognormal", ratio=1e3)
    else:
        pb = vi.tet_problem((3, 3, 2), [(0, 1, 0, 3, 0, 2)], jitter=0.2, seed=4, lam_m="lognormal", ratio=1e3)
    pb.cbar[:] = 0.0                       # the step is then linear in c
    tr = vo.DarcyTransport(pb).tr
    cfl = 0.9
    dt = cfl * tr.cfl_dt()
    M = _step_matrix(tr, dt)
    act = np.ones(tr.n, bool)
    act[pb.dir_nodes] = False
    diag = np.diag(M)[act]
    assert diag.min() == pytest.approx(1.0 - cfl, abs=1e-12)
    # the outflow that sets the bound is the one the step applies, volume by volume
    out = tr.outflow()[act]
    np.testing.assert_allclose(out, (1.0 - diag) * tr.phi[act] / dt, rtol=1e-10, atol=1e-12 * out.max())
    assert M[act].min() >= -1e-14
    # 5 % above the bound the limiting volume's diagonal entry turns negative
    M2 = _step_matrix(tr, dt / cfl * 1.05)
    assert np.diag(M2)[act].min() < 0.0
