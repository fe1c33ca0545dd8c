"""The GPU path against the paper's one-fracture analytical solution
(Sec. 5.1) on meshes up to 512 x 512: the Darcy pressure is exact for the
affine solution u = 1 - x, and the transported concentration at t_f = 1/2
(time step of Sec. 4.3: the CFL maximum, the last step shortened) converges
in L1 to the closed form, faster in the fracture than in the matrix.  At
64 x 64 the GPU concentrations equal the oracle's; at 64, 128 and 256 the
L1 errors equal the oracle's stored ones."""
import os

import numpy as np
import pytest

import vag_inputs as vi
from oracle import analytic as an
from oracle import vag_oracle as vo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T_F = 0.5
# the oracle's errors at 64, 128, 256 (tests/golden/make_one_fracture_errors.py)
GOLD = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "one_fracture_l1_errors.txt"), comments="#")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def _cell_volumes(pb, m):
    """Sum of the 24 tetrahedra (x_K, x_sigma, e) of each cell: the volume
    the scheme integrates over (pinned to the oracle's at 64 x 64 below)."""
    vol = np.zeros(pb.n_cells)
    for f in range(pb.cell_faces.shape[1]):
        fid = pb.cell_faces[:, f]
        fn = pb.faces[fid]
        xs = m.xS[fid]
        q = fn.shape[1]
        for e in range(q):
            a = pb.xyz[fn[:, e]] - m.xK
            b = pb.xyz[fn[:, (e + 1) % q]] - m.xK
            s = xs - m.xK
            vol += np.abs(np.einsum("ij,ij->i", s, np.cross(a, b))) / 6.0
    return vol


def _errors(pb, c, vol, m):
    s = an.OneFracture()
    nv, nf = pb.n_nodes, pb.n_ff
    ex_k = s.c_m(m.xK[:, 0], m.xK[:, 1], T_F)
    em = np.sum(vol * np.abs(c[nv + nf:] - ex_k)) / np.sum(vol * np.abs(ex_k))
    area = vo.fracture_local_matrices(pb, m)["area"]
    ex_f = s.c_f(m.xS[pb.ff_faces][:, 0], T_F)
    ef = np.sum(area * np.abs(c[nv:nv + nf] - ex_f)) / np.sum(area * np.abs(ex_f))
    return em, ef


def _gpu_run(ctx, pb):
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000, raise_on_error=False)
    assert info.rel_residual <= 1e-11, info.rel_residual
    c = pb.c0()
    dt = s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=0, cfl=1.0).dt_max
    n_steps = int(np.ceil(T_F / dt))
    if n_steps > 1:
        s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=n_steps - 1, cfl=0.0, dt=dt)
    s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=1, cfl=0.0, dt=T_F - (n_steps - 1) * dt)
    s.close()
    return u, c, dt, n_steps


def test_one_fracture_converges_on_gpu(ctx):
    ns = [64, 128, 256, 512]
    em, ef = [], []
    for n in ns:
        pb = vi.one_fracture_problem(n)
        u, c, dt, steps = _gpu_run(ctx, pb)
        # u = 1 - x is in the discrete space: reproduced to the solve's accuracy
        assert np.abs(u[:pb.n_nodes] - (1.0 - pb.xyz[:, 0])).max() < 1e-8
        # maximum principle under the CFL bound
        assert c.min() >= -1e-9 and c.max() <= 1.0 + 1e-7, (c.min(), c.max())
        m = vo.Mesh(pb)
        vol = _cell_volumes(pb, m)
        if n == 64:
            np.testing.assert_allclose(vol, vo.cell_local_matrices(pb, m)["vol"], rtol=1e-12)
            d = vo.DarcyTransport(pb)
            c_ref, dt_ref, steps_ref = d.run_to_time(T_F)
            assert steps == steps_ref and dt == pytest.approx(dt_ref, rel=1e-7)
            assert np.abs(c - c_ref).max() <= 1e-7
        e = _errors(pb, c, vol, m)
        em.append(e[0])
        ef.append(e[1])
        ref = GOLD[GOLD[:, 0] == n]
        if len(ref):   # the oracle's run of the same mesh: same steps, same errors
            _, steps_or, dt_or, em_or, ef_or = ref[0]
            assert steps == int(steps_or) and dt == pytest.approx(dt_or, rel=1e-7)
            assert e[0] == pytest.approx(em_or, rel=1e-4) and e[1] == pytest.approx(ef_or, rel=1e-4)
    em, ef = np.array(em), np.array(ef)
    assert np.all(np.diff(em) < 0) and np.all(np.diff(ef) < 0), (em, ef)
    assert np.all(ef < em), (em, ef)
    pm = -np.polyfit(np.log(ns), np.log(em), 1)[0]
    pf = -np.polyfit(np.log(ns), np.log(ef), 1)[0]
    # first-order upwind across a discontinuous front: about 1/2 in the
    # matrix; the fracture (a 1-D transport with a smooth source) about 1
    assert pm > 0.4, (em, pm)
    assert pf > 0.8, (ef, pf)
