"""Parity at the full size of the benchmark workload (64^3 jittered hex, four
fractures, lognormal anisotropic permeability, ratio 1e4), in the launch
configuration bench.py times: FP64 aggregation-AMG CG to 1e-10, then 200
explicit steps at CFL 0.9.

The oracle assembles this system in seconds but its tight solve would take
minutes, so the comparison is element by element where the oracle can compute
the values (every entry of the eliminated system, the cell recovery, every
flux, one transport step from the same state) and by properties that hold at
any size where it cannot (the residual of the GPU pressure in the oracle's
own system, the discrete maximum principle and the mass balance of the 200
steps)."""
import numpy as np
import pytest
import scipy.sparse as sp

import vag_inputs as vi
from oracle import vag_oracle as vo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    pb = vi.config_scale64(64)
    ctx = pkg.Context(0)
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000)
    m = vo.Mesh(pb)
    cms = vo._all_cell_matrices(pb, m)
    fm = vo.fracture_local_matrices(pb, m)
    A = vo.assemble_full(pb, m, cms, fm)
    S, b, R = vo.schur_system(pb, A)
    yield dict(pkg=pkg, pb=pb, ctx=ctx, s=s, u=u, info=info, m=m, cms=cms, fm=fm, A=A, S=sp.csr_matrix(S), b=b, R=R)
    s.close()
    ctx.close()


def test_eliminated_system_every_entry(full):
    e = full["s"].export_system()
    S, b, R = full["S"], full["b"], full["R"]
    n = len(e["rowptr"]) - 1
    assert n == len(R) == 280511
    np.testing.assert_array_equal(e["row_dof"], R)
    G = sp.csr_matrix((e["val"], e["col"], e["rowptr"]), shape=(n, n))
    scale = abs(S).max()
    assert abs(G - S).max() <= 1e-12 * scale
    assert np.abs(e["rhs"] - b).max() <= 1e-12 * max(np.abs(b).max(), scale)


def test_pressure_solves_the_oracle_system(full):
    """The GPU pressure, put into the oracle's eliminated system, leaves a
    relative residual within the requested 1e-10 (plus the 1e-12 entry gap)."""
    u, info, S, b, R = full["u"], full["info"], full["S"], full["b"], full["R"]
    assert info.rel_residual <= 1e-10
    x = u[R]
    rel = np.linalg.norm(b - S @ x) / np.linalg.norm(b)
    assert rel <= 1.5e-10, rel


def test_cell_recovery_and_fluxes(full):
    """Cell values and every flux recomputed by the oracle from the GPU's own
    node and fracture-face pressures."""
    from test_gpu_parity import gpu_fluxes_from_oracle
    pb, u, A = full["pb"], full["u"], full["A"]
    uo = vo.recover_cells(pb, A, u)
    nvf = pb.n_nodes + pb.n_ff
    assert np.abs(u[nvf:] - uo[nvf:]).max() <= 1e-12 * np.abs(uo).max()
    Fc = [vo.cell_fluxes(cm, uo) for cm in full["cms"]]
    Ff = vo.fracture_fluxes(full["fm"], uo)
    On, Of, Off = gpu_fluxes_from_oracle(pb, full["cms"], Fc, Ff)
    Fcn, Fcf, Fff = full["s"].export_fluxes()
    scale = max(np.abs(On).max(), np.abs(Off).max())
    assert np.abs(Fcn - On).max() <= 1e-10 * scale
    assert np.abs(Fcf - Of).max() <= 1e-10 * scale
    assert np.abs(Fff - Off).max() <= 1e-10 * scale


def test_transport_step_and_200_steps(full):
    """One step from the same state with the same (oracle) fluxes, element by
    element; then the benchmark's 200 steps on the GPU's own fluxes: the
    discrete maximum principle and the mass balance of the oracle's control
    volumes, step by step summed."""
    from test_gpu_parity import gpu_fluxes_from_oracle
    pb, u, A, s = full["pb"], full["u"], full["A"], full["s"]
    uo = vo.recover_cells(pb, A, u)
    Fc = [vo.cell_fluxes(cm, uo) for cm in full["cms"]]
    Ff = vo.fracture_fluxes(full["fm"], uo)
    tr = vo.Transport(pb, full["cms"], full["fm"], Fc, Ff, omega=0.5, mesh=full["m"])
    On, Of, Off = gpu_fluxes_from_oracle(pb, full["cms"], Fc, Ff)
    s.set_fluxes(On, Of, Off)
    rng = np.random.default_rng(9)
    c = rng.uniform(0, 1, tr.n)
    c[pb.dir_nodes] = pb.cbar
    dt = 0.9 * tr.cfl_dt()
    cg = c.copy()
    inf = s.transport(cg, pb.phi_m, pb.phi_f, pb.cbar, n_steps=1, cfl=0.0, dt=dt)
    assert np.abs(cg - tr.step(c, dt)).max() <= 1e-12
    assert inf.dt_max == pytest.approx(tr.cfl_dt(), rel=1e-12)
    # 200 steps at CFL 0.9 from c0, one call (as the benchmark runs them):
    # concentrations stay in [0, 1]
    c = pb.c0()
    inf = s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=200, cfl=0.9)
    assert inf.steps == 200
    # the discrete maximum principle holds for exactly conservative fluxes; a
    # pressure converged to 1e-10 leaves each volume a net flux imbalance
    # |sum F| <= delta * (its outflow), which a step at CFL 0.9 turns into an
    # overshoot of at most 0.9 delta: over 200 steps at most 180 delta
    net = np.bincount(tr.src, tr.F, tr.n) - np.bincount(tr.dst, tr.F, tr.n)
    out = tr.outflow()
    act_out = np.ones(tr.n, bool)
    act_out[pb.dir_nodes] = False
    act_out &= out > 0
    delta = float(np.max(np.abs(net[act_out]) / out[act_out]))
    assert c.min() >= -180 * delta - 1e-13 and c.max() <= 1 + 180 * delta + 1e-13, (c.min(), c.max(), delta)
    assert c.min() >= -1e-6 and c.max() <= 1 + 1e-6
    # the first 20 of those steps, element by element against the oracle's step
    c20 = pb.c0()
    s.transport(c20, pb.phi_m, pb.phi_f, pb.cbar, n_steps=20, cfl=0.0, dt=inf.dt)
    co = pb.c0()
    for _ in range(20):
        co = tr.step(co, inf.dt)
    assert np.abs(c20 - co).max() <= 1e-12
    # mass balance: over single GPU steps at that dt, the mass in the
    # non-Dirichlet volumes changes exactly by the net inflow through the
    # edges that touch a Dirichlet node
    act = np.ones(tr.n, bool)
    act[pb.dir_nodes] = False
    for _ in range(10):
        m0 = float(np.sum(tr.phi[act] * c[act]))
        gain = inf.dt * tr.boundary_inflow(c)
        s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=1, cfl=0.0, dt=inf.dt)
        m1 = float(np.sum(tr.phi[act] * c[act]))
        assert abs(m1 - (m0 + gain)) <= 1e-12 * max(m1, 1e-300) + 1e-15, (m1, m0, gain)
