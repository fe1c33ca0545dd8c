"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances (each follows from the arithmetic noted beside it):
* eliminated-system entries and right-hand side: 1e-12 of the largest entry
  (same FP64 formulas, different summation order);
* pressures: relative L2 error <= 1e-10 with both sides converged far below it;
* fluxes: 1e-9 of the largest flux (they inherit the pressure gap times the
  transmissivities);
* porous volumes: 1e-13 relative;
* one transport step from the same state with the same fluxes: 1e-12 absolute
  (concentrations lie in [0, 1]).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import vag_inputs as vi
from oracle import vag_oracle as vo

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def scale_like(dims, seed=3, ratio=1e4):
    nx, ny, nz = dims
    fr = [(0, nx // 2, 0, ny, 0, nz), (1, ny // 2, 0, nx, 0, nz), (2, nz // 2, 0, nx, 0, ny),
          (0, max(1, nx // 4), 0, max(1, ny // 2), 0, nz)]
    return vi.build_problem(dims, fr, jitter=0.2, seed=seed, lam_m="lognormal", ratio=ratio)


CASES = {
    "plain8": lambda: vi.config_plain16(8),
    "plain16": lambda: vi.config_plain16(16),
    "scale_10x7x9": lambda: scale_like((10, 7, 9)),
    "dfn12": lambda: vi.random_dfn_problem(12, 8, 1e5, seed=17),
    "nofrac_5x4x3": lambda: vi.build_problem((5, 4, 3), [], jitter=0.2, seed=2, lam_m="lognormal"),
    "wallfrac": lambda: vi.build_problem((4, 5, 4), [(1, 0, 0, 4, 0, 4), (0, 2, 0, 5, 0, 4)], jitter=0.1, seed=4),
    "onefrac20": lambda: vi.one_fracture_problem(20),
    "fourfrac20": lambda: vi.four_fracture_problem(20),
}


def gpu_fluxes_from_oracle(pb, cms, F_cell, F_frac):
    """Oracle per-cell fluxes (slots: sorted V_K then fracture faces in face
    order) re-laid out as the library's [8 nc] / [6 nc] / [4 nf] arrays."""
    nv = pb.n_nodes
    Fcn = np.zeros((pb.n_cells, 8))
    Fcf = np.zeros((pb.n_cells, 6))
    for cm, F in zip(cms, F_cell):
        cells = cm["cells"]
        d = cm["dofs"][:, 1:]
        vk = d[:, :8]
        for l in range(8):
            node = pb.cell_nodes[cells, l]
            pos = np.argmax(vk == node[:, None], axis=1)
            Fcn[cells, l] = F[np.arange(len(cells)), pos]
        isff = np.isin(pb.cell_faces[cells], pb.ff_faces)
        rank = np.cumsum(isff, axis=1) - 1
        for lf in range(6):
            sel = isff[:, lf]
            Fcf[cells[sel], lf] = F[np.nonzero(sel)[0], 8 + rank[sel, lf]]
    return Fcn, Fcf, np.asarray(F_frac).reshape(-1, 4)


@pytest.fixture(scope="module")
def runs(ctx):
    import paper_1602_03641_gb300 as pkg
    out = {}
    for name, mk in CASES.items():
        pb = mk()
        ref = vo.DarcyTransport(pb)
        sysg = pkg.assemble_problem(ctx, pb)
        u, info = sysg.solve(rtol=1e-12, maxit=20000, raise_on_error=False)
        out[name] = (pb, ref, sysg, u, info)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_eliminated_system_matches(runs, name):
    pb, ref, sysg, u, info = runs[name]
    S, b, R = vo.schur_system(pb, ref.A)
    e = sysg.export_system()
    n = len(e["rowptr"]) - 1
    assert n == len(R)
    np.testing.assert_array_equal(e["row_dof"], R)
    G = sp.csr_matrix((e["val"], e["col"], e["rowptr"]), shape=(n, n))
    scale = abs(S).max()
    assert abs(G - S).max() <= 1e-12 * scale
    assert np.abs(e["rhs"] - b).max() <= 1e-12 * max(np.abs(b).max(), scale)
    # the pattern has no explicit zeros beyond what the oracle's sparsity allows
    assert G.nnz >= S.nnz - np.sum(np.abs(S.data) < 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_pressure_matches(runs, name):
    pb, ref, sysg, u, info = runs[name]
    # 1e-12 is requested; a few cases have their FP64 rounding floor near 2e-12
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations, info.ret)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-10, err


@pytest.mark.parametrize("name", list(CASES))
def test_fluxes_match(runs, name):
    pb, ref, sysg, u, info = runs[name]
    Fcn, Fcf, Fff = sysg.export_fluxes()
    On, Of, Off = gpu_fluxes_from_oracle(pb, ref.cellmats, ref.F_cell, ref.F_frac)
    scale = max(np.abs(On).max(), np.abs(Off).max() if Off.size else 0.0)
    assert np.abs(Fcn - On).max() <= 1e-9 * scale
    assert np.abs(Fcf - Of).max() <= 1e-9 * scale
    if pb.n_ff:
        assert np.abs(Fff - Off).max() <= 1e-9 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_transport_single_step_matches(runs, name):
    """One explicit step from the same state c^n with the oracle's fluxes."""
    pb, ref, sysg, u, info = runs[name]
    On, Of, Off = gpu_fluxes_from_oracle(pb, ref.cellmats, ref.F_cell, ref.F_frac)
    sysg.set_fluxes(On, Of, Off)
    rng = np.random.default_rng(5)
    c = rng.uniform(0, 1, ref.tr.n)
    c[pb.dir_nodes] = pb.cbar
    dt = 0.8 * ref.tr.cfl_dt()
    cg = c.copy()
    inf = sysg.transport(cg, pb.phi_m, pb.phi_f, pb.cbar, n_steps=1, cfl=0.0, dt=dt)
    assert inf.dt == dt
    co = ref.tr.step(c, dt)
    assert np.abs(cg - co).max() <= 1e-12
    phi = sysg.export_porous_volumes()
    assert np.abs(phi - ref.tr.phi).max() <= 1e-13 * ref.tr.phi.max()
    assert inf.dt_max == pytest.approx(ref.tr.cfl_dt(), rel=1e-12)


@pytest.mark.parametrize("name", ["plain16", "scale_10x7x9", "dfn12", "fourfrac20"])
def test_transport_ten_steps_end_to_end(ctx, name):
    """Solve + fluxes + CFL + 10 steps on the GPU's own fluxes vs the oracle's
    whole path (the gap inherits the pressure tolerance)."""
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    sysg = pkg.assemble_problem(ctx, pb)
    sysg.solve(rtol=1e-12, maxit=20000, raise_on_error=False)
    c = pb.c0()
    inf = sysg.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=10, cfl=0.9)
    co, dto = ref.run_transport(10, cfl=0.9)
    assert inf.dt == pytest.approx(dto, rel=1e-9)
    assert np.abs(c - co).max() <= 1e-9
    assert c.min() >= -1e-14 and c.max() <= 1 + 1e-14


def test_transport_step_entry_point(ctx):
    """vag_transport_step is vag_transport with the step returned: same
    concentrations bitwise, dt_used = info.dt."""
    import paper_1602_03641_gb300 as pkg
    pb = CASES["dfn12"]()
    s = pkg.assemble_problem(ctx, pb)
    s.solve(rtol=1e-12, maxit=20000, raise_on_error=False)
    c1, c2 = pb.c0(), pb.c0()
    i1 = s.transport(c1, pb.phi_m, pb.phi_f, pb.cbar, n_steps=7, cfl=0.9)
    i2, used = s.transport_step(c2, pb.phi_m, pb.phi_f, pb.cbar, n_steps=7, cfl=0.9)
    np.testing.assert_array_equal(c1, c2)
    assert used == i2.dt == i1.dt and i2.steps == 7
    s.close()


def test_spmv_matches(runs):
    pb, ref, sysg, u, info = runs["dfn12"]
    S, b, R = vo.schur_system(pb, ref.A)
    x = np.random.default_rng(1).normal(size=S.shape[0])
    y = sysg.spmv(x)
    assert np.abs(y - S @ x).max() <= 1e-12 * np.abs(S).max() * np.abs(x).max() * 30


def test_device_and_host_inputs_agree_bitwise(ctx, runs):
    import paper_1602_03641_gb300 as pkg
    pb, ref, sysg, u, info = runs["scale_10x7x9"]
    s2 = pkg.assemble_problem(ctx, pb, device=True)
    out = torch.empty(len(u), dtype=torch.float64, device="cuda")
    s2.solve(out=out, rtol=1e-12, maxit=20000, raise_on_error=False)
    np.testing.assert_array_equal(out.cpu().numpy(), u)


def test_single_cell_all_dirichlet(ctx):
    """Degenerate case: every node is Dirichlet, no Krylov unknowns."""
    import paper_1602_03641_gb300 as pkg
    pb = vi.build_problem((1, 1, 1), [])
    ref = vo.DarcyTransport(pb)
    sysg = pkg.assemble_problem(ctx, pb)
    assert sysg.info().n_rows == 0
    u, info = sysg.solve(rtol=1e-12)
    assert np.abs(u - ref.u).max() < 1e-14
    assert u[-1] == pytest.approx(0.5)


def test_error_paths(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = vi.config_plain16(4)
    bad = vi.config_plain16(4)
    bad.cell_nodes = bad.cell_nodes.copy()
    bad.cell_nodes[3, 2] = bad.n_nodes          # out of range
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, bad)
    assert e.value.code == pkg.VAG_EINVAL
    notface = vi.config_plain16(4)
    notface.ff_nodes = notface.ff_nodes.copy()
    notface.ff_nodes[0] = [0, 1, 7, 30]          # not a face of any cell
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, notface)
    assert e.value.code == pkg.VAG_EMESH
    dup = vi.config_plain16(4)
    dup.ff_nodes = np.concatenate([dup.ff_nodes, dup.ff_nodes[:1, ::-1]])
    dup.lambda_f = np.concatenate([dup.lambda_f, dup.lambda_f[:1]])
    dup.d_f = np.concatenate([dup.d_f, dup.d_f[:1]])
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, dup)
    assert e.value.code == pkg.VAG_EMESH
    dd = vi.config_plain16(4)
    dd.dir_nodes = np.concatenate([dd.dir_nodes, dd.dir_nodes[:1]])
    dd.dir_values = np.concatenate([dd.dir_values, dd.dir_values[:1]])
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, dd)
    assert e.value.code == pkg.VAG_EINVAL
    s = pkg.assemble_problem(ctx, pb)
    with pytest.raises(pkg.VagError) as e:
        s.transport(pb.c0(), pb.phi_m, pb.phi_f, pb.cbar, 1)
    assert e.value.code == pkg.VAG_EINVAL                 # no fluxes yet
    u, info = s.solve(rtol=1e-14, maxit=2, raise_on_error=False)
    assert info.ret == pkg.VAG_ENOTCONVERGED and info.iterations == 2
    small = pkg.Context(0, budget_bytes=4096)
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(small, pb)
    assert e.value.code == pkg.VAG_EBUDGET
    assert small.bytes_in_use() == 0
    small.close()


def test_invalid_inputs_are_reported(ctx):
    """Bad physical inputs end in a status code, never a crash or a silent
    result: negative or NaN permeabilities and NaN coordinates at assembly, a
    non-positive porosity at transport, an indefinite permeability tensor at
    the solve."""
    import paper_1602_03641_gb300 as pkg
    neg = vi.config_plain16(4)
    neg.lambda_m = -np.asarray(neg.lambda_m)
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, neg)
    assert e.value.code == pkg.VAG_EINVAL
    nanf = vi.config_plain16(4)
    nanf.lambda_f = np.asarray(nanf.lambda_f, float).copy()
    nanf.lambda_f[3] = np.nan
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, nanf)
    assert e.value.code == pkg.VAG_EINVAL
    nanx = vi.config_plain16(4)
    nanx.xyz = np.asarray(nanx.xyz, float).copy()
    nanx.xyz[30, 1] = np.nan
    with pytest.raises(pkg.VagError) as e:
        pkg.assemble_problem(ctx, nanx)
    assert e.value.code in (pkg.VAG_EMESH, pkg.VAG_EINVAL)
    pb = vi.config_plain16(4)
    s = pkg.assemble_problem(ctx, pb)
    s.solve(rtol=1e-10, maxit=1000)
    phi = np.asarray(pb.phi_m, float).copy()
    phi[5] = -0.1
    with pytest.raises(pkg.VagError) as e:
        s.transport(pb.c0(), phi, pb.phi_f, pb.cbar, 1)
    assert e.value.code == pkg.VAG_EINVAL
    s.close()
    # an indefinite tensor with a positive diagonal: Lambda = [[1, 3, 0], [3, 1, 0], [0, 0, 1]]
    ind = vi.build_problem((4, 4, 4), [], jitter=0.0, seed=1)
    lam = np.zeros((ind.n_cells, 6))
    lam[:, 0] = lam[:, 1] = lam[:, 2] = 1.0
    lam[:, 3] = 3.0
    ind.lambda_m = lam
    try:
        s = pkg.assemble_problem(ctx, ind)
    except pkg.VagError as err:        # caught at assembly: a non-positive diagonal
        assert err.code == pkg.VAG_EINVAL
    else:
        for pc in (pkg.VAG_PC_JACOBI, pkg.VAG_PC_AMG):
            _, info = s.solve(precond=pc, rtol=1e-10, maxit=500, raise_on_error=False)
            assert info.ret != pkg.VAG_OK, (pc, info.ret, info.rel_residual)
        s.close()


def test_deterministic_bitwise(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = vi.random_dfn_problem(14, 10, 1e4, seed=3)
    u1, _ = pkg.assemble_problem(ctx, pb).solve(rtol=1e-12)
    u2, _ = pkg.assemble_problem(ctx, pb).solve(rtol=1e-12)
    np.testing.assert_array_equal(u1, u2)


def test_context_destroyed_before_its_systems():
    """Destroying a context first is allowed: its systems stay usable and the
    context is released with the last of them."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1602_03641_gb300 as pkg
    c = pkg.Context(0)
    pb = vi.config_plain16(4)
    s1 = pkg.assemble_problem(c, pb)
    s2 = pkg.assemble_problem(c, pb)
    c.close()
    u1, _ = s1.solve(rtol=1e-12)
    s1.close()
    u2, _ = s2.solve(rtol=1e-12)
    np.testing.assert_array_equal(u1, u2)
    s2.close()


@pytest.mark.parametrize("name", ["plain16", "scale_10x7x9", "dfn12", "fourfrac20", "nofrac_5x4x3"])
def test_mixed_precision_reaches_fp64_accuracy(runs, name):
    """FP32 inner CG inside FP64 refinement: the residual is FP64, so the
    refinement reaches FP64 accuracy (same 1e-10 pressure bar as FP64 CG)."""
    import paper_1602_03641_gb300 as pkg
    pb, ref, sysg, u64, info64 = runs[name]
    u, info = sysg.solve(precision=pkg.VAG_MIXED, rtol=1e-11, maxit=20000, raise_on_error=False)
    assert info.ret == pkg.VAG_OK, (info.ret, info.rel_residual, info.outer)
    assert info.rel_residual <= 1e-11
    assert info.outer >= 2
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-10, err


def test_mixed_precision_at_1e8(runs):
    import paper_1602_03641_gb300 as pkg
    pb, ref, sysg, u64, info64 = runs["dfn12"]
    u, info = sysg.solve(precision=pkg.VAG_MIXED, rtol=1e-8, maxit=20000)
    assert info.rel_residual <= 1e-8
    # a 1e-8 residual bounds the error by cond(A) * 1e-8; here it stays small
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-6
