"""The general-cell workloads at the paper's sizes, checked where the oracle
cannot run whole (the meshes of `bench.py --workload tet54 / prism55`):

* the tetrahedral DFN of Sec. 5.4's size (6.0 M tetrahedra) and the prism
  mesh with wells of Sec. 5.5's size (12.4 M prisms, no Dirichlet node), in
  the benchmark's configuration (FP64 refinement around FP32 CG with the
  classical V-cycle, to 1e-8);
* the residual recomputed on the CPU from the exported system, the residual
  of sampled rows in the system built from the oracle's own local matrices
  of the cells and fracture faces around them, and the cell rows of those
  cells (the recovery);
* with wells: production equals injection, and the perforation rates equal
  WI (u_sigma - p_w) - q from the exported pressures;
* 100 transport steps: concentrations within the bound the flux imbalance of
  a 1e-8 pressure allows."""
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


def sampled_rows(pb, u, nodes, ffs):
    """Rows of the full system (oracle local matrices) for the given nodes
    and fracture faces, and the largest relative cell-row residual of the
    cells around them."""
    m = vo.Mesh(pb)
    nv, nf = pb.n_nodes, pb.n_ff
    want = np.zeros(nv + nf + pb.n_cells, bool)
    want[nodes] = True
    want[nv + np.asarray(ffs)] = True
    around = np.isin(pb.cell_nodes, nodes).any(axis=1) | np.isin(pb.cell_faces, pb.ff_faces[ffs]).any(axis=1)
    r = np.zeros(want.shape[0])
    worst = 0.0
    fm = vo.fracture_local_matrices(pb, m)
    mats = [(fm["dofs"], fm["M"], False)]
    for cells, _, _, _ in m.groups:
        sel = cells[around[cells]]
        if sel.size:
            cm = vo.cell_local_matrices(pb, m, sel)
            mats.append((cm["dofs"], cm["M"], True))
    for d, M, is_cell in mats:
        ok = d >= 0
        ud = np.where(ok, u[np.where(ok, d, 0)], 0.0)
        contrib = np.einsum("bij,bj->bi", M, ud)
        sel = ok & want[np.where(ok, d, 0)]
        np.add.at(r, d[sel], contrib[sel])
        if is_cell:
            rk = np.einsum("bj,bj->b", M[:, 0, :], ud)
            sk = np.einsum("bj,bj->b", np.abs(M[:, 0, :]), np.abs(ud))
            worst = max(worst, float(np.max(np.abs(rk) / sk)))
    return r, worst


def check(ctx, pb, well_arrays=None):
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG_RS, rtol=1e-8, maxit=5000)
    assert info.rel_residual <= 1e-8 and info.outer >= 2, (info.rel_residual, info.outer)
    e = s.export_system()
    n = len(e["rowptr"]) - 1
    A = sp.csr_matrix((e["val"], e["col"], e["rowptr"]), shape=(n, n))
    x = u[e["row_dof"]]
    nb = np.linalg.norm(e["rhs"])
    rel = np.linalg.norm(e["rhs"] - A @ x) / nb
    assert rel <= 1.01e-8, rel
    rng = np.random.default_rng(23)
    free = np.setdiff1d(np.arange(pb.n_nodes), pb.dir_nodes)
    nodes = rng.choice(free, size=2000, replace=False)
    perforated = set() if well_arrays is None else set(well_arrays["ff"].tolist())
    ffs = rng.choice([f for f in range(pb.n_ff) if f not in perforated], size=300, replace=False)
    r, cell_rel = sampled_rows(pb, u, nodes, ffs)
    rows = np.concatenate([r[nodes], r[pb.n_nodes + ffs]])
    # each full-system row is minus a component of the eliminated residual
    assert np.abs(rows).max() <= 1.01e-8 * nb, np.abs(rows).max() / nb
    assert cell_rel <= 1e-11, cell_rel
    rates = None
    if well_arrays is not None:
        w = well_arrays
        rates = s.well_rates(len(w["ff"]))
        expect = w["wi"] * (u[pb.n_nodes + w["ff"]] - w["pw"]) - w["q"]
        assert np.abs(rates - expect).max() <= 1e-12 * np.abs(expect).max()
        inj = -rates[rates < 0].sum()
        assert abs(rates.sum()) <= 1e-6 * inj, (rates.sum(), inj)
    c = pb.c0()
    tinf = s.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=100, cfl=0.9)
    assert tinf.steps == 100 and 0 < tinf.dt <= tinf.dt_max
    assert np.isfinite(c).all() and c.min() >= -1e-5 and c.max() <= 1 + 1e-5, (c.min(), c.max())
    s.close()
    return rates


def test_tet54_full_size(ctx):
    pb = vi.config_tet54()
    assert pb.n_cells == 6_000_000
    check(ctx, pb)


def test_prism55_full_size_with_wells(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = vi.config_prism55()
    assert pb.n_cells == 12_409_920 and len(pb.dir_nodes) == 0
    g = pb.meta["well_geometry"]
    pb.wells = vi.well_arrays(pb, pkg.peaceman_wi(g["dx"], g["dz"], g["d_f"], g["lam_f"], g["r_w"], mu=pb.mu))
    rates = check(ctx, pb, pb.wells)
    assert -rates[rates < 0].sum() == pytest.approx(5.0e6 / (365.0 * 86400.0), rel=1e-12)
