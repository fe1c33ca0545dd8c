"""Peaceman wells (Sec. 5.5) on the GPU against the oracle: the well index
of the C ABI equals the oracle's closed form; with wells alone fixing the
pressure on a fractured prism mesh, the pressure (relative L2 1e-10), the
perforation rates (1e-9 of the largest) and ten transport steps (1e-9
absolute) match; production equals injection; updated wells re-run the
numeric phase; inconsistent well data is rejected."""
import numpy as np
import pytest

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


def _pair(pb):
    """(oracle problem, library problem): each side computes its own WI."""
    import copy
    import paper_1602_03641_gb300 as pkg
    g = pb.meta["well_geometry"]
    po, pg = copy.deepcopy(pb), copy.deepcopy(pb)
    po.wells = vi.well_arrays(po, vo.peaceman_wi(g["dx"], g["dz"], g["d_f"], g["lam_f"], g["r_w"], mu=pb.mu))
    pg.wells = vi.well_arrays(pg, pkg.peaceman_wi(g["dx"], g["dz"], g["d_f"], g["lam_f"], g["r_w"], mu=pb.mu))
    return po, pg


def test_peaceman_index_matches_the_oracle():
    import paper_1602_03641_gb300 as pkg
    rng = np.random.default_rng(3)
    dx = rng.uniform(1, 60, 50)
    dz = rng.uniform(1, 20, 50)
    df = rng.uniform(0.01, 2, 50)
    lam = 10 ** rng.uniform(-13, -9, 50)
    rw = np.full(50, 0.1)
    wo = vo.peaceman_wi(dx, dz, df, lam, rw, mu=1e-3)
    wg = pkg.peaceman_wi(dx, dz, df, lam, rw, mu=1e-3)
    assert np.abs(wg - wo).max() <= 1e-14 * np.abs(wo).max()
    with pytest.raises(pkg.VagError):
        pkg.peaceman_wi(1.0, 1.0, 1.0, 1.0, 5.0)   # r_0 < r_w


CASES = {
    "prism": lambda: vi.well_problem((9, 6), 4, jitter=0.15, seed=2),
    "prism_half": lambda: vi.well_problem((12, 8), 6, split="half", jitter=0.1, seed=4),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wells_match_the_oracle(ctx, name, prec):
    import paper_1602_03641_gb300 as pkg
    po, pg = _pair(CASES[name]())
    ref = vo.DarcyTransport(po)
    s = pkg.assemble_problem(ctx, pg)
    precision = pkg.VAG_FP64 if prec == "fp64" else pkg.VAG_MIXED
    u, info = s.solve(precision=precision, precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000, raise_on_error=False)
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.ret)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10
    q = s.well_rates(len(pg.wells["ff"]))
    assert np.abs(q - ref.q_well).max() <= 1e-9 * np.abs(ref.q_well).max()
    assert abs(q.sum()) <= 1e-8 * np.abs(q).max()
    c = pg.c0()
    inf = s.transport(c, pg.phi_m, pg.phi_f, pg.cbar, n_steps=10, cfl=0.9)
    co, dto = ref.run_transport(10, cfl=0.9)
    assert inf.dt == pytest.approx(dto, rel=1e-9)
    assert np.abs(c - co).max() <= 1e-9
    assert c.min() >= -1e-14 and c.max() <= 1 + 1e-14
    s.close()


def test_updated_wells_and_a_dirichlet_boundary(ctx):
    """update_props with other wells equals a fresh assembly; wells also
    work next to Dirichlet nodes (both sources of the pressure level)."""
    import paper_1602_03641_gb300 as pkg
    po, pg = _pair(vi.well_problem((9, 6), 4, jitter=0.15, seed=2, dirichlet="x"))
    s = pkg.assemble_problem(ctx, pg)
    u0, _ = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000)
    ref = vo.DarcyTransport(po)
    assert np.linalg.norm(u0 - ref.u) / np.linalg.norm(ref.u) <= 1e-10
    for p in (po, pg):
        p.wells = dict(p.wells)
        p.wells["pw"] = p.wells["pw"] + 1.0e5 * (p.wells["wi"] > 0)
        p.wells["q"] = 2.0 * p.wells["q"]
    w = {k: np.ascontiguousarray(v) for k, v in pg.wells.items()}
    w["ff"] = w["ff"].astype(np.int32)
    s.update_props(np.ascontiguousarray(pg.lambda_m.ravel()), pg.lambda_f, pg.d_f, pg.mu, w)
    u1, _ = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000)
    ref1 = vo.DarcyTransport(po)
    assert np.linalg.norm(u1 - ref1.u) / np.linalg.norm(ref1.u) <= 1e-10
    s2 = pkg.assemble_problem(ctx, pg)
    u2, _ = s2.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000)
    assert np.array_equal(u1, u2)
    s.close()
    s2.close()


def test_wells_in_a_batch_and_the_server(ctx):
    import paper_1602_03641_gb300 as pkg
    _, pa = _pair(CASES["prism"]())
    _, pb = _pair(CASES["prism_half"]())
    bs = ctx.assemble_batch([pkg.general_arrays(pa), pkg.general_arrays(pb)])
    ub, _ = bs.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=5000)
    lay = bs.batch_layout()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    nv, nf = ns[-1], fs[-1]
    srv = pkg.Server(0, slots=1)
    for i, p in enumerate((pa, pb)):
        s = pkg.assemble_problem(ctx, p)
        ua, _ = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=5000)
        got = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]],
                              ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        assert np.array_equal(got, ua), i
        t = srv.submit(p, n_steps=0, precond=pkg.VAG_PC_AMG, rtol=1e-10)
        uu, _, r = srv.wait(t, 60000)
        assert r.status == pkg.VAG_OK and np.array_equal(uu, ua), i
        s.close()
    srv.close()
    bs.close()


def test_bad_wells_are_rejected(ctx):
    import paper_1602_03641_gb300 as pkg
    _, pg = _pair(CASES["prism"]())
    q = pkg.general_arrays(pg)

    def go(wells):
        return ctx.assemble_general(q["xyz"], q["face_node_ptr"], q["face_node_idx"], q["cell_face_ptr"],
                                    q["cell_face_idx"], q["ff_face_ids"], q["lambda_m"], q["lambda_f"], q["d_f"],
                                    q["mu"], q["dir_nodes"], q["dir_values"], wells)
    w = q["wells"]
    dup = dict(w, ff=np.concatenate([w["ff"][:1], w["ff"][:-1]]).astype(np.int32))
    bad_ff = dict(w, ff=w["ff"].copy())
    bad_ff["ff"][0] = pg.n_ff
    neg = dict(w, wi=w["wi"].copy())
    neg["wi"][-1] = -1.0
    no_level = dict(w, wi=np.zeros_like(w["wi"]))     # no Dirichlet node and no producer
    for bad in (dup, bad_ff, neg, no_level):
        with pytest.raises(pkg.VagError) as e:
            go(bad)
        assert e.value.code == pkg.VAG_EINVAL
