"""Batches of independent realisations (disjoint-union assembly, per-system CG
scalars and CFL steps) against the same systems solved alone and against the
oracle.  A system must give bitwise the same pressures, fluxes, CFL step and
concentrations alone and inside any batch."""
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


def mixed_problems():
    return [
        vi.random_dfn_problem(9, 5, 1e3, seed=1),
        vi.config_plain16(6),
        vi.build_problem((5, 7, 4), [], jitter=0.2, seed=9, lam_m="lognormal"),
        vi.random_dfn_problem(12, 12, 1e6, seed=2),
        vi.build_problem((1, 1, 1), []),                 # no Krylov unknowns at all
        vi.random_dfn_problem(7, 3, 1e4, seed=3),
    ]


def slices(lay, i, nv, nf):
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    return (slice(ns[i], ns[i + 1]), slice(nv + fs[i], nv + fs[i + 1]), slice(nv + nf + cs[i], nv + nf + cs[i + 1]))


def concat_cv(pbs, arrs):
    """Union [nodes | ffaces | cells] vector from per-system ones."""
    nodes = [a[:p.n_nodes] for p, a in zip(pbs, arrs)]
    ffs = [a[p.n_nodes:p.n_nodes + p.n_ff] for p, a in zip(pbs, arrs)]
    cells = [a[p.n_nodes + p.n_ff:] for p, a in zip(pbs, arrs)]
    return np.concatenate(nodes + ffs + cells)


def test_batch_equals_alone_bitwise_and_matches_oracle(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = mixed_problems()
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    assert lay["n_sys"] == len(pbs)
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, info = bs.solve(rtol=1e-12, maxit=20000, raise_on_error=False)
    infos = bs.solve_infos()
    Fb = bs.export_fluxes()
    c0 = concat_cv(pbs, [p.c0() for p in pbs])
    phm = np.concatenate([p.phi_m for p in pbs])
    phf = np.concatenate([p.phi_f for p in pbs])
    cb = np.concatenate([p.cbar for p in pbs])
    cbat = c0.copy()
    bs.transport(cbat, phm, phf, cb, n_steps=25, cfl=0.9)
    dmaxb, dtb = bs.transport_dts()
    cstart = lay["cell_start"]
    fstart = lay["ff_start"]
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(rtol=1e-12, maxit=20000, raise_on_error=False)
        sn, sf, sc = slices(lay, i, nv, nf)
        ui = np.concatenate([ub[sn], ub[sf], ub[sc]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        assert infos[i].rel_residual == inf1.rel_residual
        F1 = s1.export_fluxes()
        np.testing.assert_array_equal(Fb[0][cstart[i]:cstart[i + 1]], F1[0])
        np.testing.assert_array_equal(Fb[1][cstart[i]:cstart[i + 1]], F1[1])
        np.testing.assert_array_equal(Fb[2][fstart[i]:fstart[i + 1]], F1[2])
        c1 = pb.c0()
        t1 = s1.transport(c1, pb.phi_m, pb.phi_f, pb.cbar, n_steps=25, cfl=0.9)
        assert dtb[i] == t1.dt
        ci = np.concatenate([cbat[sn], cbat[sf], cbat[sc]])
        np.testing.assert_array_equal(ci, c1)
        ref = vo.DarcyTransport(pb)
        assert np.linalg.norm(u1 - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        s1.close()


def test_batch_order_does_not_matter(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = mixed_problems()
    a = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    b = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs[::-1]])
    ua, _ = a.solve(rtol=1e-12, raise_on_error=False)
    ub, _ = b.solve(rtol=1e-12, raise_on_error=False)
    la, lb = a.batch_layout(), b.batch_layout()
    na, fa = la["node_start"][-1], la["ff_start"][-1]
    n = len(pbs)
    for i in range(n):
        j = n - 1 - i
        sa = slices(la, i, na, fa)
        sb = slices(lb, j, na, fa)
        for x, y in zip(sa, sb):
            np.testing.assert_array_equal(ua[x], ub[y])


def test_batch_device_inputs(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = mixed_problems()[:3]
    hb = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    db = ctx.assemble_batch([pkg.problem_arrays(p, device=True) for p in pbs])
    uh, _ = hb.solve(rtol=1e-12, raise_on_error=False)
    out = torch.empty(len(uh), dtype=torch.float64, device="cuda")
    db.solve(out=out, rtol=1e-12, raise_on_error=False)
    np.testing.assert_array_equal(out.cpu().numpy(), uh)


def test_batch_rejects_mixed_mu(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = mixed_problems()[:2]
    qs = [pkg.problem_arrays(p) for p in pbs]
    qs[1]["mu"] = 2.0
    with pytest.raises(pkg.VagError) as e:
        ctx.assemble_batch(qs)
    assert e.value.code == pkg.VAG_EINVAL


def test_mixed_batch_equals_alone_bitwise(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = mixed_problems()
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, _ = bs.solve(precision=pkg.VAG_MIXED, rtol=1e-10, raise_on_error=False)
    infos = bs.solve_infos()
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precision=pkg.VAG_MIXED, rtol=1e-10, raise_on_error=False)
        sn, sf, sc = slices(lay, i, nv, nf)
        np.testing.assert_array_equal(np.concatenate([ub[sn], ub[sf], ub[sc]]), u1)
        assert infos[i].iterations == inf1.iterations and infos[i].outer == inf1.outer
        assert infos[i].rel_residual <= 1e-10
        s1.close()
