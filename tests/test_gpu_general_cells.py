"""General polyhedral cells on the GPU (Sec. 3.1; the tetrahedral meshes of
Sec. 5.4, the extruded triangular prisms of Sec. 5.5, pyramids, and prisms
mixed with hexahedra) through the general descriptor of the C ABI, against
the oracle element by element.

Tolerances as in the hexahedral parity tests: eliminated system 1e-12 of
its largest entry; pressure relative L2 1e-10 with both sides converged to
1e-12; fluxes 1e-9 of the largest; porous volumes 1e-13 relative; one
transport step from the same state 1e-12 absolute; ten steps on the GPU's
own fluxes 1e-9."""
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


def _prisms(split, nxy=(6, 5), nz=4, seed=1):
    nx, ny = nxy
    fr = [("x", nx // 2, 0, ny, 0, nz), ("d", 0, 0, min(nx, ny) // 2, 0, nz), ("y", ny // 2, 1, nx, 1, nz)]
    return vi.prism_problem(nxy, nz, fr, split=split, jitter=0.2, seed=seed, lam_m="lognormal", ratio=1e4)


CASES = {
    "tet": lambda: vi.tet_problem((5, 4, 4), [(0, 2, 0, 4, 0, 4), (1, 2, 0, 3, 0, 4)], jitter=0.2, seed=3,
                                  lam_m="lognormal", ratio=1e4),
    "prism": lambda: _prisms("all"),
    "prism_half": lambda: _prisms("half"),
    "prism_checker": lambda: _prisms("checker"),
    "pyramid": lambda: vi.pyramid_problem((4, 3, 3), [(0, 2, 0, 3, 0, 3), (2, 1, 0, 4, 0, 3)], jitter=0.2,
                                          seed=5, lam_m="lognormal", ratio=1e4),
    # several thousand cells: many thread blocks and ragged last ones
    "tet_large": lambda: vi.tet_problem((11, 9, 8), [(0, 5, 0, 9, 0, 8), (2, 4, 0, 11, 0, 9)], jitter=0.2,
                                        seed=7, lam_m="lognormal", ratio=1e4),
    "prism_large": lambda: _prisms("checker", (15, 13), 9, seed=4),
}


def oracle_fluxes(pb, ref, cn, sh, ffn):
    """The oracle's F_{K,nu} and F_{sigma,s} in the library's slots, matched
    by node ids (cells), by face node sets (fracture faces of cells) and by
    node ids (fracture faces)."""
    import paper_1602_03641_gb300 as pkg
    nv = pb.n_nodes
    Fcn = np.zeros((pb.n_cells, 8))
    Fcf = np.zeros((pb.n_cells, 6))
    ffkey = {tuple(sorted(int(v) for v in f if v >= 0)): i for i, f in enumerate(pb.ff_nodes)}
    for cm, F in zip(ref.cellmats, ref.F_cell):
        for b, K in enumerate(cm["cells"]):
            slot = {int(d): j for j, d in enumerate(cm["dofs"][b, 1:]) if d >= 0}
            for l in range(8):
                if cn[K, l] >= 0:
                    Fcn[K, l] = F[b, slot[int(cn[K, l])]]
            for lf, face in enumerate(pkg.SHAPE_FACES[int(sh[K])]):
                f = ffkey.get(tuple(sorted(int(cn[K, t]) for t in face)))
                if f is not None:
                    Fcf[K, lf] = F[b, slot[nv + f]]
    Fff = np.zeros((pb.n_ff, 4))
    for i in range(pb.n_ff):
        d = ref.fracmats["dofs"][i, 1:]
        for t in range(4):
            if ffn[i, t] >= 0:
                Fff[i, t] = ref.F_frac[i, int(np.nonzero(d == ffn[i, t])[0][0])]
    return Fcn, Fcf, Fff


@pytest.fixture(scope="module")
def runs(ctx):
    import paper_1602_03641_gb300 as pkg
    out = {}
    for name, mk in CASES.items():
        pb = mk()
        assert not pkg.is_hex_problem(pb)
        ref = vo.DarcyTransport(pb)
        s = pkg.assemble_problem(ctx, pb)
        u, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000, raise_on_error=False)
        out[name] = (pb, ref, s, u, info)
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_numbering_shapes(runs, name):
    import paper_1602_03641_gb300 as pkg
    pb, ref, s, u, info = runs[name]
    cn, sh, ffn = s.export_cells()
    nn = np.array([8, 4, 6, 5])[sh]
    assert np.all((cn >= 0) == (np.arange(8)[None, :] < nn[:, None]))
    for K in range(pb.n_cells):   # the same node set as the input cell
        assert set(cn[K, :nn[K]].tolist()) == set(pb.cell_nodes[K][pb.cell_nodes[K] >= 0].tolist())
    want = {"tet": {1}, "tet_large": {1}, "prism": {2}, "prism_half": {0, 2}, "prism_checker": {0, 2},
            "prism_large": {0, 2}, "pyramid": {3}}[name]
    assert set(np.unique(sh).tolist()) == want
    for i in range(pb.n_ff):
        assert sorted(ffn[i][ffn[i] >= 0].tolist()) == sorted(pb.ff_nodes[i][pb.ff_nodes[i] >= 0].tolist())
    assert pkg.VAG_SHAPE_TET == 1


@pytest.mark.parametrize("name", list(CASES))
def test_eliminated_system_matches(runs, name):
    pb, ref, s, u, info = runs[name]
    S, b, R = vo.schur_system(pb, ref.A)
    e = s.export_system()
    n = len(e["rowptr"]) - 1
    assert n == len(R)
    np.testing.assert_array_equal(e["row_dof"], R)
    G = sp.csr_matrix((e["val"], e["col"], e["rowptr"]), shape=(n, n))
    scale = abs(S).max()
    assert abs(G - S).max() <= 1e-12 * scale
    assert np.abs(e["rhs"] - b).max() <= 1e-12 * max(np.abs(b).max(), scale)


@pytest.mark.parametrize("name", list(CASES))
def test_pressure_and_fluxes_match(runs, name):
    pb, ref, s, u, info = runs[name]
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations, info.ret)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10
    cn, sh, ffn = s.export_cells()
    Fcn, Fcf, Fff = s.export_fluxes()
    On, Of, Off = oracle_fluxes(pb, ref, cn, sh, ffn)
    scale = max(np.abs(On).max(), np.abs(Off).max() if Off.size else 0.0)
    assert np.abs(Fcn - On).max() <= 1e-9 * scale
    assert np.abs(Fcf - Of).max() <= 1e-9 * scale
    if pb.n_ff:
        assert np.abs(Fff - Off).max() <= 1e-9 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_transport_matches(ctx, runs, name):
    """One step from the same state on the oracle's fluxes, porous volumes
    and CFL bound; then ten steps of the whole path on the GPU's own fluxes."""
    import paper_1602_03641_gb300 as pkg
    pb, ref, s, u, info = runs[name]
    cn, sh, ffn = s.export_cells()
    On, Of, Off = oracle_fluxes(pb, ref, cn, sh, ffn)
    s.set_fluxes(On, Of, Off)
    rng = np.random.default_rng(5)
    c = rng.uniform(0, 1, ref.tr.n)
    c[pb.dir_nodes] = pb.cbar
    dt = 0.8 * ref.tr.cfl_dt()
    cg = c.copy()
    inf = s.transport(cg, pb.phi_m, pb.phi_f, pb.cbar, n_steps=1, cfl=0.0, dt=dt)
    assert np.abs(cg - ref.tr.step(c, dt)).max() <= 1e-12
    phi = s.export_porous_volumes()
    assert np.abs(phi - ref.tr.phi).max() <= 1e-13 * ref.tr.phi.max()
    assert inf.dt_max == pytest.approx(ref.tr.cfl_dt(), rel=1e-12)
    s2 = pkg.assemble_problem(ctx, pb)
    s2.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=5000, raise_on_error=False)
    c = pb.c0()
    inf = s2.transport(c, pb.phi_m, pb.phi_f, pb.cbar, n_steps=10, cfl=0.9)
    co, dto = ref.run_transport(10, cfl=0.9)
    assert inf.dt == pytest.approx(dto, rel=1e-9)
    assert np.abs(c - co).max() <= 1e-9
    s2.close()


@pytest.mark.parametrize("name", ["tet", "prism_half", "pyramid"])
def test_mixed_precision_and_classical_amg(ctx, runs, name):
    import paper_1602_03641_gb300 as pkg
    pb, ref, s, u, info = runs[name]
    for prec, pc in ((pkg.VAG_MIXED, pkg.VAG_PC_AMG), (pkg.VAG_MIXED, pkg.VAG_PC_AMG_RS),
                     (pkg.VAG_FP64, pkg.VAG_PC_AMG_RS), (pkg.VAG_FP64_PC32, pkg.VAG_PC_AMG)):
        um, im = s.solve(precision=prec, precond=pc, rtol=1e-12, maxit=5000, raise_on_error=False)
        assert im.rel_residual <= 1e-11, (prec, pc, im.rel_residual)
        assert np.linalg.norm(um - ref.u) / np.linalg.norm(ref.u) <= 1e-10, (prec, pc)


def test_mixed_shapes_batch_equals_alone_bitwise(ctx):
    """A batch of a hexahedral fast-path mesh, a tetrahedral, a mixed
    prism/hexahedral and a pyramidal mesh gives each system bitwise its
    result alone."""
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.config_plain16(6), CASES["tet"](), CASES["prism_half"](), CASES["pyramid"]()]
    arrs = [pkg.problem_arrays(pbs[0])] + [pkg.general_arrays(p) for p in pbs[1:]]
    bs = ctx.assemble_batch(arrs)
    lay = bs.batch_layout()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    nv, nf = ns[-1], fs[-1]
    ub, _ = bs.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=5000, raise_on_error=False)
    cb = np.concatenate([np.concatenate([p.c0()[:p.n_nodes] for p in pbs]),
                         np.concatenate([p.c0()[p.n_nodes:p.n_nodes + p.n_ff] for p in pbs]),
                         np.concatenate([p.c0()[p.n_nodes + p.n_ff:] for p in pbs])])
    bs.transport(cb, np.concatenate([p.phi_m for p in pbs]), np.concatenate([p.phi_f for p in pbs]),
                 np.concatenate([p.cbar for p in pbs]), n_steps=7, cfl=0.9)
    _, shb, _ = bs.export_cells()
    for i, pb in enumerate(pbs):
        s = pkg.assemble_problem(ctx, pb)
        ua, _ = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=5000, raise_on_error=False)
        ca = pb.c0()
        s.transport(ca, pb.phi_m, pb.phi_f, pb.cbar, n_steps=7, cfl=0.9)

        def part(v):
            return np.concatenate([v[ns[i]:ns[i + 1]], v[nv + fs[i]:nv + fs[i + 1]],
                                   v[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        assert np.array_equal(part(ub), ua), i
        assert np.array_equal(part(cb), ca), i
        _, sha, _ = s.export_cells()
        assert np.array_equal(shb[cs[i]:cs[i + 1]], sha), i
        s.close()
    bs.close()


def test_server_takes_general_cells(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = CASES["prism_half"]()
    srv = pkg.Server(0, slots=1)
    t = srv.submit(pb, n_steps=5, precond=pkg.VAG_PC_AMG, rtol=1e-10)
    u1, c1, r1 = srv.wait(t, 60000)
    assert r1.status == pkg.VAG_OK
    s = pkg.assemble_problem(ctx, pb)
    u2, _ = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=20000)
    c2 = pb.c0()
    s.transport(c2, pb.phi_m, pb.phi_f, pb.cbar, n_steps=5, cfl=0.9)
    assert np.array_equal(u1, u2) and np.array_equal(c1, c2)
    srv.close()
    s.close()


def test_bad_general_cells_are_rejected(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = CASES["prism"]()
    q = pkg.general_arrays(pb)
    # drop a prism's last face: four faces (two triangles, two quadrilaterals)
    cptr = q["cell_face_ptr"].copy()
    cidx = np.delete(q["cell_face_idx"], cptr[1] - 1).astype(np.int32)
    cptr[1:] -= 1
    with pytest.raises(pkg.VagError) as e:
        ctx.assemble_general(q["xyz"], q["face_node_ptr"], q["face_node_idx"], cptr, cidx, q["ff_face_ids"],
                             q["lambda_m"], q["lambda_f"], q["d_f"], q["mu"], q["dir_nodes"], q["dir_values"])
    assert e.value.code == pkg.VAG_EMESH
