"""The two forms of the mesh at the C ABI (Sec. 3.1): the general polyhedral
descriptor (faces as cyclic node lists, cells as face lists, fracture faces
as face ids) and the hexahedral fast path give bitwise the same eliminated
system and solution for the same hexahedral mesh, from host or device arrays,
alone, in a batch and through the server, whatever the order of the cells'
faces and of the non-fracture faces' nodes; a cell that is not a hexahedron
is VAG_EMESH and an id out of range VAG_EINVAL."""
import numpy as np
import pytest

import vag_inputs as vi

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


def _assemble_general(ctx, q):
    return ctx.assemble_general(q["xyz"], q["face_node_ptr"], q["face_node_idx"], q["cell_face_ptr"],
                                q["cell_face_idx"], q["ff_face_ids"], q["lambda_m"], q["lambda_f"], q["d_f"], q["mu"],
                                q["dir_nodes"], q["dir_values"])


def _same_system(a, b):
    ea, eb = a.export_system(), b.export_system()
    for k in ("rowptr", "col", "val", "rhs", "row_dof"):
        assert np.array_equal(ea[k], eb[k]), k


@pytest.mark.parametrize("device", [False, True])
def test_both_descriptors_give_the_same_system(ctx, device):
    import paper_1602_03641_gb300 as pkg
    pb = vi.random_dfn_problem(12, 9, 1e4, seed=41)
    s_hex = pkg.assemble_problem(ctx, pb, device=device)
    s_gen = _assemble_general(ctx, pkg.general_arrays(pb, device=device))
    _same_system(s_hex, s_gen)
    u1, i1 = s_hex.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000)
    u2, i2 = s_gen.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000)
    assert np.array_equal(u1, u2) and i1.iterations == i2.iterations
    s_hex.close()
    s_gen.close()


def test_face_and_node_order_do_not_matter(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = vi.random_dfn_problem(9, 6, 1e3, seed=7)
    q = pkg.general_arrays(pb)
    rng = np.random.default_rng(2)
    faces = q["face_node_idx"].reshape(-1, 4).copy()
    isff = np.zeros(len(faces), bool)
    isff[pb.ff_faces] = True
    for f in np.nonzero(~isff)[0]:   # fracture faces keep their cycle: it orders their triangles
        k = int(rng.integers(0, 4))
        faces[f] = np.roll(faces[f], k)[::(-1 if rng.random() < 0.5 else 1)]
    q["face_node_idx"] = np.ascontiguousarray(faces.ravel())
    cf = q["cell_face_idx"].reshape(-1, 6).copy()
    for K in range(len(cf)):
        cf[K] = rng.permutation(cf[K])
    q["cell_face_idx"] = np.ascontiguousarray(cf.ravel())
    s_hex = pkg.assemble_problem(ctx, pb)
    s_gen = _assemble_general(ctx, q)
    _same_system(s_hex, s_gen)
    s_hex.close()
    s_gen.close()


def test_batch_and_server_take_the_general_descriptor(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(8, 4, 1e3, seed=1), vi.config_plain16(6), vi.random_dfn_problem(7, 3, 1e5, seed=2)]
    b_hex = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    b_gen = ctx.assemble_batch([pkg.general_arrays(p) if i != 1 else pkg.problem_arrays(p)
                                for i, p in enumerate(pbs)])
    _same_system(b_hex, b_gen)
    b_hex.close()
    b_gen.close()
    srv = pkg.Server(0, budget_bytes=2 * 2**30, slots=1, max_batch=4)
    t1 = srv.submit(pbs[0], n_steps=5, precond=pkg.VAG_PC_AMG, rtol=1e-10)
    t2 = srv.submit(pbs[0], n_steps=5, precond=pkg.VAG_PC_AMG, rtol=1e-10, general=True)
    u1, c1, r1 = srv.wait(t1, 60000)
    u2, c2, r2 = srv.wait(t2, 60000)
    assert r1.status == pkg.VAG_OK and r2.status == pkg.VAG_OK
    assert np.array_equal(u1, u2) and np.array_equal(c1, c2)
    srv.close()


def test_non_hexahedra_and_bad_ids(ctx):
    import paper_1602_03641_gb300 as pkg
    pb = vi.config_plain16(4)
    q = pkg.general_arrays(pb)
    # split nothing, but give the first cell only five of its faces
    cf = q["cell_face_idx"].reshape(-1, 6)
    cptr = np.concatenate([[0], 5 + 6 * np.arange(len(cf), dtype=np.int32)]).astype(np.int32)
    cidx = np.concatenate([cf[0, :5], cf[1:].ravel()]).astype(np.int32)
    bad = dict(q, cell_face_ptr=cptr, cell_face_idx=cidx)
    with pytest.raises(pkg.VagError) as e:
        _assemble_general(ctx, bad)
    assert e.value.code == pkg.VAG_EMESH
    # a face id out of range
    cidx2 = q["cell_face_idx"].copy()
    cidx2[3] = len(q["face_node_ptr"]) + 5
    with pytest.raises(pkg.VagError) as e:
        _assemble_general(ctx, dict(q, cell_face_idx=cidx2))
    assert e.value.code == pkg.VAG_EINVAL
    # a triangular fracture face
    fptr = q["face_node_ptr"].copy()
    fidx = q["face_node_idx"].copy()
    f = int(q["ff_face_ids"][0])
    tri = np.concatenate([fidx[:fptr[f] + 3], fidx[fptr[f] + 4:]]).astype(np.int32)
    fptr2 = fptr.copy()
    fptr2[f + 1:] -= 1
    with pytest.raises(pkg.VagError) as e:
        _assemble_general(ctx, dict(q, face_node_ptr=fptr2, face_node_idx=tri))
    assert e.value.code == pkg.VAG_EMESH
