"""BiCGStab (right-preconditioned, the Krylov method of the paper's solver
experiments, §5.3) on the GPU: the same pressures as the oracle with the
Jacobi and the AMG preconditioner, FP64 and with the FP32 hierarchy, and a
system's result bitwise the same alone or in a batch."""
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


CASES = {
    "plain16": lambda: vi.config_plain16(16),
    "dfn14_1e5": lambda: vi.random_dfn_problem(14, 9, 1e5, seed=21),
    "fourfrac20": lambda: vi.four_fracture_problem(20),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", ["fp64_jacobi", "fp64_amg", "mixed_amg"])
def test_bicgstab_matches_oracle(ctx, name, variant):
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    s = pkg.assemble_problem(ctx, pb)
    prec = pkg.VAG_MIXED if variant.startswith("mixed") else pkg.VAG_FP64
    pc = pkg.VAG_PC_AMG if variant.endswith("amg") else pkg.VAG_PC_JACOBI
    u, info = s.solve(precision=prec, precond=pc, rtol=1e-12, maxit=20000, raise_on_error=False,
                      krylov=pkg.VAG_KRYLOV_BICGSTAB)
    # the true residual (recomputed in FP64) reaches the CG bar
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations, info.status)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-10, err
    _, icg = s.solve(precision=prec, precond=pc, rtol=1e-12, maxit=20000, raise_on_error=False)
    # one BiCGStab iteration applies A and M twice: it needs fewer iterations than CG
    assert info.iterations <= icg.iterations + 5, (info.iterations, icg.iterations)
    s.close()


def test_bicgstab_batch_equals_alone_bitwise(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(10, 6, 1e3, seed=1), vi.config_plain16(8), vi.build_problem((1, 1, 1), []),
           vi.random_dfn_problem(12, 9, 1e6, seed=2)]
    for pc in (pkg.VAG_PC_JACOBI, pkg.VAG_PC_AMG):
        bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
        lay = bs.batch_layout()
        nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
        ub, _ = bs.solve(precond=pc, rtol=1e-10, maxit=5000, raise_on_error=False, krylov=pkg.VAG_KRYLOV_BICGSTAB)
        infos = bs.solve_infos()
        ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
        for i, pb in enumerate(pbs):
            s1 = pkg.assemble_problem(ctx, pb)
            u1, inf1 = s1.solve(precond=pc, rtol=1e-10, maxit=5000, raise_on_error=False,
                                krylov=pkg.VAG_KRYLOV_BICGSTAB)
            ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]],
                                 ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
            np.testing.assert_array_equal(ui, u1)
            assert infos[i].iterations == inf1.iterations
            assert inf1.rel_residual <= 1e-10, (pc, i, inf1.rel_residual, inf1.status)
            s1.close()
        bs.close()


def test_bicgstab_rejects_mixed_jacobi(ctx):
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, vi.config_plain16(6))
    _, info = s.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_JACOBI, raise_on_error=False,
                      krylov=pkg.VAG_KRYLOV_BICGSTAB)
    assert info.ret == pkg.VAG_EINVAL
    s.close()
