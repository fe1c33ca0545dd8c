"""The Chebyshev-Jacobi preconditioner (Sec. 4.2 solve; Chebyshev acceleration
of Jacobi with Lanczos bounds) against the oracle's direct solution, against
Jacobi-CG, alone against in a batch, and its rejected combinations."""
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
    "scale20": lambda: vi.config_scale64(20),
    "dfn12_1e6": lambda: vi.random_dfn_problem(12, 8, 1e6, seed=17),
    "fourfrac20": lambda: vi.four_fracture_problem(20),
    "nofrac_5x4x3": lambda: vi.build_problem((5, 4, 3), [], jitter=0.2, seed=2, lam_m="lognormal"),
    "four_rows": lambda: vi.build_problem((2, 1, 1), []),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("krylov", ["cg", "bicgstab"])
def test_chebyshev_matches_oracle(ctx, name, krylov):
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    s = pkg.assemble_problem(ctx, pb)
    kr = pkg.VAG_KRYLOV_CG if krylov == "cg" else pkg.VAG_KRYLOV_BICGSTAB
    u, info = s.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-12, maxit=20000, raise_on_error=False, krylov=kr)
    # 1e-12 is requested; the FP64 rounding floor of a few cases is near 2e-12
    assert info.rel_residual <= 1e-11, (info.ret, info.iterations, info.rel_residual)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-10, err
    s.close()


def test_chebyshev_cuts_cg_iterations(ctx):
    """A degree-3 polynomial in D^-1 A: CG needs well under half the Jacobi-CG
    iterations (about a quarter when the interval is right)."""
    import paper_1602_03641_gb300 as pkg
    pb = vi.config_scale64(24)
    s = pkg.assemble_problem(ctx, pb)
    _, ij = s.solve(precond=pkg.VAG_PC_JACOBI, rtol=1e-10, maxit=20000)
    _, ic = s.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-10, maxit=20000)
    assert ic.iterations < 0.45 * ij.iterations, (ic.iterations, ij.iterations)
    assert ic.ms_setup > 0.0
    s.close()


def test_chebyshev_batch_equals_alone_bitwise(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(9, 5, 1e3, seed=1), vi.config_plain16(6), vi.build_problem((1, 1, 1), []),
           vi.random_dfn_problem(12, 12, 1e6, seed=2), vi.build_problem((5, 7, 4), [], jitter=0.2, seed=9,
                                                                          lam_m="lognormal")]
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, info = bs.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-12, maxit=20000, raise_on_error=False)
    infos = bs.solve_infos()
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-12, maxit=20000, raise_on_error=False)
        ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
        ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]],
                             ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        assert infos[i].rel_residual == inf1.rel_residual
        ref = vo.DarcyTransport(pb)
        assert np.linalg.norm(u1 - ref.u) <= 1e-10 * np.linalg.norm(ref.u)
        s1.close()
    bs.close()


def test_chebyshev_repeat_is_deterministic(ctx):
    """The second solve reuses the cached CUDA graph with a fresh coefficient
    table; both solves give bitwise the same result."""
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, vi.random_dfn_problem(10, 6, 1e4, seed=5))
    u1, i1 = s.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-11)
    u2, i2 = s.solve(precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-11)
    np.testing.assert_array_equal(u1, u2)
    assert i1.iterations == i2.iterations
    s.close()


def test_chebyshev_rejects_mixed_precision(ctx):
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, vi.config_plain16(4))
    for prec in (pkg.VAG_MIXED, pkg.VAG_MIXED_F16):
        with pytest.raises(pkg.VagError) as e:
            s.solve(precision=prec, precond=pkg.VAG_PC_CHEBYSHEV, rtol=1e-8)
        assert e.value.code == pkg.VAG_EINVAL
    with pytest.raises(pkg.VagError) as e:
        s.solve(precond=7, rtol=1e-8)
    assert e.value.code == pkg.VAG_EINVAL
    s.close()
