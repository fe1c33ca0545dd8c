"""Aggregation-AMG preconditioned CG on the GPU: the same pressures as the
oracle, far fewer iterations than Jacobi, robustness in the fracture/matrix
permeability ratio (the regime where the paper's aggregation AMG stopped
converging, Table solver_cpg_perm), and a hierarchy that depends on each
system alone (bitwise the same result alone or in a batch)."""
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
    "scale_14x11x12": lambda: vi.build_problem(
        (14, 11, 12), [(0, 7, 0, 11, 0, 12), (1, 5, 0, 14, 0, 12), (2, 6, 0, 14, 0, 11), (0, 3, 0, 5, 0, 12)],
        jitter=0.2, seed=3, lam_m="lognormal", ratio=1e4),
    "dfn16_1e6": lambda: vi.random_dfn_problem(16, 12, 1e6, seed=31),
    "fourfrac24": lambda: vi.four_fracture_problem(24),
    "nofrac": lambda: vi.build_problem((9, 7, 8), [], jitter=0.2, seed=2, lam_m="lognormal"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_amg_pcg_matches_oracle(ctx, name):
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000, raise_on_error=False)
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations, info.ret)
    err = np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u)
    assert err <= 1e-10, err
    _, ij = s.solve(precond=pkg.VAG_PC_JACOBI, rtol=1e-12, maxit=20000, raise_on_error=False)
    if name != "plain16":   # plain16 is effectively one-dimensional: Jacobi-CG needs only ~25 iterations
        assert info.iterations * 3 < ij.iterations, (info.iterations, ij.iterations)
    assert info.iterations <= 80
    assert info.ms_setup > 0.0


def test_amg_iterations_do_not_grow_with_the_ratio(ctx):
    import paper_1602_03641_gb300 as pkg
    its = []
    for ratio in (1e2, 1e4, 1e6):
        pb = vi.random_dfn_problem(20, 15, ratio, seed=5)
        s = pkg.assemble_problem(ctx, pb)
        _, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000)
        its.append(info.iterations)
        s.close()
    assert max(its) <= 80, its
    assert max(its) <= 2 * min(its) + 10, its


def test_amg_batch_equals_alone_bitwise(ctx):
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(10, 6, 1e3, seed=1), vi.config_plain16(8), vi.build_problem((1, 1, 1), []),
           vi.random_dfn_problem(13, 9, 1e6, seed=2), vi.build_problem((6, 5, 7), [], jitter=0.2, seed=9,
                                                                       lam_m="lognormal")]
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, _ = bs.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
    infos = bs.solve_infos()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
        ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]], ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        s1.close()


@pytest.mark.parametrize("name", ["scale_14x11x12", "dfn16_1e6", "fourfrac24"])
def test_fp32_hierarchy_preconditions_fp64_cg(ctx, name):
    """VAG_MIXED + AMG: FP64 CG (FP64 residuals and iterates) preconditioned by
    the FP32 copy of the hierarchy reaches the FP64 accuracy."""
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000, raise_on_error=False)
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10
    _, i64 = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000, raise_on_error=False)
    assert info.iterations <= i64.iterations + 10


def test_fp32_hierarchy_batch_equals_alone_bitwise(ctx):
    """The FP32 V-cycle (grid kernels on the big levels, one-kernel tail on
    the small ones) keeps a system's result independent of its batch."""
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(18, 9, 1e5, seed=11), vi.config_plain16(6), vi.random_dfn_problem(11, 4, 1e3, seed=12),
           vi.build_problem((1, 1, 1), [])]
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, _ = bs.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
    infos = bs.solve_infos()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000,
                            raise_on_error=False)
        ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]], ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        assert inf1.rel_residual <= 1e-10
        s1.close()


@pytest.mark.parametrize("index", [252, 144])
def test_amg_on_rows_where_damped_jacobi_diverges(ctx, index):
    """Realisations of the 256-system batch (seed 99) whose eliminated matrix
    has lambda_max(D^-1 A) > 3: a damped-Jacobi smoother with omega = 2/3 is
    not convergent there, the V-cycle is indefinite and CG breaks down.  The
    l1-Jacobi smoother keeps the preconditioner positive definite."""
    import paper_1602_03641_gb300 as pkg
    pb = vi.random_dfn_problem(*vi.batch_params(256, seed=99)[index])
    s = pkg.assemble_problem(ctx, pb)
    for prec in (pkg.VAG_FP64, pkg.VAG_MIXED):
        _, info = s.solve(precision=prec, precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
        assert info.status == pkg.VAG_OK and info.rel_residual <= 1e-10, (prec, info.status, info.rel_residual)
        assert info.iterations <= 80, info.iterations
    if index == 252:
        u, info = s.solve(precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000, raise_on_error=False)
        assert info.rel_residual <= 1e-11, (info.status, info.rel_residual)
        ref = vo.DarcyTransport(pb)
        assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10


@pytest.mark.parametrize("name", ["scale_14x11x12", "dfn16_1e6", "fourfrac24"])
def test_fp16_finest_level_preconditions_fp64_cg(ctx, name):
    """VAG_MIXED_F16: the V-cycle's finest level in FP16 after symmetric
    diagonal scaling, inside FP64 CG: FP64 accuracy, a few more iterations at
    most."""
    import paper_1602_03641_gb300 as pkg
    pb = CASES[name]()
    ref = vo.DarcyTransport(pb)
    s = pkg.assemble_problem(ctx, pb)
    u, info = s.solve(precision=pkg.VAG_MIXED_F16, precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000,
                      raise_on_error=False)
    assert info.rel_residual <= 1e-11, (info.rel_residual, info.iterations)
    assert np.linalg.norm(u - ref.u) / np.linalg.norm(ref.u) <= 1e-10
    _, i32 = s.solve(precision=pkg.VAG_MIXED, precond=pkg.VAG_PC_AMG, rtol=1e-12, maxit=2000, raise_on_error=False)
    assert info.iterations <= i32.iterations + 20, (info.iterations, i32.iterations)
    s.close()


def test_fp16_finest_level_batch_equals_alone_bitwise(ctx):
    """Including a system solved densely on its finest level (one cell)."""
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(14, 7, 1e4, seed=13), vi.build_problem((1, 1, 1), []), vi.config_plain16(7)]
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, _ = bs.solve(precision=pkg.VAG_MIXED_F16, precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000,
                     raise_on_error=False)
    infos = bs.solve_infos()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    for i, pb in enumerate(pbs):
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precision=pkg.VAG_MIXED_F16, precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000,
                            raise_on_error=False)
        ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]], ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        assert inf1.rel_residual <= 1e-10
        s1.close()
    bs.close()


def test_fp16_needs_amg(ctx):
    import paper_1602_03641_gb300 as pkg
    s = pkg.assemble_problem(ctx, vi.config_plain16(6))
    _, info = s.solve(precision=pkg.VAG_MIXED_F16, precond=pkg.VAG_PC_JACOBI, raise_on_error=False)
    assert info.ret == pkg.VAG_EINVAL
    s.close()


def test_fp64_amg_batch24_equals_alone_bitwise(ctx):
    """A batch of 24 realisations with 3 to 7 fractures and ratios 1e2 to 1e6
    under the FP64 AMG V-cycle: each sampled system bitwise the same alone and
    in the batch (its hierarchy, smoother and reductions depend on the system
    alone), and within the oracle's tolerance."""
    import paper_1602_03641_gb300 as pkg
    pbs = [vi.random_dfn_problem(10 + (i % 6) * 2, 3 + i % 5, 10.0 ** (2 + i % 5), seed=40 + i) for i in range(24)]
    bs = ctx.assemble_batch([pkg.problem_arrays(p) for p in pbs])
    lay = bs.batch_layout()
    nv, nf = lay["node_start"][-1], lay["ff_start"][-1]
    ub, _ = bs.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
    infos = bs.solve_infos()
    ns, fs, cs = lay["node_start"], lay["ff_start"], lay["cell_start"]
    for i in (5, 11, 17, 23):
        pb = pbs[i]
        s1 = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s1.solve(precond=pkg.VAG_PC_AMG, rtol=1e-10, maxit=2000, raise_on_error=False)
        ui = np.concatenate([ub[ns[i]:ns[i + 1]], ub[nv + fs[i]:nv + fs[i + 1]], ub[nv + nf + cs[i]:nv + nf + cs[i + 1]]])
        np.testing.assert_array_equal(ui, u1)
        assert infos[i].iterations == inf1.iterations
        assert inf1.rel_residual <= 1e-10
        ref = vo.DarcyTransport(pb)
        assert np.linalg.norm(u1 - ref.u) <= 1e-8 * np.linalg.norm(ref.u)
        s1.close()
    bs.close()
