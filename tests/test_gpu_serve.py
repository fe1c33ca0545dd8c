"""Continuous-batching server: every request's pressures, concentrations and
CFL step are bitwise those of the same problem solved alone, whatever batch
it landed in; admission respects the memory budget; waits are bounded."""
import threading
import time

import numpy as np
import pytest

import vag_inputs as vi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as p
    return p


def problems(k, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(5, 14))
        out.append(vi.random_dfn_problem(n, int(rng.integers(1, 8)), float(10 ** rng.uniform(2, 6)), seed=100 + i))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_results_equal_alone_bitwise(pkg, precision):
    pbs = problems(14)
    srv = pkg.Server(0, slots=2, max_batch=5)
    tickets = []

    def producer():
        for pb in pbs:   # arrivals spread over time: later ones join while earlier batches run
            tickets.append(srv.submit(pb, n_steps=15, precision=precision, rtol=1e-10))
            time.sleep(0.002)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    results = [srv.wait(t, timeout_ms=60000) for t in tickets]
    st = srv.stats()
    assert st.completed == len(pbs) and st.in_queue == 0 and st.in_flight == 0
    assert st.p99_ms >= st.p50_ms > 0
    assert max(r[2].batch_size for r in results) > 1          # batching happened
    ctx = pkg.Context(0)
    for pb, (u, c, r) in zip(pbs, results):
        assert r.status == 0
        s = pkg.assemble_problem(ctx, pb)
        u1, inf1 = s.solve(precision=precision, rtol=1e-10, raise_on_error=False)
        np.testing.assert_array_equal(u, u1)
        assert r.solve.iterations == inf1.iterations
        c1 = pb.c0()
        t1 = s.transport(c1, pb.phi_m, pb.phi_f, pb.cbar, n_steps=15, cfl=0.9)
        assert r.transport.dt == t1.dt
        np.testing.assert_array_equal(c, c1)
        s.close()
    ctx.close()
    srv.close()


def test_budget_admission_and_bounded_wait(pkg):
    pbs = problems(3, seed=3)
    small = pkg.Server(0, budget_bytes=1 << 20, slots=1)
    with pytest.raises(pkg.VagError) as e:
        small.submit(pbs[0], n_steps=5)
    assert e.value.code == pkg.VAG_EBUDGET
    assert small.stats().rejected == 1
    small.close()
    srv = pkg.Server(0, slots=1)
    big = vi.random_dfn_problem(40, 10, 1e4, seed=1)
    t = srv.submit(big, n_steps=50, rtol=1e-10)
    try:
        srv.wait(t, timeout_ms=0)
        finished_early = True
    except pkg.VagError as err:
        assert err.code == pkg.VAG_ETIMEOUT
        finished_early = False
    if not finished_early:
        u, c, r = srv.wait(t, timeout_ms=120000)
        assert r.status == 0
    with pytest.raises(pkg.VagError):
        srv.wait(123456789, timeout_ms=0)                        # unknown ticket
    srv.close()
