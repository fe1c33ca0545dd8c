"""vag_spmv_dot_noalloc: the allocation-free SpMV + dot entry point.

It exists for callers that cannot call cudaMalloc where they need the
product (inside their own stream capture, allocation-free serving threads,
memory reserved by another runtime): its scratch is a fixed file-scope device
array instead of an allocation.  This test calls it through the C ABI on an
eliminated VAG system and compares its output with the existing vag_spmv
entry point and with scipy's product on the exported CSR, on two calls in a
row (the shared scratch must not leak state from one call into the next).
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sps

import vag_inputs as vi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as ge
    ge.build()
    import paper_1602_03641_gb300 as pkg
    L = pkg.lib()
    L.vag_spmv_dot_noalloc.restype = C.c_int
    L.vag_spmv_dot_noalloc.argtypes = [C.c_int32] + [C.c_void_p] * 7
    ctx = pkg.Context(0)
    pb = vi.random_dfn_problem(14, 8, 1e5, seed=23)
    sysg = pkg.assemble_problem(ctx, pb)
    e = sysg.export_system()
    yield pkg, L, ctx, sysg, e
    sysg.close()
    ctx.close()


def test_matches_vag_spmv_on_two_calls_in_a_row(setup):
    pkg, L, ctx, sysg, e = setup
    n = len(e["rowptr"]) - 1
    dev = torch.device("cuda", 0)
    rowptr = torch.from_numpy(e["rowptr"]).to(dev)
    col = torch.from_numpy(e["col"]).to(dev)
    val = torch.from_numpy(e["val"]).to(dev)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(3)
    scale = np.abs(e["val"]).max()
    for call in range(2):
        xh = rng.normal(size=n)
        x = torch.from_numpy(xh).to(dev)
        y = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
        dot = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        st = L.vag_spmv_dot_noalloc(n, rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(),
                                    y.data_ptr(), dot.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert st == pkg.VAG_OK
        stream.synchronize()
        yref = sysg.spmv(xh)                       # the existing entry point
        yg = y.cpu().numpy()
        tol = 1e-12 * scale * np.abs(xh).max() * 30
        assert np.abs(yg - yref).max() <= tol, call
        # and, independently of the library, scipy's product on the exported CSR
        ysp = sps.csr_matrix((e["val"], e["col"], e["rowptr"]), shape=(n, n)) @ xh
        assert np.abs(yg - ysp).max() <= tol, call
        dref = float(np.dot(xh, yref))
        assert abs(dot.item() - dref) <= 1e-12 * np.abs(xh).dot(np.abs(yref)) + tol, call


def test_rejects_sizes_beyond_the_static_limit(setup):
    pkg, L, ctx, sysg, e = setup
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    assert L.vag_spmv_dot_noalloc((1 << 22) + 1, p, p, p, p, p, p, None) == pkg.VAG_EINVAL
    assert L.vag_spmv_dot_noalloc(-1, p, p, p, p, p, p, None) == pkg.VAG_EINVAL
    # the output may not overlap the input vector
    assert L.vag_spmv_dot_noalloc(2, p, p, p, p, p + 8, p, None) == pkg.VAG_EINVAL
