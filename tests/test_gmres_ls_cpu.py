"""The small least-squares problem of GMRES (csrc/vag_gmres_ls.h, the code the
GMRES kernels run per system, compiled here with g++): rotating the
Hessenberg columns one at a time and back-substituting must give the
least-squares solution of min ||beta e_1 - H y|| and its residual norm
|g_k|, for every k.  CPU only."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_03641_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "vag_gmres_ls.h"
// input: m beta, then the (m+1) x m Hessenberg matrix by columns (j+2 entries each)
// output per k = 1..m: ok |g_k| y_0..y_{k-1}
int main() {
  int m; double beta;
  if (std::scanf("%d %lf", &m, &beta) != 2) return 1;
  std::vector<double> R(m * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), c(m + 1), y(m);
  g[0] = beta;
  for (int j = 0; j < m; ++j) {
    for (int q = 0; q <= j + 1; ++q) std::scanf("%lf", &c[q]);
    const bool ok = vag::gm_rotate_column(j, c.data(), cs.data(), sn.data(), g.data());
    for (int q = 0; q <= j; ++q) R[j * m + q] = c[q];
    vag::gm_back_substitute(j + 1, R.data(), m, g.data(), y.data());
    std::printf("%d %.17g", ok ? 1 : 0, g[j + 1] < 0 ? -g[j + 1] : g[j + 1]);
    for (int i = 0; i <= j; ++i) std::printf(" %.17g", y[i]);
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "g.cpp")
    out = os.path.join(d, "g")
    open(src, "w").write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, src, "-o", out], check=True)
    return out


def _run(exe, H, beta):
    m = H.shape[1]
    parts = [str(m), f"{beta:.17g}"]
    for j in range(m):
        parts += [f"{v:.17g}" for v in H[:j + 2, j]]
    out = subprocess.run([exe], input=" ".join(parts) + "\n", capture_output=True, text=True, check=True).stdout
    return [list(map(float, line.split())) for line in out.strip().splitlines()]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rotations_and_back_substitution_solve_the_least_squares_problem(exe, seed):
    rng = np.random.default_rng(seed)
    m, beta = 30, 2.5
    H = np.triu(rng.normal(size=(m + 1, m)), -1)
    H[np.arange(1, m + 1), np.arange(m)] = np.abs(H[np.arange(1, m + 1), np.arange(m)]) + 0.1
    rows = _run(exe, H, beta)
    assert len(rows) == m
    for k in range(1, m + 1):
        ok, res, *y = rows[k - 1]
        assert ok == 1
        Hk = H[:k + 1, :k]
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        y_ref, *_ = np.linalg.lstsq(Hk, rhs, rcond=None)
        np.testing.assert_allclose(y, y_ref, rtol=1e-9, atol=1e-12)
        assert res == pytest.approx(np.linalg.norm(rhs - Hk @ y_ref), rel=1e-9, abs=1e-14)


def test_a_column_in_the_span_gives_a_zero_residual(exe):
    """h_{j+1,j} = 0 (the Krylov space holds the solution): the rotated
    residual is exactly zero and y solves H y = beta e_1."""
    H = np.array([[2.0, 1.0], [1.0, 3.0], [0.0, 0.0]])
    rows = _run(exe, H, 1.0)
    ok, res, *y = rows[1]
    assert ok == 1 and res == 0.0
    np.testing.assert_allclose(H[:2] @ np.array(y), [1.0, 0.0], atol=1e-15)


def test_a_zero_column_is_reported(exe):
    H = np.zeros((2, 1))
    rows = _run(exe, H, 1.0)
    assert rows[0][0] == 0
