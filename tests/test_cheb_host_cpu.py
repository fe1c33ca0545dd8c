"""Arithmetic of the Chebyshev-Jacobi preconditioner (csrc/vag_cheb_host.h,
compiled here with g++): the Sturm-bisection top eigenvalue of a tridiagonal
matrix, the interval from CG's Lanczos coefficients, and the recurrence table
applied by the kernel's own per-row step (cheb_row_step) to a scalar, which
must give the residual polynomial T_k((theta - l)/delta) / T_k(theta/delta).
CPU only."""
import os
import subprocess
import tempfile

import numpy as np
import pytest


def _f(v):
    return f"{float(v):.17g}"


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_03641_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "vag_cheb_host.h"
int main() {
  char op[16];
  while (std::scanf("%15s", op) == 1) {
    if (op[0] == 'T') {                 // T m a_0..a_{m-1} e_0..e_{m-2}
      int m; std::scanf("%d", &m);
      std::vector<double> a(m), e(m > 1 ? m - 1 : 0);
      for (auto &v : a) std::scanf("%lf", &v);
      for (auto &v : e) std::scanf("%lf", &v);
      std::printf("%.17g\n", vag::tridiag_max_eig(a, e));
    } else if (op[0] == 'B') {          // B m safety alpha_0.. beta_0..
      int m; double sf; std::scanf("%d %lf", &m, &sf);
      std::vector<double> al(m > 0 ? m : 1), be(m > 0 ? m : 1);
      for (int j = 0; j < m; ++j) std::scanf("%lf", &al[j]);
      for (int j = 0; j < m; ++j) std::scanf("%lf", &be[j]);
      std::printf("%.17g\n", vag::cheb_upper_bound(al.data(), be.data(), m, sf));
    } else {                            // P a b degree lambda: p(lambda) by the kernel's steps
      double a, b, lam; int k; std::scanf("%lf %lf %d %lf", &a, &b, &k, &lam);
      std::vector<double> c(2 * k);
      vag::cheb_table(a, b, k, c.data());
      const double r = 1.0, w = r;      // D = 1: w = D^-1 r
      double d = 0.0, z = 0.0;
      for (int j = 1; j < k; ++j) {      // the kernel's per-row step, A = lambda
        const double din = j == 1 ? w : d, zin = j == 1 ? w : z;
        vag::cheb_row_step(c.data(), j, r, lam * zin, 1.0, din, zin, &d, &z);
      }
      if (k == 1) z = c[0] * w;
      std::printf("%.17g\n", z);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def run():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    open(src, "w").write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)

    def call(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return np.array([float(x) for x in out.stdout.split()])
    return call


def test_tridiagonal_top_eigenvalue(run):
    rng = np.random.default_rng(3)
    lines, ref = [], []
    for m in range(1, 13):
        a = rng.uniform(0.5, 3.0, m)
        e = rng.normal(0.0, 1.0, m - 1)
        T = np.diag(a) + np.diag(e, 1) + np.diag(e, -1)
        lines.append(" ".join(["T", str(m)] + [_f(v) for v in a] + [_f(v) for v in e]))
        ref.append(np.linalg.eigvalsh(T).max())
    got = run(lines)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_interval_from_cg_coefficients(run):
    """The Lanczos tridiagonal of m Jacobi-CG steps: its top Ritz value lies
    below lambda_max(D^-1 A) and, after the full n steps, equals it."""
    rng = np.random.default_rng(5)
    n = 9
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    dinv = 1.0 / np.diag(A)
    lam_max = np.linalg.eigvals(dinv[:, None] * A).real.max()
    b = rng.uniform(-1, 1, n)
    x = np.zeros(n); r = b.copy(); z = dinv * r; p = z.copy(); rz = r @ z
    al, be = [], []
    for _ in range(n):
        q = A @ p; a = rz / (p @ q); x += a * p; r -= a * q; z = dinv * r
        rzn = r @ z; be.append(rzn / rz); rz = rzn; p = z + be[-1] * p; al.append(a)
    lines = []
    for m in (3, n):
        lines.append(" ".join(["B", str(m), "1.0"] + [_f(v) for v in al[:m]] + [_f(v) for v in be[:m]]))
    lines.append("B 0 1.2")
    lines.append(" ".join(["B", "2", "1.2"] + [_f(v) for v in al[:2]] + [_f(v) for v in be[:2]]))
    got = run(lines)
    assert got[0] <= lam_max * (1 + 1e-12)
    assert got[1] == pytest.approx(lam_max, rel=1e-9)
    assert got[2] == 2.0
    # the safety factor scales the Ritz value
    d = [1 / al[0], 1 / al[1] + be[0] / al[0]]
    T = np.array([[d[0], np.sqrt(be[0]) / al[0]], [np.sqrt(be[0]) / al[0], d[1]]])
    assert got[3] == pytest.approx(1.2 * np.linalg.eigvalsh(T).max(), rel=1e-12)


def _cheb_T(k, x):
    x = np.asarray(x, float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(k * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** k * np.cosh(k * np.arccosh(np.abs(xo)))
    return out


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_recurrence_gives_the_chebyshev_residual_polynomial(run, k):
    a, b = 0.03, 3.1
    theta, delta = (b + a) / 2, (b - a) / 2
    lams = np.concatenate([np.linspace(1e-3, (b + a) * (1 - 1e-6), 41), [a, b]])   # 0 < l < b + a
    got = run([f"P {_f(a)} {_f(b)} {k} {_f(l)}" for l in lams])
    resid = 1.0 - lams * got
    expect = _cheb_T(k, (theta - lams) / delta) / _cheb_T(k, np.array([theta / delta]))[0]
    np.testing.assert_allclose(resid, expect, atol=1e-12)
    # positive definite below b + a: p(l) > 0 there
    assert np.all(got > 0)
