"""The oracle against the paper's two analytical solutions (Sec. 5.1, 5.2).

First the closed forms are checked against the equations they solve (so a
printing error, such as the sign in the stationary c_{f,3}, cannot hide), then
the oracle's discrete transport is compared with them on refined meshes.
The paper prints no numeric convergence order, only that the errors converge
and that they converge faster in the fractures; the thresholds here encode
that statement (first-order upwind on a discontinuous front: about 1/2).
"""
import numpy as np
import pytest

import vag_inputs as vi
from oracle import analytic as an
from oracle import vag_oracle as vo


def _d(f, x, h=1e-6):
    return (f(x + h) - f(x - h)) / (2 * h)


def test_four_fracture_closed_forms_solve_their_odes():
    s = an.FourFractures()
    x1 = np.linspace(0.01, s.x0 - 0.01, 7)
    # Gamma_1: k1 c' + b1 c = b1 c_m1 = 0
    assert np.abs(s.k1 * _d(s.cf1, x1) + s.b1 * s.cf1(x1)).max() < 1e-6
    # Gamma_4: -k2 c' + b2 c = b2 c_m1 = 0, c(1) = 1
    y4 = np.linspace(s.y0 + 0.01, 0.99, 7)
    assert np.abs(-s.k2 * _d(s.cf4, y4) + s.b2 * s.cf4(y4)).max() < 1e-6
    assert s.cf4(1.0) == pytest.approx(1.0)
    # Gamma_2: k1 c' + b1 c = b1 c_m2(x, line1(x)), c_m2(x, y) = c_f4(y)
    x2 = np.linspace(s.x0 + 0.01, 0.99, 7)
    res2 = s.k1 * _d(s.cf2, x2) + s.b1 * s.cf2(x2) - s.b1 * s.cf4(s.line1_y(x2))
    assert np.abs(res2).max() < 1e-6
    # Gamma_3: -k2 c' + b2 c = b2 c_m3(line2(y), y)
    y3 = np.concatenate([np.linspace(0.01, 0.24, 4), np.linspace(0.26, s.y0 - 0.01, 4)])
    cm3 = np.where(y3 > 0.25, s.cf1((y3 - 0.25) / s.tan1), 0.0)
    res3 = -s.k2 * _d(s.cf3, y3) + s.b2 * s.cf3(y3) - s.b2 * cm3
    assert np.abs(res3).max() < 1e-6
    # intersection: continuity and flux mixing
    assert s.cf2(s.x0) == pytest.approx(s.c0)
    assert s.cf3(s.y0) == pytest.approx(s.c0)
    assert (s.r + 1) * s.c0 - s.cf1(s.x0) - s.r * s.cf4(s.y0) == pytest.approx(0.0, abs=1e-14)
    # the intersection point lies on both lines
    assert s.line1_y(s.x0) == pytest.approx(s.y0)
    assert s.line2_x(s.y0) == pytest.approx(s.x0)


def test_one_fracture_closed_form_solves_its_pde():
    s = an.OneFracture()
    for x, t in [(0.3, 0.2), (0.6, 0.3), (0.8, 0.5), (0.45, 0.1)]:
        assert x / s.k < t < x
        ct = (s.c_f(np.array([x]), t + 1e-6) - s.c_f(np.array([x]), t - 1e-6))[0] / 2e-6
        cx = (s.c_f(np.array([x + 1e-6]), t) - s.c_f(np.array([x - 1e-6]), t))[0] / 2e-6
        c = s.c_f(np.array([x]), t)[0]
        cm1 = 0.0   # t < x: the matrix front has not arrived above the fracture
        assert ct + s.k * cx + s.beta * c - s.beta * cm1 == pytest.approx(0.0, abs=1e-6)


def _l1(pb, mesh, tr, c, cm_fun, cf_fun):
    nv, nf = pb.n_nodes, pb.n_ff
    vol = tr.vol
    ck = c[nv + nf:]
    ex_k = cm_fun(mesh.xK[:, 0], mesh.xK[:, 1])
    em = np.sum(vol * np.abs(ck - ex_k)) / np.sum(vol * np.abs(ex_k))
    xs = mesh.xS[pb.ff_faces]
    area = vo.fracture_local_matrices(pb, mesh)["area"]
    ex_f = cf_fun(xs)
    ef = np.sum(area * np.abs(c[nv:nv + nf] - ex_f)) / np.sum(area * np.abs(ex_f))
    return em, ef


def test_one_fracture_transport_converges():
    s = an.OneFracture()
    tf = 0.5
    errs = []
    ns = [16, 32, 64]
    for n in ns:
        pb = vi.one_fracture_problem(n)
        d = vo.DarcyTransport(pb)
        # Darcy part: u = 1 - x exactly
        assert np.abs(d.u[:pb.n_nodes] - (1 - pb.xyz[:, 0])).max() < 1e-10
        c, dt, N = d.run_to_time(tf)
        errs.append(_l1(pb, d.mesh, d.tr, c, lambda x, y: s.c_m(x, y, tf),
                        lambda xs: s.c_f(xs[:, 0], tf)))
    em = np.array([e[0] for e in errs]); ef = np.array([e[1] for e in errs])
    assert np.all(np.diff(em) < 0) and np.all(np.diff(ef) < 0)
    pm = -np.polyfit(np.log(ns), np.log(em), 1)[0]
    pf = -np.polyfit(np.log(ns), np.log(ef), 1)[0]
    assert pm > 0.4, (em, pm)
    assert pf > 0.6, (ef, pf)
    assert ef[-1] < em[-1]


def test_four_fracture_stationary_converges():
    s = an.FourFractures()
    ns = [16, 32, 64]
    errs = []
    for n in ns:
        pb = vi.four_fracture_problem(n)
        d = vo.DarcyTransport(pb)
        assert np.abs(d.u[:pb.n_nodes] - (1 - pb.xyz[:, 0])).max() < 1e-10
        c = vo.stationary_concentration(d.tr)
        ff = pb.ff_frac

        def cf(xs):
            out = np.empty(xs.shape[0])
            for k, fun in enumerate([lambda p: s.cf1(p[:, 0]), lambda p: s.cf2(p[:, 0]),
                                     lambda p: s.cf3(p[:, 1]), lambda p: s.cf4(p[:, 1])]):
                sel = ff == k
                out[sel] = fun(xs[sel])
            return out
        errs.append(_l1(pb, d.mesh, d.tr, c, s.c_m, cf))
    em = np.array([e[0] for e in errs]); ef = np.array([e[1] for e in errs])
    assert np.all(np.diff(em) < 0) and np.all(np.diff(ef) < 0)
    pf = -np.polyfit(np.log(ns), np.log(ef), 1)[0]
    pm = -np.polyfit(np.log(ns), np.log(em), 1)[0]
    assert pm > 0.4, (em, pm)
    assert pf > 0.6, (ef, pf)
