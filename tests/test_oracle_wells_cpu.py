"""Peaceman wells of Sec. 5.5 in the oracle.

* The cell diagonal of the VAG scheme on a box dx x d_f x dz with unit
  permeability is the paper's C = 4/3 (dx dz/d_f + dx d_f/dz + dz d_f/dx)
  (the step of Sec. 5.5 from which r_0 follows).
* Solving that box with the scheme (the well's radial pressure at the eight
  corners, its rate at the centre) gives the closed-form well index.
* With wells alone fixing the pressure, production equals injection, and
  the transport conserves mass with the wells' inflow and outflow and stays
  in [0, 1].  CPU only."""
import copy

import numpy as np
import pytest

import vag_inputs as vi
from oracle import vag_oracle as vo


def _box(dx, dy, dz, lam=1.0):
    pb = vi.build_problem((1, 1, 1), [])
    pb.xyz = pb.xyz * np.array([dx, dy, dz])
    pb.lambda_m = np.array([[lam, lam, lam, 0.0, 0.0, 0.0]])
    return pb


@pytest.mark.parametrize("dims", [(2.0, 0.5, 3.0), (1.0, 1.0, 1.0), (10.0, 0.01, 5.0), (44.0, 1.0, 10.0)])
def test_box_cell_diagonal_is_C(dims):
    dx, df, dz = dims
    cm = vo.cell_local_matrices(_box(dx, df, dz))
    C = 4.0 / 3.0 * (dx * dz / df + dx * df / dz + dz * df / dx)
    assert cm["M"][0, 0, 0] == pytest.approx(C, rel=1e-13)


@pytest.mark.parametrize("dims", [(44.0, 1.0, 10.0), (3.5, 1.0, 10.4), (20.0, 0.5, 2.0)])
def test_well_index_from_the_scheme_on_the_box(dims):
    """Sec. 5.5's construction done with the scheme: the box centred on the
    well axis, the analytic injection pressure p(r) = p_w - q/(2 pi Lam)
    log(r / r_w) at the corners (all at r = D), the rate q dz put into the
    cell; then WI = q dz / (p_w - p_c)."""
    dx, df, dz = dims
    lam, r_w, pw, q = 1e-11 / 1e-3, 0.1, 3.0e6, 0.02
    pb = _box(dx, df, dz, lam)
    pb.xyz = pb.xyz - np.array([dx / 2, df / 2, 0.0])
    A = vo.assemble_full(pb)
    r = np.hypot(pb.xyz[:, 0], pb.xyz[:, 1])
    p_corner = pw - q / (2 * np.pi * lam) * np.log(r / r_w)
    nv = pb.n_nodes
    # cell equation: A_KK p_c + sum_s A_Ks p_s = q dz
    row = A[nv].toarray().ravel()
    p_c = (q * dz - row[:nv] @ p_corner) / row[nv]
    wi_scheme = q * dz / (pw - p_c)
    wi = vo.peaceman_wi(dx, dz, df, 1e-11, r_w, mu=1e-3)
    assert wi_scheme == pytest.approx(wi, rel=1e-12)


@pytest.fixture(scope="module")
def wells_case():
    pb = vi.well_problem((9, 6), 4, jitter=0.15, seed=2)
    g = pb.meta["well_geometry"]
    pb.wells = vi.well_arrays(pb, vo.peaceman_wi(g["dx"], g["dz"], g["d_f"], g["lam_f"], g["r_w"], mu=pb.mu))
    return pb, vo.DarcyTransport(pb)


def test_production_equals_injection(wells_case):
    pb, d = wells_case
    q = d.q_well
    inj = -q[q < 0].sum()
    assert inj == pytest.approx(sum(w["rate"] for w in pb.meta["wells"]), rel=1e-13)
    assert abs(q.sum()) <= 1e-10 * inj
    assert np.all(q[pb.wells["wi"] > 0] > 0)          # the producers produce
    # the conservation equations hold with the well terms
    wd, g = vo.well_terms(pb)
    r = d.A @ d.u + wd * d.u - g
    assert np.abs(r).max() <= 1e-9 * np.abs(g).max()


def test_well_transport_mass_balance_and_bounds(wells_case):
    pb, d = wells_case
    tr = d.tr
    dt = 0.9 * tr.cfl_dt()
    c = pb.c0()
    inflow = 0.0
    for _ in range(40):
        m0 = float(np.sum(tr.phi * c))
        gain = dt * tr.boundary_inflow(c)
        inflow += gain
        c = tr.step(c, dt)
        m1 = float(np.sum(tr.phi * c))
        assert abs(m1 - (m0 + gain)) <= 1e-12 * max(m1, 1e-300) + 1e-15
    assert c.min() >= -1e-12 and c.max() <= 1 + 1e-12
    assert inflow > 0


def test_a_dropped_well_term_fails_the_balance(wells_case):
    """The balance above detects a well left out of the transport."""
    pb, d = wells_case
    tr = copy.copy(d.tr)
    tr.w_F = tr.w_F.copy()
    tr.w_F[0] = 0.0
    dt = 0.9 * d.tr.cfl_dt()
    c = pb.c0()
    m0 = float(np.sum(tr.phi * c))
    gain = dt * d.tr.boundary_inflow(c)
    c = tr.step(c, dt)
    assert abs(float(np.sum(tr.phi * c)) - (m0 + gain)) > 1e-6 * abs(gain)
