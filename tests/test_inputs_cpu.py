"""The seeded input generators produce the workloads they describe: sizes,
jitter bounds, frozen fracture-normal coordinates, permeability fields,
boundary data and the batch recipe; and they are reproducible.  CPU only."""
import numpy as np

import vag_inputs as vi


def _sym(l6):
    return np.array([[l6[0], l6[3], l6[4]], [l6[3], l6[1], l6[5]], [l6[4], l6[5], l6[2]]])


def test_plain16_recipe():
    pb = vi.config_plain16(16)
    assert (pb.n_cells, pb.n_nodes, pb.n_ff) == (4096, 4913, 256)
    h = 1.0 / 16
    # no jitter: every node on the lattice
    assert np.abs(pb.xyz / h - np.round(pb.xyz / h)).max() < 1e-12
    # the fracture is the node plane x = 0.5
    assert np.all(pb.xyz[pb.ff_nodes.ravel(), 0] == 0.5)
    np.testing.assert_array_equal(pb.lambda_m, np.tile([1.0, 1, 1, 0, 0, 0], (4096, 1)))
    assert np.all(pb.lambda_f == 1e4) and np.all(pb.d_f == 1e-2)
    # p = 1 - x on x = 0 and x = 1, inflow c = 1 on x = 0
    assert len(pb.dir_nodes) == 2 * 17 * 17
    x = pb.xyz[pb.dir_nodes, 0]
    assert set(np.unique(x)) == {0.0, 1.0}
    np.testing.assert_array_equal(pb.dir_values, 1.0 - x)
    np.testing.assert_array_equal(pb.cbar, (x == 0.0).astype(float))


def test_scale_recipe_at_16():
    n = 16
    pb = vi.config_scale64(n)
    h = 1.0 / n
    # fractures x = y = z = 0.5 full planes and x = 0.25 for y < 0.5: 3.5 n^2 faces
    assert pb.n_ff == 3 * n * n + n * n // 2
    lat = vi.config_plain16(n).xyz
    d = pb.xyz - lat
    assert np.abs(d).max() <= 0.2 * h + 1e-15
    assert np.abs(d).max() > 0.1 * h                      # it is jittered
    on_bnd = np.any((lat == 0.0) | (lat == 1.0), axis=1)
    assert np.all(d[on_bnd] == 0.0)                       # boundary nodes stay
    # fracture-normal coordinates are frozen: every fracture face stays in its plane
    fxyz = pb.xyz[pb.ff_nodes]                            # [n_ff, 4, 3]
    planar = np.zeros(pb.n_ff, bool)
    for ax in range(3):
        planar |= np.all(fxyz[:, :, ax] == fxyz[:, :1, ax], axis=1)
    assert planar.all()
    # lognormal anisotropic matrix permeability: k (I + 9 a a^T), one axis
    ev = np.linalg.eigvalsh(np.array([_sym(l) for l in pb.lambda_m[:200]]))
    assert np.all(ev > 0)
    np.testing.assert_allclose(ev[:, 2] / ev[:, 0], 10.0, rtol=1e-9)
    np.testing.assert_allclose(ev[:, 1] / ev[:, 0], 1.0, rtol=1e-9)
    logk = np.log10(np.array([np.linalg.eigvalsh(_sym(l))[0] for l in pb.lambda_m]))
    assert abs(np.median(logk)) < 0.1 and 0.9 < logk.std() < 1.1
    assert np.all(pb.lambda_f == 1e4)                     # ratio to the median k = 1


def test_generators_are_reproducible():
    a = vi.random_dfn_problem(10, 6, 1e4, seed=7)
    b = vi.random_dfn_problem(10, 6, 1e4, seed=7)
    for f in ("xyz", "ff_faces", "lambda_m", "lambda_f", "dir_nodes", "dir_values"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = vi.random_dfn_problem(10, 6, 1e4, seed=8)
    assert not np.array_equal(a.xyz, c.xyz)


def test_batch_recipe():
    p = np.array(vi.batch_params(256, seed=99))
    n, nf, ratio = p[:, 0], p[:, 1], p[:, 2]
    assert n.min() >= 16 and n.max() <= 48 and len(np.unique(n)) > 25
    assert nf.min() >= 1 and nf.max() <= 20
    assert ratio.min() >= 1e2 and ratio.max() <= 1e6
    lr = np.log10(ratio)
    assert abs(lr.mean() - 4.0) < 0.3                     # log-uniform on [2, 6]
    assert vi.batch_params(3, seed=99) == vi.batch_params(256, seed=99)[:3]
