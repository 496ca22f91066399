"""Checks of the seeded input generators (mesh, FEM matrices, observations, RNG)."""
import numpy as np
import scipy.sparse as sp

from synth import Stream, build, ccd_design, config_model, grid_fem, line_points, locate, theta_batch


def test_rng_is_counter_based_and_reproducible():
    a = Stream(0, 3)
    x = np.concatenate([a.uniform(5), a.uniform(7)])
    assert np.array_equal(x, Stream(0, 3).uniform(12))
    assert not np.array_equal(x, Stream(0, 4).uniform(12))
    assert not np.array_equal(x, Stream(1, 3).uniform(12))
    u = Stream(7, 1).uniform(200_000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = Stream(7, 2).normal(200_001)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2
    k = Stream(7, 3).integers(100_000, 5)
    assert set(np.unique(k)) == {0, 1, 2, 3, 4}
    mu = np.full(100_000, 3.5)
    p = Stream(7, 4).poisson(mu)
    assert abs(p.mean() - 3.5) < 0.03 and abs(p.var() - 3.5) < 0.08


def test_fem_matrices_on_grid():
    for nx in (2, 3, 8):
        C, rp, col, val = grid_fem(nx)
        G = sp.csr_matrix((val, col, rp), shape=(nx * nx, nx * nx)).toarray()
        assert np.isclose(C.sum(), 1.0, rtol=1e-14)          # area of the unit square
        assert np.allclose(G, G.T)
        assert np.allclose(G.sum(1), 0.0, atol=1e-12)        # constants are in the kernel
        assert np.all(np.linalg.eigvalsh(G) > -1e-12)
    # interior rows of right-triangle P1 stiffness are the 5-point Laplacian
    nx = 6
    C, rp, col, val = grid_fem(nx)
    G = sp.csr_matrix((val, col, rp), shape=(nx * nx, nx * nx)).toarray()
    k = 2 + nx * 3
    row = np.zeros(nx * nx)
    row[k] = 4.0
    for dk in (1, -1, nx, -nx):
        row[k + dk] = -1.0
    assert np.allclose(G[k], row, atol=1e-13)
    h = 1.0 / (nx - 1)
    assert np.isclose(C[k], h * h)
    # every triangle edge is stored, including the diagonal ones with value 0
    assert set(col[rp[k]:rp[k + 1]]) == {k, k - 1, k + 1, k - nx, k + nx, k - nx - 1, k + nx + 1}


def test_barycentric_weights_reproduce_linear_functions():
    nx = 7
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 1, (500, 2))
    p[:5] = [[0, 0], [1, 1], [1, 0], [0, 1], [0.5, 0.5]]
    verts, w = locate(nx, p[:, 0], p[:, 1])
    assert np.all(w >= -1e-15) and np.allclose(w.sum(1), 1.0)
    h = 1.0 / (nx - 1)
    vx, vy = (verts % nx) * h, (verts // nx) * h
    f = lambda x, y: 2.0 - 3.0 * x + 0.5 * y
    assert np.allclose((w * f(vx, vy)).sum(1), f(p[:, 0], p[:, 1]), atol=1e-13)


def test_observation_matrix_layout():
    mdl = build("t", 4, 5, 3, 400)
    assert np.all(np.diff(mdl.A_rowptr) == 6)
    cols = mdl.A_col.reshape(400, 6)
    t = cols[:, 0] // mdl.n_s
    assert np.array_equal(t, mdl.obs_t)
    assert np.all(cols[:, :3] // mdl.n_s == t[:, None])
    assert np.all(np.diff(cols[:, :3], axis=1) > 0)
    assert np.array_equal(cols[:, 3:], np.tile(np.arange(3) + 4 * 25, (400, 1)))
    vals = mdl.A_val.reshape(400, 6)
    assert np.allclose(vals[:, :3].sum(1), 1.0)
    mp = build("p", 2, 4, 2, 300, "poisson")
    assert np.all((mp.E >= 0.5) & (mp.E <= 2.0))
    assert np.all(mp.y == np.round(mp.y)) and mp.y.min() >= 0


def test_theta_batches():
    m1 = config_model(1)
    assert theta_batch(1, m1).shape == (9, 4)
    ccd = ccd_design(np.zeros(4), 0.1)
    assert ccd.shape == (25, 4)
    assert np.allclose(ccd.mean(0), 0.0)
    assert len({tuple(r) for r in ccd}) == 25
    lp = line_points(np.zeros(4), np.array([1.0, 0, 0, 0]))
    assert lp.shape == (16, 4) and np.isclose(lp[:, 0].max(), 0.5) and np.isclose(lp[:, 0].min(), -0.1)


def test_negative_binomial_draws_have_the_nb_moments():
    from synth.rng import Stream
    mean = np.full(200_000, 3.0)
    y = Stream(11, 5).negbinomial(4, mean).astype(float)
    # NB(mean 3, size 4): variance mean + mean^2 / size = 5.25
    assert abs(y.mean() - 3.0) < 0.02
    assert abs(y.var() - 5.25) < 0.1
    assert y.min() >= 0 and np.all(y == np.floor(y))
