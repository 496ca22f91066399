"""Host drivers: BFGS with the parallel line search (Sec. 3.2, Eq. bfgs_update)
and the integration stage (Sec. 2.2-2.3), checked on functions with known
minimisers and moments, and on a tiny model through the oracle."""
import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2204_04678_gb300.driver import (BISQUARE_C, bfgs, bisquare_quadratic, ccd_unit_design, integrate,
                                           line_search_steps, parallel_line_search)
from synth import Stream


def _grid():
    return np.concatenate([[0.0], line_search_steps(1.0)])


def test_line_search_points():
    a = line_search_steps(0.5)
    assert a.size == 16
    np.testing.assert_allclose(a[:14], 0.5 * np.arange(1, 15) / 14)          # 14 points on (0, gamma]
    assert np.all(a[14:] < 0) and np.all(a[14:] > -0.5)                    # 2 just behind theta_l


def test_bisquare_exact_quadratic_is_least_squares():
    a = _grid()
    coef, w = bisquare_quadratic(a, 3.0 - 2.0 * a + 5.0 * a * a)
    np.testing.assert_allclose(coef, [3.0, -2.0, 5.0], atol=1e-10)
    np.testing.assert_allclose(w, 1.0)


def test_bisquare_rejects_gross_outliers():
    a = _grid()
    f = 3.0 - 2.0 * a + 5.0 * a * a + 1e-4 * np.sin(7.0 * a)
    g = f.copy()
    g[[4, 9]] += [40.0, -25.0]
    coef, w = bisquare_quadratic(a, g)
    ls = np.polynomial.polynomial.polyfit(a, f, 2)        # least squares on the clean data
    np.testing.assert_allclose(coef, ls, atol=1e-3)
    assert w[4] == 0.0 and w[9] == 0.0
    bad = np.polynomial.polynomial.polyfit(a, g, 2)       # plain least squares is dragged away
    assert np.abs(bad - ls).max() > 1.0


def test_bisquare_weights_are_a_fixed_point():
    a = _grid()
    s = Stream(11, 0)
    f = 1.0 + a - 2.0 * a * a + 0.05 * s.normal(a.size)
    coef, w = bisquare_quadratic(a, f, max_iter=500)
    X = np.stack([np.ones_like(a), a, a * a], 1)
    r = f - X @ coef
    scale = np.median(np.abs(r - np.median(r))) / 0.6745
    u = r / (BISQUARE_C * scale)
    np.testing.assert_allclose(w, np.where(np.abs(u) < 1, (1 - u * u) ** 2, 0.0), atol=1e-8)
    np.testing.assert_allclose(X.T @ (w * r), 0.0, atol=1e-9)    # weighted normal equations


def _quadratic(H, mu):
    def fg(t):
        d = t - mu
        return 0.5 * d @ H @ d, H @ d

    def fb(P):
        D = P - mu
        return 0.5 * np.einsum("ki,ij,kj->k", D, H, D)
    return fg, fb


def _spd(seed, d=4):
    s = Stream(seed, 0)
    M = s.normal(d * d).reshape(d, d)
    return M @ M.T + d * np.eye(d)


def test_line_search_finds_exact_minimiser_of_quadratic():
    H, mu = _spd(3), np.array([0.3, -0.2, 0.1, 0.4])
    fg, fb = _quadratic(H, mu)
    th = np.zeros(4)
    f0, g = fg(th)
    d = -g / np.linalg.norm(g)
    exact = -(g @ d) / (d @ H @ d)
    assert 0 < exact < 1
    step, gamma, pts, fv = parallel_line_search(fb, th, f0, d, 1.0)
    assert gamma == 1.0
    np.testing.assert_allclose(step, exact, rtol=1e-9)
    np.testing.assert_allclose(fv, fb(pts))


def test_line_search_shrinks_the_interval_when_nothing_improves():
    H, mu = _spd(3) * 1e4, np.array([0.3, -0.2, 0.1, 0.4])
    fg, fb = _quadratic(H, mu)
    th = np.zeros(4)
    f0, g = fg(th)
    d = -g
    exact = -(g @ d) / (d @ H @ d)
    assert exact < 1.0 / 28                     # below the first point's half: no grid point improves
    step, gamma, pts, fv = parallel_line_search(fb, th, f0, d, 1.0)
    assert gamma < 1.0 and np.min(fv[:14]) < f0
    np.testing.assert_allclose(step, exact, rtol=1e-9)


def test_bfgs_converges_on_quadratic():
    H, mu = _spd(5), np.array([1.0, -1.0, 0.5, 2.0])
    fg, fb = _quadratic(H, mu)
    r = bfgs(fg, fb, np.zeros(4), max_iter=60, gtol=1e-9)
    assert r["iterations"] <= 12
    np.testing.assert_allclose(r["theta"], mu, atol=1e-8)
    assert np.all(np.diff(r["history"]) <= 1e-12)


def test_bfgs_matches_scipy_on_smooth_convex_function():
    H = _spd(7)
    c = np.array([0.5, -0.3, 0.2, 0.1])

    def fg(t):
        e = np.exp(t)
        return 0.5 * t @ H @ t + e.sum() - c @ t * 3, H @ t + e - 3 * c

    def fb(P):
        return np.array([fg(p)[0] for p in P])
    r = bfgs(fg, fb, np.ones(4), max_iter=100, gtol=1e-8)
    assert np.abs(r["grad"]).max() < 1e-8
    ref = minimize(lambda t: fg(t)[0], np.ones(4), jac=lambda t: fg(t)[1], method="BFGS", tol=1e-12)
    np.testing.assert_allclose(r["theta"], ref.x, atol=1e-7)


def test_bfgs_on_badly_scaled_quadratic():
    """Curvatures 1e4 apart (as for f with ~1e5 observations): the first
    steepest-descent steps overshoot the grid and the interval shrinks."""
    H = np.diag([2e4, 3e3, 50.0, 2.0]) + 0.5
    mu = np.array([1.0, -1.0, 0.1, 1.5])
    fg, fb = _quadratic(H, mu)
    r = bfgs(fg, fb, mu + np.array([0.3, -0.3, 0.2, -0.4]), max_iter=60, gtol=1e-6)
    assert np.abs(r["grad"]).max() < 1e-6
    np.testing.assert_allclose(r["theta"], mu, atol=1e-6)


def test_ccd_design_is_rotatable():
    Z = ccd_unit_design(4)
    assert Z.shape == (25, 4)
    np.testing.assert_allclose(np.linalg.norm(Z[1:], axis=1), 2.0)           # all on the sphere of radius 2
    M2 = Z.T @ Z
    np.testing.assert_allclose(M2, np.diag(np.diag(M2)))                       # orthogonal
    np.testing.assert_allclose(np.diag(M2), 24.0)                              # 8 + 16 per axis
    assert np.sum(Z[:, 0] ** 4) == pytest.approx(3 * np.sum(Z[:, 0] ** 2 * Z[:, 1] ** 2))   # rotatability


def test_integrate_on_exact_gaussian_posterior():
    """f quadratic in theta: the Hessian is exact, the weights are exp(-|z|^2/2)
    normalised, and the mixture moments have closed forms."""
    H, mu = _spd(9), np.array([0.2, -0.4, 1.0, 0.3])
    s = Stream(13, 0)
    Mx = s.normal(6 * 4).reshape(6, 4)
    v0 = 0.5 + s.uniform(6)

    def grads(P):
        return (P - mu) @ H

    def full(P):
        D = P - mu
        return 0.5 * np.einsum("ki,ij,kj->k", D, H, D) + 7.0, P @ Mx.T, np.tile(v0, (len(P), 1))
    r = integrate(grads, full, mu, h=1e-2)
    np.testing.assert_allclose(r["hessian"], H, rtol=1e-10)
    Z = ccd_unit_design(4)
    w = np.exp(-0.5 * np.sum(Z * Z, 1))
    np.testing.assert_allclose(r["weights"], w / w.sum(), rtol=1e-10)
    np.testing.assert_allclose(r["theta_mean"], mu, atol=1e-12)
    # weighted second moment of z along one axis: 2 axial points at z^2 = 4 and
    # 16 corners at z^2 = 1, all of weight e^-2, over the total 1 + 24 e^-2
    m2 = (2 * 4 + 16) * np.exp(-2.0) / (1 + 24 * np.exp(-2.0))
    np.testing.assert_allclose(r["theta_cov"], m2 * np.linalg.inv(H), rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(r["x_mean"], Mx @ mu, atol=1e-12)
    np.testing.assert_allclose(r["x_var"], v0 + np.einsum("ij,jk,ik->i", Mx, r["theta_cov"], Mx), rtol=1e-9)


def _oracle_evaluators(mdl):
    from oracle import bta

    def fg(t):
        r = bta.gaussian(mdl, np.asarray(t, float), want_grad=True)
        return r["f"], np.asarray(r["grad"])

    def f_or_nan(p):
        try:
            return bta.gaussian(mdl, p)["f"]
        except np.linalg.LinAlgError:        # not positive definite: a failed point
            return np.nan

    def fb(P):
        return np.array([f_or_nan(p) for p in P])

    def gb(P):
        return np.array([bta.gaussian(mdl, p, want_grad=True)["grad"] for p in P])

    def full(P):
        rs = [bta.gaussian(mdl, p, want_var=True) for p in P]
        return (np.array([r["f"] for r in rs]), np.array([r["x"] for r in rs]),
                np.array([r["var"] for r in rs]))
    return fg, fb, gb, full


def test_bfgs_and_integration_on_tiny_model_with_the_oracle():
    from synth import build
    mdl = build("tiny", 3, 4, 1, 150, "gaussian", seed=2)
    fg, fb, gb, full = _oracle_evaluators(mdl)
    t0 = np.asarray(mdl.theta_true) + np.array([0.3, -0.3, 0.2, -0.4])
    r = bfgs(fg, fb, t0, max_iter=80, gtol=1e-5)
    assert np.abs(r["grad"]).max() < 1e-5
    ref = minimize(lambda t: fg(t)[0], t0, jac=lambda t: fg(t)[1], method="BFGS", tol=1e-10)
    np.testing.assert_allclose(r["theta"], ref.x, atol=1e-4)
    assert r["f"] <= ref.fun + 1e-8
    integ = integrate(gb, full, r["theta"])
    assert integ["weights"].sum() == pytest.approx(1.0)
    assert np.all(np.linalg.eigvalsh(integ["hessian"]) > 0)
    assert np.all(integ["x_var"] > 0)


def test_bfgs_checkpoint_and_resume_reproduce_an_uninterrupted_run(tmp_path):
    from paper_2204_04678_gb300.driver import load_state, save_state
    H = np.diag([2e4, 3e3, 50.0, 2.0]) + 0.5
    mu = np.array([1.0, -1.0, 0.1, 1.5])
    fg, fb = _quadratic(H, mu)
    t0 = mu + np.array([0.3, -0.3, 0.2, -0.4])
    full = bfgs(fg, fb, t0, max_iter=60, gtol=1e-8)
    path = tmp_path / "bfgs.json"
    bfgs(fg, fb, t0, max_iter=3, gtol=1e-8, on_iteration=lambda st: save_state(path, st))
    st = load_state(path)
    assert st["iteration"] == 3
    resumed = bfgs(fg, fb, None, max_iter=60, gtol=1e-8, state=st)
    assert resumed["iterations"] == full["iterations"]
    np.testing.assert_array_equal(resumed["theta"], full["theta"])
    np.testing.assert_array_equal(resumed["history"], full["history"])
