"""BFGS with the parallel line search and the integration stage driven by the
CUDA path, against the same drivers over the oracle (n_t = 8, 8 x 8 grid,
n_b = 2, m = 2000 Gaussian observations)."""
import numpy as np
import pytest

from oracle import bta
from synth import config_model, theta_batch
from paper_2204_04678_gb300.driver import bfgs, integrate, model_evaluators

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2204_04678_gb300 as p
    p.build()
    mdl = config_model(1)
    model = p.Model(mdl)
    yield mdl, model
    model.close()


def _oracle(mdl):
    def fg(t):
        r = bta.gaussian(mdl, np.asarray(t, float), want_grad=True)
        return r["f"], np.asarray(r["grad"])

    def f_or_nan(p):
        try:
            return bta.gaussian(mdl, p)["f"]
        except np.linalg.LinAlgError:
            return np.nan

    def fb(P):
        return np.array([f_or_nan(p) for p in P])

    def gb(P):
        return np.array([bta.gaussian(mdl, p, want_grad=True)["grad"] for p in P])

    def full(P):
        rs = [bta.gaussian(mdl, p, want_var=True) for p in P]
        return np.array([r["f"] for r in rs]), np.array([r["x"] for r in rs]), np.array([r["var"] for r in rs])
    return fg, fb, gb, full


@pytest.fixture(scope="module")
def oracle_run(setup):
    mdl, _ = setup
    fg, fb, gb, full = _oracle(mdl)
    start = theta_batch(2, mdl)[0] + np.array([0.3, -0.3, 0.2, -0.4])
    r = bfgs(fg, fb, start, max_iter=40, gtol=1e-4)
    return start, r, integrate(gb, full, r["theta"])


def test_bfgs_adjoint_fp64_follows_the_oracle(setup, oracle_run):
    mdl, model = setup
    start, ref, _ = oracle_run
    fg, fb, _, _ = model_evaluators(model, grad="adjoint", precision="fp64")
    r = bfgs(fg, fb, start, max_iter=40, gtol=1e-4)
    assert r["iterations"] == ref["iterations"]
    np.testing.assert_allclose(r["history"], ref["history"], rtol=1e-9)
    np.testing.assert_allclose(r["theta"], ref["theta"], atol=1e-6)


def test_bfgs_fd_and_mixed_reach_the_same_mode(setup, oracle_run):
    mdl, model = setup
    start, ref, _ = oracle_run
    for grad, prec in (("fd", "fp64"), ("adjoint", "mixed")):
        fg, fb, _, _ = model_evaluators(model, grad=grad, precision=prec)
        r = bfgs(fg, fb, start, max_iter=40, gtol=1e-4)
        np.testing.assert_allclose(r["theta"], ref["theta"], atol=1e-2)
        # the oracle's f at the point reached is the minimum to 1e-8 relative
        f_there = bta.gaussian(mdl, r["theta"])["f"]
        assert f_there - ref["f"] <= 1e-8 * abs(ref["f"]), (grad, prec, f_there, ref["f"])


def test_integration_stage_matches_the_oracle(setup, oracle_run):
    mdl, model = setup
    _, ref_b, ref = oracle_run
    _, _, gb, full = model_evaluators(model, grad="adjoint", precision="fp64")
    r = integrate(gb, full, ref_b["theta"])
    np.testing.assert_allclose(r["hessian"], ref["hessian"], rtol=1e-6, atol=1e-6 * np.abs(ref["hessian"]).max())
    np.testing.assert_allclose(r["design"], ref["design"], atol=1e-6)
    np.testing.assert_allclose(r["weights"], ref["weights"], rtol=1e-6)
    np.testing.assert_allclose(r["x_mean"], ref["x_mean"], rtol=1e-6, atol=1e-8 * np.abs(ref["x_mean"]).max())
    np.testing.assert_allclose(r["x_var"], ref["x_var"], rtol=1e-6)
