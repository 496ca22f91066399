"""Degenerate and extreme inputs of the CUDA path (through the C ABI) against
the CPU oracle, at the FP64 parity tolerances of test_gpu_parity.py:

* time steps with no observations (the Schur recursion then runs on the prior
  blocks alone for those steps), and a single observation;
* hyperparameters far from the data-generating values: rho close to 1, a
  range much shorter and much longer than the mesh spacing, very small and
  very large observation precision and field scale (the oracle's block and
  dense evaluations agree to 1e-13 at all of them);
* an empty batch, which the library rejects as an argument error;
* batches whose points share the range parameter (a central composite
  design: five distinct ranges among 25 points), where one inversion of the
  spatial precision serves every point with that range: each point of the
  batch agrees with the same point evaluated alone.
"""
import ctypes

import numpy as np
import pytest

from synth import build, ccd_design
from oracle import bta

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F, RTOL_X, RTOL_V, RTOL_G = 1e-10, 1e-9, 1e-9, 1e-8


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def check(r, b, ref):
    assert int(r["status"][b]) == 0
    f = float(r["f"][b])
    assert abs(f - ref["f"]) <= RTOL_F * abs(ref["f"]), (f, ref["f"])
    x = r["x_mode"][b].cpu().numpy()
    assert np.abs(x - ref["x"]).max() <= RTOL_X * np.abs(ref["x"]).max()
    v = r["marg_var"][b].cpu().numpy()
    assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= RTOL_V
    g = r["grad"][b].cpu().numpy()
    assert np.abs(g - ref["grad"]).max() <= RTOL_G * max(1.0, np.abs(ref["grad"]).max()), (g, ref["grad"])


@pytest.mark.parametrize("lik,n_t,nx,n_b,m", [("gaussian", 6, 5, 1, 4), ("poisson", 5, 5, 1, 6),
                                              ("binomial", 5, 5, 1, 6), ("gaussian", 3, 4, 2, 1)])
def test_time_steps_without_observations(pkg, lik, n_t, nx, n_b, m):
    mdl = build("sparse data", n_t, nx, n_b, m, lik, seed=3)
    assert np.any(np.bincount(mdl.obs_t, minlength=n_t) == 0)
    th = mdl.theta_true[None, :] + np.array([[0.0, 0.0, 0.0, 0.0], [0.2, -0.3, 0.1, -0.5]])
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        check(r, b, bta.evaluate(mdl, th[b], want_grad=True, want_var=True))


EXTREME = np.array([
    [1.0, -1.0, 0.0, 6.0],     # rho = 0.9975
    [1.0, -3.0, 0.0, 1.5],     # range 0.05, a quarter of the mesh spacing
    [1.0, 1.5, 0.0, 1.5],      # range 4.5, longer than the domain
    [-5.0, -1.0, 0.0, 1.5],    # observation noise sd 12
    [8.0, -1.0, 0.0, 1.5],     # observation noise sd 0.018
    [1.0, -1.0, 3.0, 1.5],     # field sd 20
    [1.0, -1.0, -3.0, -4.0],   # field sd 0.05, rho = 0.018
])


def test_extreme_hyperparameters(pkg):
    mdl = build("g", 4, 6, 2, 300, "gaussian", seed=4)
    model = pkg.Model(mdl)
    r = model.eval(cuda(EXTREME), grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    for b in range(EXTREME.shape[0]):
        check(r, b, bta.evaluate(mdl, EXTREME[b], want_grad=True, want_var=True))


def test_empty_batch_is_rejected(pkg):
    mdl = build("g", 2, 4, 1, 100, "gaussian")
    model = pkg.Model(mdl)
    th = cuda(mdl.theta_true[None, :])
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    so = pkg.capi.inla_eval_out()
    so.f_dev, so.status_dev = f.data_ptr(), st.data_ptr()
    o = pkg.make_opts()
    code = model.lib.inla_eval_batch(model.handle, 0, ctypes.c_void_p(th.data_ptr()), ctypes.byref(o),
                                     ctypes.byref(so), None)
    assert code == pkg.capi.INLA_ERR_ARG
    assert model.lib.inla_last_error().decode()
    # the model stays usable after the rejected call
    r = model.eval(th)
    torch.cuda.synchronize()
    assert int(r["status"][0]) == 0 and np.isfinite(float(r["f"][0]))


def test_points_sharing_the_range_parameter(pkg):
    mdl = build("g", 3, 7, 2, 300, "gaussian", seed=6)
    pts = ccd_design(mdl.theta_true, 0.1)
    assert len(np.unique(pts[:, 1])) == 5
    model = pkg.Model(mdl)
    r = model.eval(cuda(pts), grad="adjoint")
    torch.cuda.synchronize()
    f, g = r["f"].cpu().numpy(), r["grad"].cpu().numpy()
    assert np.all(r["status"].cpu().numpy() == 0)
    for b in range(pts.shape[0]):
        one = model.eval(cuda(pts[b:b + 1]), grad="adjoint")   # its own representative
        torch.cuda.synchronize()
        assert abs(f[b] - float(one["f"][0])) <= 1e-12 * abs(f[b])
        assert np.abs(g[b] - one["grad"][0].cpu().numpy()).max() <= 1e-10 * max(1.0, np.abs(g[b]).max())
    for b in (0, 3, 9, 24):
        ref = bta.evaluate(mdl, pts[b], want_grad=True)
        assert abs(f[b] - ref["f"]) <= RTOL_F * abs(ref["f"])
        assert np.abs(g[b] - ref["grad"]).max() <= RTOL_G * max(1.0, np.abs(ref["grad"]).max())
