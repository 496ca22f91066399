"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64 path): relative 1e-10 on f and the log-determinants,
||dx||_inf / ||x||_inf <= 1e-9 on the mode, max_i |dv_i| / v_i <= 1e-9 on
the marginal variances, and 1e-8 relative (to max(1, |grad|_inf)) on the
adjoint gradient, whose terms are sums of n_t * nnz products of selected
inverse entries.
"""
import math

import numpy as np
import pytest

from synth import build, config_model, fd_stencil, theta_batch
from oracle import bta, dense, fd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F, RTOL_X, RTOL_V, RTOL_G = 1e-10, 1e-9, 1e-9, 1e-8


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def thetas(mdl, k=3, seed=0):
    rng = np.random.default_rng(seed)
    return mdl.theta_true[None, :] + 0.15 * rng.standard_normal((k, 4))


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def check_point(r, b, ref, n, grad=True, var=True, mode=True):
    assert int(r["status"][b]) == 0
    f = float(r["f"][b])
    assert abs(f - ref["f"]) <= RTOL_F * abs(ref["f"]), (f, ref["f"])
    if mode:
        x = r["x_mode"][b].cpu().numpy()
        assert np.abs(x - ref["x"]).max() <= RTOL_X * np.abs(ref["x"]).max()
    if var:
        v = r["marg_var"][b].cpu().numpy()
        assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= RTOL_V
    if grad:
        g = r["grad"][b].cpu().numpy()
        assert np.abs(g - ref["grad"]).max() <= RTOL_G * max(1.0, np.abs(ref["grad"]).max()), (g, ref["grad"])


GAUSS_CASES = [
    (1, 4, 0, 60),      # one time step (no chain), no fixed effects
    (2, 3, 1, 50),      # n_s = 9 < one tile
    (3, 8, 2, 400),     # n_s = 64: exactly one tile
    (4, 10, 3, 600),    # n_s = 100: two tiles, ragged tail
    (6, 13, 2, 1500),   # n_s = 169: three tiles, ragged tail
]


@pytest.mark.parametrize("n_t,nx,n_b,m", GAUSS_CASES)
def test_gaussian_batch_matches_oracle(pkg, n_t, nx, n_b, m):
    mdl = build("g", n_t, nx, n_b, m, "gaussian", seed=n_t + nx)
    th = thetas(mdl)
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        ref = bta.gaussian(mdl, th[b], want_grad=True, want_var=True)
        check_point(r, b, ref, mdl.n)
        if mdl.n <= 1200:
            d = dense.gaussian_eval(mdl, th[b])
            assert abs(float(r["f"][b]) - d["f"]) <= RTOL_F * abs(d["f"])


@pytest.mark.parametrize("lik,n_t,nx,n_b,m", [("poisson", 3, 4, 2, 250), ("poisson", 2, 10, 1, 400),
                                              ("poisson", 1, 3, 0, 80), ("binomial", 3, 4, 2, 250),
                                              ("binomial", 2, 10, 1, 400), ("binomial", 1, 3, 0, 80),
                                              ("negbinomial", 3, 4, 2, 250), ("negbinomial", 2, 10, 1, 400),
                                              ("negbinomial", 1, 3, 0, 80), ("negbinomial", 3, 16, 2, 900)])
def test_poisson_batch_matches_oracle(pkg, lik, n_t, nx, n_b, m):
    mdl = build("p", n_t, nx, n_b, m, lik, seed=5)
    th = thetas(mdl, k=3, seed=1)
    th[:, 0] = np.log(np.array([1e-3, 0.1, 1.0]))
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        ref = bta.poisson(mdl, th[b], want_grad=True, want_var=True)
        check_point(r, b, ref, mdl.n)
        assert abs(int(r["newton_iters"][b]) - ref["iters"]) <= 1


def test_forward_difference_gradient_matches_oracle(pkg):
    mdl = build("g", 3, 6, 2, 400, "gaussian", seed=9)
    th = thetas(mdl, 2, seed=4)
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="fd_forward")
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        f = lambda t: bta.gaussian(mdl, t)["f"]
        ref = fd.forward_gradient(f, th[b], 1e-3)
        assert int(r["status"][b]) == 0
        assert abs(float(r["f"][b]) - f(th[b])) <= RTOL_F * abs(f(th[b]))
        # differences of f values that agree to 1e-10 relative, divided by eps
        g = r["grad"][b].cpu().numpy()
        assert np.abs(g - ref).max() <= 1e-10 * abs(f(th[b])) / 1e-3 * 4


def test_prior_modes_agree(pkg):
    mdl = build("g", 4, 9, 2, 500, "gaussian", seed=3)
    th = thetas(mdl, 2)
    model = pkg.Model(mdl)
    a = model.eval(cuda(th), grad="adjoint", prior="kronecker")
    b = model.eval(cuda(th), grad="adjoint", prior="bta")
    torch.cuda.synchronize()
    fa, fb = a["f"].cpu().numpy(), b["f"].cpu().numpy()
    assert np.all(np.abs(fa - fb) <= RTOL_F * np.abs(fa))
    ga, gb = a["grad"].cpu().numpy(), b["grad"].cpu().numpy()
    assert np.abs(ga - gb).max() <= RTOL_G * max(1.0, np.abs(ga).max())


def test_config1_fd_gradient_and_closed_form(pkg):
    mdl = config_model(1)
    centre = mdl.theta_true
    model = pkg.Model(mdl)
    r = model.eval(cuda(centre[None, :]), grad="fd", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    f = float(r["f"][0])
    cf = dense.gaussian_closed_form(mdl, centre)
    assert abs(f - cf) <= RTOL_F * abs(cf)
    pts = fd_stencil(centre)
    fo = [bta.gaussian(mdl, p)["f"] for p in pts]
    g_ref = fd.gradient_from_stencil(fo)
    g = r["grad"][0].cpu().numpy()
    assert np.abs(g - g_ref).max() <= 2 * RTOL_F * abs(cf) / 1e-3
    ref = bta.gaussian(mdl, centre, want_var=True)
    assert np.abs(r["x_mode"][0].cpu().numpy() - ref["x"]).max() <= RTOL_X * np.abs(ref["x"]).max()
    assert np.max(np.abs(r["marg_var"][0].cpu().numpy() - ref["var"]) / ref["var"]) <= RTOL_V
    # the adjoint gradient agrees with the central differences to O(eps^2)
    ra = model.eval(cuda(centre[None, :]), grad="adjoint")
    assert np.abs(ra["grad"][0].cpu().numpy() - g).max() <= 1e-4 * max(1.0, np.abs(g).max())


def test_fd_batch_of_centres_matches_single_evaluations(pkg):
    mdl = build("g", 3, 6, 2, 300, "gaussian", seed=11)
    th = thetas(mdl, 3, seed=4)
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="fd")
    flat = model.eval(cuda(np.concatenate([fd_stencil(t) for t in th])), grad="none")
    torch.cuda.synchronize()
    fv = flat["f"].cpu().numpy().reshape(3, 9)
    assert np.array_equal(r["f"].cpu().numpy(), fv[:, 0])
    g = np.array([fd.gradient_from_stencil(v) for v in fv])
    assert np.allclose(r["grad"].cpu().numpy(), g, rtol=0, atol=1e-12 * np.abs(fv).max() / 1e-3)


def test_status_codes_for_failures(pkg):
    mdl = build("g", 2, 4, 1, 100, "gaussian")
    model = pkg.Model(mdl)
    th = thetas(mdl, 3)
    th[1, 1] = np.nan                       # invalid point: pivots are not positive
    r = model.eval(cuda(th), grad="adjoint", want_mode=True)
    torch.cuda.synchronize()
    st = r["status"].cpu().numpy()
    assert st[0] == 0 and st[2] == 0 and st[1] == pkg.capi.INLA_ERR_NOT_SPD
    assert math.isinf(float(r["f"][1])) and np.isnan(r["grad"][1].cpu().numpy()).all()
    assert np.isfinite(r["f"][[0, 2]].cpu().numpy()).all()
    mp = build("p", 2, 4, 1, 200, "poisson")
    rp = pkg.Model(mp).eval(cuda(mp.theta_true[None, :]), max_newton=1)
    torch.cuda.synchronize()
    assert int(rp["status"][0]) == pkg.capi.INLA_ERR_NO_CONVERGENCE and math.isinf(float(rp["f"][0]))


def test_invalid_calls_raise(pkg):
    mdl = build("g", 2, 4, 1, 100, "gaussian")
    model = pkg.Model(mdl)
    th = cuda(thetas(mdl, 1))
    with pytest.raises(pkg.capi.InlaError):
        o = pkg.make_opts(grad="adjoint")
        so = pkg.capi.inla_eval_out()
        so.f_dev = th.data_ptr()
        so.status_dev = None
        import ctypes
        pkg.capi.check(model.lib.inla_eval_batch(model.handle, 1, ctypes.c_void_p(th.data_ptr()),
                                                 ctypes.byref(o), ctypes.byref(so), None))


def test_host_api_and_determinism(pkg):
    mdl = build("g", 3, 7, 2, 300, "gaussian", seed=2)
    th = thetas(mdl, 2)
    model = pkg.Model(mdl)
    d1 = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True)
    d2 = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True)
    h = model.eval_host(th, grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    for k in ("f", "grad", "x_mode", "marg_var"):
        assert np.array_equal(d1[k].cpu().numpy(), d2[k].cpu().numpy()), k
        assert np.array_equal(d1[k].cpu().numpy(), h[k]), k


def test_autograd_function(pkg):
    mdl = build("g", 3, 5, 1, 200, "gaussian", seed=9)
    model = pkg.Model(mdl)
    th = cuda(thetas(mdl, 2)).requires_grad_(True)
    f = pkg.log_posterior(th, model)
    w = torch.tensor([0.3, -1.7], dtype=torch.float64, device="cuda")
    (f * w).sum().backward()
    r = model.eval(th.detach(), grad="adjoint")
    torch.cuda.synchronize()
    assert torch.equal(f.detach(), r["f"])
    assert torch.allclose(th.grad, w[:, None] * r["grad"], rtol=0, atol=0)


# ---------------------------------------------------------------- mixed precision
# Dense blocks in FP32, pivots' log-determinants accumulated in FP64, the mode
# refined with FP64 residuals, and every FP32 block update summed before it is
# added to the block (one rounding per block step).  Held to the stated error
# budget of the mixed form: 1e-6 relative on f and 1e-5 on the gradient (of its
# largest component); the refined mode to the FP64 tolerance.  The marginal
# variances are read from FP32 selected-inverse blocks (entries ~1e-6 relative,
# amplified by the block condition numbers): 5e-5.
MIX_F, MIX_G, MIX_X, MIX_V = 1e-6, 1e-5, 1e-9, 5e-5


@pytest.mark.parametrize("lik,n_t,nx,n_b,m", [("gaussian", 4, 10, 3, 600), ("gaussian", 6, 13, 2, 1500),
                                              ("gaussian", 1, 4, 0, 60), ("poisson", 3, 6, 2, 400),
                                              ("binomial", 3, 6, 2, 400), ("negbinomial", 3, 6, 2, 400),
                                              ("gaussian", 3, 16, 2, 900), ("negbinomial", 3, 16, 2, 900)])
def test_mixed_precision_matches_oracle(pkg, lik, n_t, nx, n_b, m):
    mdl = build("mx", n_t, nx, n_b, m, lik, seed=7)
    th = thetas(mdl, 3, seed=3)
    if lik != "gaussian":
        th[:, 0] = np.log(np.array([1e-3, 0.1, 1.0]))
    model = pkg.Model(mdl)
    r = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True, precision="mixed")
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        ref = bta.evaluate(mdl, th[b], want_grad=True, want_var=True)
        assert int(r["status"][b]) == 0
        assert abs(float(r["f"][b]) - ref["f"]) <= MIX_F * abs(ref["f"])
        g = r["grad"][b].cpu().numpy()
        assert np.abs(g - ref["grad"]).max() <= MIX_G * max(1.0, np.abs(ref["grad"]).max()), (g, ref["grad"])
        x = r["x_mode"][b].cpu().numpy()
        assert np.abs(x - ref["x"]).max() <= MIX_X * np.abs(ref["x"]).max()
        v = r["marg_var"][b].cpu().numpy()
        assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= MIX_V


def test_cuda_graph_replay_matches_eager(pkg):
    mdl = build("g", 4, 9, 2, 500, "gaussian", seed=12)
    model = pkg.Model(mdl)
    for kw in (dict(grad="adjoint", want_mode=True, want_marg_var=True), dict(grad="fd"),
               dict(grad="adjoint", precision="mixed")):
        for k in (3, 2, 3):     # the third call replays the graph captured by the first
            th = cuda(thetas(mdl, k, seed=k))
            eager = model.eval(th, **kw)
            graph = model.eval(th, use_graph=True, **kw)
            torch.cuda.synchronize()
            for key in ("f", "grad", "x_mode", "marg_var", "status"):
                if key in eager:
                    assert torch.equal(eager[key], graph[key]), (kw, k, key)


@pytest.mark.parametrize("lik", ["poisson", "binomial", "negbinomial"])
def test_cuda_graph_newton_loop_matches_eager(pkg, lik):
    # uneven Newton counts in one graph launch: the loop is a conditional while-node
    mdl = build("p", 3, 6, 2, 400, lik, seed=13)
    model = pkg.Model(mdl)
    th = thetas(mdl, 4, seed=2)
    th[:, 0] = np.log(np.array([1e-3, 0.1, 1.0, 10.0]))
    for kw in (dict(grad="adjoint", want_mode=True, want_marg_var=True), dict(grad="fd"),
               dict(grad="adjoint", precision="mixed")):
        for rep in range(2):    # capture, then replay
            eager = model.eval(cuda(th), **kw)
            graph = model.eval(cuda(th), use_graph=True, **kw)
            torch.cuda.synchronize()
            for key in ("f", "grad", "x_mode", "marg_var", "status", "newton_iters"):
                if key in eager:
                    assert torch.equal(eager[key], graph[key]), (lik, kw, rep, key)
        it = eager["newton_iters"].cpu().numpy()
        assert it.min() >= 1
    # an iteration limit ends the device loop with the status, as on the eager path
    r = model.eval(cuda(th[:1]), max_newton=1, use_graph=True)
    torch.cuda.synchronize()
    assert int(r["status"][0]) == pkg.capi.INLA_ERR_NO_CONVERGENCE


@pytest.mark.parametrize("nx", [16, 23])
def test_fp64_selinv_products_tensor_cores_match_oracle(pkg, nx):
    # n_s = 256 and 529 (padded to 256 and 640, multiples of 128): the FP64 selected
    # inversion's products through BF16 digit slices on the tensor cores, against the
    # oracle and against the same products with FP64 FMA on the CUDA cores
    mdl = build("z", 3, nx, 2, 800, "gaussian", seed=nx)
    th = thetas(mdl, 2, seed=5)
    model = pkg.Model(mdl)
    kw = dict(grad="adjoint", want_mode=True, want_marg_var=True)
    t = model.eval(cuda(th), **kw)
    model.set_fp64_products(False)
    c = model.eval(cuda(th), **kw)
    torch.cuda.synchronize()
    for b in range(th.shape[0]):
        ref = bta.gaussian(mdl, th[b], want_grad=True, want_var=True)
        check_point(t, b, ref, mdl.n)
        check_point(c, b, ref, mdl.n)
    vt, vc = t["marg_var"].cpu().numpy(), c["marg_var"].cpu().numpy()
    assert np.max(np.abs(vt - vc) / vc) <= 1e-11


def test_autotune_keeps_results(pkg):
    mdl = build("g", 3, 10, 2, 500, "gaussian", seed=21)
    th = thetas(mdl, 2, seed=8)
    model = pkg.Model(mdl)
    for prec, tol in (("fp64", RTOL_F), ("mixed", MIX_F)):
        choice = model.autotune(cuda(th), grad="adjoint", precision=prec)
        assert choice[0] in (32, 64) and choice[1] in (32, 64, pkg.capi.INLA_SWEEP_TF32X3, pkg.capi.INLA_INV_BLOCKED)
        assert choice[2] in (64, 128, pkg.capi.INLA_GEMM_TF32X3)
        r = model.eval(cuda(th), grad="adjoint", precision=prec)
        torch.cuda.synchronize()
        for b in range(th.shape[0]):
            ref = bta.gaussian(mdl, th[b], want_grad=True)
            assert abs(float(r["f"][b]) - ref["f"]) <= tol * abs(ref["f"])
    # every tile shape is the same algorithm: results agree to rounding
    for prec, tol in (("fp64", RTOL_F), ("mixed", MIX_F)):
        outs = []
        for tiles in ((32, 32, 64), (64, 64, 128), (32, 64, pkg.capi.INLA_GEMM_TF32X3)):
            model.set_tiles(*tiles)
            outs.append(model.eval(cuda(th), grad="adjoint", precision=prec))
        torch.cuda.synchronize()
        fa = outs[0]["f"].cpu().numpy()
        for o in outs[1:]:
            assert np.all(np.abs(fa - o["f"].cpu().numpy()) <= tol * np.abs(fa))
    with pytest.raises(pkg.capi.InlaError):
        model.set_tiles(48, 64, 128)
