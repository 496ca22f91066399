"""The library's C generator of the synthetic workloads (inla_synth_build,
host code) against the Python generator: same patterns, times, locations and
counts; floating values equal to rounding."""
import numpy as np
import pytest

from synth import build


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


CASES = [(8, 8, 2, 2000, "gaussian"), (3, 13, 0, 700, "gaussian"), (4, 10, 3, 900, "poisson"),
         (3, 9, 2, 1500, "binomial"),
         (2, 32, 4, 20000, "gaussian")]


@pytest.mark.parametrize("n_t,nx,n_b,m,lik", CASES)
def test_c_generator_matches_python(pkg, n_t, nx, n_b, m, lik):
    c = pkg.synth_build(n_t, nx, n_b, m, lik, seed=0)
    p = build("ref", n_t, nx, n_b, m, lik, seed=0)
    for name in ("G_rowptr", "G_col", "A_rowptr", "A_col"):
        assert np.array_equal(getattr(c, name), getattr(p, name)), name
    np.testing.assert_array_equal(c.C_diag, p.C_diag)
    np.testing.assert_array_equal(c.G_val, p.G_val)
    np.testing.assert_allclose(c.A_val, p.A_val, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(c.prior_mean, p.prior_mean)
    np.testing.assert_allclose(c.prior_sd, p.prior_sd)
    assert c.tau_b == p.tau_b
    if lik == "gaussian":
        assert c.E is None
        np.testing.assert_allclose(c.y, p.y, rtol=1e-12, atol=1e-12)
    else:
        np.testing.assert_array_equal(c.E, p.E)
        diff = np.abs(c.y - p.y)
        assert diff.max() <= 1 and np.count_nonzero(diff) <= max(1, m // 10000)   # CDF-boundary draws only


def test_benchmark_workload_ids(pkg):
    from paper_2204_04678_gb300 import capi
    import ctypes
    lib = capi.load()
    desc = capi.inla_model_desc()
    owner = ctypes.c_void_p()
    capi.check(lib.inla_synth_grid_model(1, 0, ctypes.byref(desc), ctypes.byref(owner)))
    try:
        assert (desc.n_t, desc.n_s, desc.n_b, desc.m, desc.lik) == (8, 64, 2, 2000, capi.INLA_LIK_GAUSSIAN)
        p = build("ref", 8, 8, 2, 2000, "gaussian", seed=0)
        y = np.ctypeslib.as_array(desc.y, (2000,))
        np.testing.assert_allclose(y, p.y, rtol=1e-12, atol=1e-12)
    finally:
        lib.inla_synth_free(owner)
    for bad in (0, 6):
        assert lib.inla_synth_grid_model(bad, 0, ctypes.byref(desc), ctypes.byref(owner)) == capi.INLA_ERR_ARG
    assert lib.inla_synth_build(0, 8, 2, 10, 0, 0, None, ctypes.byref(desc), ctypes.byref(owner)) == capi.INLA_ERR_ARG
    lib.inla_synth_free(None)


@pytest.mark.gpu
def test_c_generated_model_evaluates_like_python(pkg):
    torch = pytest.importorskip("torch")
    from synth import fd_stencil
    c = pkg.synth_build(8, 8, 2, 2000, "gaussian", seed=0)
    p = build("ref", 8, 8, 2, 2000, "gaussian", seed=0)
    th = torch.tensor(fd_stencil(p.theta_true), dtype=torch.float64, device="cuda")
    mc, mp = pkg.Model(c), pkg.Model(p)
    try:
        fc = mc.eval(th, grad="adjoint")
        fp = mp.eval(th, grad="adjoint")
        torch.cuda.synchronize()
        np.testing.assert_allclose(fc["f"].cpu().numpy(), fp["f"].cpu().numpy(), rtol=1e-12)
        np.testing.assert_allclose(fc["grad"].cpu().numpy(), fp["grad"].cpu().numpy(), rtol=1e-9, atol=1e-9)
    finally:
        mc.close()
        mp.close()
