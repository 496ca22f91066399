"""inla_eval_batch_static: the evaluation with the library's fixed device
array as workspace (no device allocation in the call).  Checked against
inla_eval_batch on the same inputs, on two calls in a row, within the
parity tolerances, and for the clear rejection of a batch that does not fit.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from synth import build, config_model, theta_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F, RTOL_X, RTOL_V, RTOL_G = 1e-10, 1e-9, 1e-9, 1e-8


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def close(a, b, rtol):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(b), 1.0))


@pytest.mark.parametrize("lik", ["gaussian", "poisson"])
def test_static_scratch_matches_allocating_entry_point(pkg, lik):
    mdl = config_model(1) if lik == "gaussian" else build("p", 3, 6, 2, 400, "poisson", seed=3)
    th = torch.tensor(theta_batch(1, config_model(1))[:3] if lik == "gaussian"
                      else mdl.theta_true[None, :] + 0.1 * np.arange(3)[:, None],
                      dtype=torch.float64, device="cuda")
    model = pkg.Model(mdl)
    for grad in ("adjoint", "fd"):
        kw = dict(grad=grad, want_mode=True, want_marg_var=True)
        ref = model.eval(th, **kw)
        for _ in range(2):   # two calls in a row share (and reuse) the static array
            got = model.eval_static(th, **kw)
            torch.cuda.synchronize()
            assert torch.equal(got["status"], ref["status"]) and int(ref["status"].abs().sum()) == 0
            assert close(got["f"], ref["f"], RTOL_F)
            assert close(got["grad"], ref["grad"], RTOL_G)
            assert close(got["x_mode"], ref["x_mode"], RTOL_X)
            assert close(got["marg_var"], ref["marg_var"], RTOL_V)


@pytest.mark.parametrize("case", ["mixed", "bta_prior"])
def test_static_scratch_other_layouts(pkg, case):
    # mixed precision on a block size that is a multiple of 128 carves the FP32
    # blocks and the TF32 hi / lo operand arrays of the tensor-core products out
    # of the static array; the BTA prior mode runs a second factorisation on it
    mdl = build("s", 3, 16 if case == "mixed" else 6, 2, 600, "gaussian", seed=4)
    th = torch.tensor(mdl.theta_true[None, :] + 0.05 * np.arange(3)[:, None], dtype=torch.float64, device="cuda")
    model = pkg.Model(mdl)
    kw = dict(grad="adjoint", want_mode=True, want_marg_var=True)
    kw.update(precision="mixed" if case == "mixed" else "fp64", prior="bta" if case == "bta_prior" else "kronecker")
    ref = model.eval(th, **kw)
    for _ in range(2):
        got = model.eval_static(th, **kw)
        torch.cuda.synchronize()
        assert torch.equal(got["status"], ref["status"]) and int(ref["status"].abs().sum()) == 0
        assert close(got["f"], ref["f"], RTOL_F)
        assert close(got["grad"], ref["grad"], RTOL_G)
        assert close(got["x_mode"], ref["x_mode"], RTOL_X)
        assert close(got["marg_var"], ref["marg_var"], RTOL_V)


def test_static_scratch_first_call_on_a_fresh_model_allocates_nothing(pkg):
    mdl = build("s", 3, 6, 2, 400, "gaussian", seed=6)
    th = torch.tensor(mdl.theta_true[None, :] + 0.05 * np.arange(2)[:, None], dtype=torch.float64, device="cuda")
    kw = dict(grad="adjoint", want_mode=True, want_marg_var=True)
    warm = pkg.Model(mdl)            # loads the kernels' code (lazy module loading) once per process
    out = warm.eval_static(th, **kw)
    torch.cuda.synchronize()
    warm.close()
    model = pkg.Model(mdl)           # the fresh model: its first evaluation is the static entry point
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    got = model.eval_static(th, out=out, **kw)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = model.eval(th, **kw)
    torch.cuda.synchronize()
    assert torch.equal(got["status"], ref["status"]) and int(ref["status"].abs().sum()) == 0
    assert close(got["f"], ref["f"], RTOL_F)
    assert close(got["marg_var"], ref["marg_var"], RTOL_V)


def test_static_scratch_rejects_a_batch_that_does_not_fit(pkg):
    mdl = build("big", 40, 32, 2, 5000, "gaussian")      # ~340 MB of workspace per point
    model = pkg.Model(mdl)
    th = torch.tensor(mdl.theta_true[None, :], dtype=torch.float64, device="cuda")
    o = pkg.make_opts()
    out = pkg.capi.inla_eval_out()
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    out.f_dev, out.status_dev = f.data_ptr(), st.data_ptr()
    code = model.lib.inla_eval_batch_static(model.handle, 1, ctypes.c_void_p(th.data_ptr()), ctypes.byref(o),
                                            ctypes.byref(out), None)
    assert code == pkg.capi.INLA_ERR_ARG
    assert "static array" in model.lib.inla_last_error().decode()
