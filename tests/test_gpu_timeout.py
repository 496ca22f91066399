"""Failure detection without a GPU fault: the tensor-core kernels' bounded
waits for their own asynchronous copies and products.

With the wait limit set below 1 us every wait is a single non-blocking test,
which the first TMA copy of each tile cannot pass, so every CTA of the mixed
selected inversion's 3xTF32 product gives up: the points must come back as
INLA_ERR_TIMEOUT (f = +inf, NaN gradient and variances), the kernels must
have waited for their copies in flight before releasing their memory, and the
context must stay usable -- the same call with the default limit reproduces
the earlier results bit for bit.
"""
import math

import numpy as np
import pytest

from synth import build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def test_wait_limit_marks_points_timed_out(pkg):
    # n_s = 256: the padded block size is a multiple of 128, so the mixed selected
    # inversion's products run on the tensor cores with TMA-fed operands
    mdl = build("t", 3, 16, 2, 600, "gaussian", seed=5)
    th = torch.tensor(mdl.theta_true[None, :] + 0.05 * np.arange(3)[:, None], dtype=torch.float64, device="cuda")
    model = pkg.Model(mdl)
    kw = dict(grad="adjoint", want_marg_var=True, precision="mixed")
    ok = model.eval(th, **kw)
    torch.cuda.synchronize()
    assert int(ok["status"].abs().sum()) == 0
    lib = pkg.capi.load()
    try:
        pkg.capi.check(lib.inla_set_wait_limit(1e-9))
        r = model.eval(th, **kw)
        torch.cuda.synchronize()
    finally:
        pkg.capi.check(lib.inla_set_wait_limit(2.0))
    st = r["status"].cpu().numpy()
    assert np.all(st == pkg.capi.INLA_ERR_TIMEOUT), st
    assert all(math.isinf(float(v)) for v in r["f"].cpu())
    assert np.isnan(r["grad"].cpu().numpy()).all()
    assert np.isnan(r["marg_var"].cpu().numpy()).all()
    again = model.eval(th, **kw)
    torch.cuda.synchronize()
    for k in ("f", "grad", "marg_var", "status"):
        assert torch.equal(again[k], ok[k]), k


def test_wait_limit_rejects_invalid_values(pkg):
    lib = pkg.capi.load()
    for v in (0.0, -1.0, 2.5, float("nan")):
        assert lib.inla_set_wait_limit(v) == pkg.capi.INLA_ERR_ARG
    assert lib.inla_set_wait_limit(2.0) == pkg.capi.INLA_OK
