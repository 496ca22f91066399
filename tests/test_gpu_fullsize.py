"""Parity with the CPU oracle on the benchmark workloads at full size.

The 32 x 32 model (n_t = 50, n_s = 1024, n_b = 4, m = 100 000) at full size:
f, x*, every marginal variance and the adjoint gradient in FP64; the FD
gradient against central differences of oracle f values; the mixed form
against the oracle (not against the GPU's FP64 path).  The larger models are
run at full mesh, n_b and likelihood with fewer time steps (the oracle's dense
per-block factorisations of 2025 x 2025 to 4096 x 4096 blocks take tens of
seconds per time step on the host, times the Newton iterations for Poisson
data): 45 x 45 with n_t = 20, 50 x 50 with n_t = 12 and 64 x 64 Poisson with
n_t = 2, observations per time step as in the full workloads.  The oracle jobs run in a spawn process pool started before the
first GPU call of this module, in parallel with the GPU work.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle_jobs as J
from synth import fd_stencil

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F, RTOL_X, RTOL_V, RTOL_G = 1e-10, 1e-9, 1e-9, 1e-8
MIX_F, MIX_G, MIX_X, MIX_V = 1e-6, 1e-5, 1e-9, 5e-5
ORACLE_WAIT = 1500


@pytest.fixture(scope="module")
def oracle():
    """Oracle results, computed asynchronously: {name: AsyncResult}.  The largest
    case (64 x 64 blocks) gets a worker with four BLAS threads of its own."""
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    # the workers import numpy before any initializer runs, so their BLAS thread
    # counts come from the environment they are started with
    saved = {v: os.environ.get(v) for v in J.BLAS_ENV}
    try:
        J.set_threads(min(4, cores))
        big = ctx.Pool(1)
        J.set_threads(1)
        small = ctx.Pool(max(1, min(12, cores - 4)))
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    jobs = {"c5s": big.apply_async(J.evaluate, ("c5s", J.centre("c5s"), True))}
    for key in ("c2", "c3s", "c4s"):
        jobs[key] = small.apply_async(J.evaluate, (key, J.centre(key), True))
    for k, p in enumerate(fd_stencil(J.centre("c2"))):
        jobs[f"c2_fd{k}"] = small.apply_async(J.evaluate, ("c2", p, False))
    yield jobs
    for pool in (big, small):
        pool.terminate()
        pool.join()


@pytest.fixture(scope="module")
def pkg(oracle):
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def check(r, ref, tf, tx, tv, tg, b=0):
    assert int(r["status"][b]) == 0
    f = float(r["f"][b])
    assert abs(f - ref["f"]) <= tf * abs(ref["f"]), (f, ref["f"])
    x = r["x_mode"][b].cpu().numpy()
    assert np.abs(x - ref["x"]).max() <= tx * np.abs(ref["x"]).max()
    v = r["marg_var"][b].cpu().numpy()
    assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= tv
    g = r["grad"][b].cpu().numpy()
    assert np.abs(g - ref["grad"]).max() <= tg * max(1.0, np.abs(ref["grad"]).max()), (g, ref["grad"])


@pytest.mark.parametrize("key", ["c2", "c3s", "c4s", "c5s"])
def test_fp64_adjoint_matches_oracle(pkg, oracle, key):
    """f, x*, all of diag(Q_c^-1) and the adjoint gradient, FP64."""
    model = pkg.Model(J.model(key))
    r = model.eval(cuda(J.centre(key)[None]), grad="adjoint", want_mode=True, want_marg_var=True)
    torch.cuda.synchronize()
    check(r, oracle[key].get(ORACLE_WAIT), RTOL_F, RTOL_X, RTOL_V, RTOL_G)


@pytest.mark.parametrize("key", ["c2", "c3s", "c4s", "c5s"])
def test_mixed_matches_oracle(pkg, oracle, key):
    """The mixed form's error against the FP64 oracle, within its stated budget."""
    model = pkg.Model(J.model(key))
    r = model.eval(cuda(J.centre(key)[None]), grad="adjoint", want_mode=True, want_marg_var=True, precision="mixed")
    torch.cuda.synchronize()
    check(r, oracle[key].get(ORACLE_WAIT), MIX_F, MIX_X, MIX_V, MIX_G)


def test_fd_gradient_full_size_config2(pkg, oracle):
    """The benchmark step itself: FD gradient of the 9-point stencil against central
    differences of the oracle's f at the same 9 points."""
    model = pkg.Model(J.model("c2"))
    c = J.centre("c2")
    r = model.eval(cuda(c[None]), grad="fd")
    torch.cuda.synchronize()
    fo = np.array([oracle[f"c2_fd{k}"].get(ORACLE_WAIT)["f"] for k in range(9)])
    pts = fd_stencil(c)
    g_ref = np.array([(fo[1 + 2 * j] - fo[2 + 2 * j]) / (pts[1 + 2 * j][j] - pts[2 + 2 * j][j]) for j in range(4)])
    assert abs(float(r["f"][0]) - fo[0]) <= RTOL_F * abs(fo[0])
    g = r["grad"][0].cpu().numpy()
    assert np.abs(g - g_ref).max() <= 2 * RTOL_F * np.abs(fo).max() / 1e-3, (g, g_ref)
