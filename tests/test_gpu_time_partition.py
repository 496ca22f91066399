"""Nested dissection of the time chain (Sec. 3.3): every factorisation splits
the chain at its middle block into two independent elimination chains on two
streams, and the block substitution and the selected inversion follow the split
order (the separator first on the way back).  The split order reaches the same f,
mode, marginal variances and gradient as the one-chain order (the oracle's), up
to rounding: held to the FP64 tolerances of the parity tests, and to a few ulps'
worth against the one-chain path.
"""
import numpy as np
import pytest

from synth import build, fd_stencil
from oracle import bta, fd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_F, RTOL_X, RTOL_V, RTOL_G = 1e-10, 1e-9, 1e-9, 1e-8
MIX_F, MIX_X = 1e-6, 1e-9


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def thetas(mdl, k, seed, counts=False):
    rng = np.random.default_rng(seed)
    th = mdl.theta_true[None, :] + 0.15 * rng.standard_normal((k, 4))
    if counts:
        th[:, 0] = np.log(np.array([1e-3, 0.1, 1.0, 10.0]))[:k]
    return th


def both(model, th, **kw):
    model.set_time_partition(1)
    one = model.eval(cuda(th), **kw)
    model.set_time_partition(2)
    two = model.eval(cuda(th), **kw)
    torch.cuda.synchronize()
    return one, two


# (n_t, nx, n_b, m): odd and even n_t (chains of equal and unequal length), the
# shortest split chain (n_t = 3: one block each side), no fixed effects, ragged
# tiles, and n_s = 625 (padded to 640 = 5 x 128: the blocked inversion with its
# products on the tensor cores, in both chains at once)
CASES = [(3, 4, 0, 60), (3, 8, 2, 400), (4, 10, 3, 600), (5, 13, 2, 1500), (8, 6, 1, 500), (5, 25, 2, 2500)]


@pytest.mark.parametrize("n_t,nx,n_b,m", CASES)
def test_gaussian_split_chain_matches_oracle(pkg, n_t, nx, n_b, m):
    mdl = build("tp", n_t, nx, n_b, m, "gaussian", seed=n_t * nx)
    th = thetas(mdl, 3, seed=n_t)
    model = pkg.Model(mdl)
    one, two = both(model, th, grad="adjoint", want_mode=True, want_marg_var=True)
    for b in range(th.shape[0]):
        ref = bta.gaussian(mdl, th[b], want_grad=True, want_var=True)
        assert int(two["status"][b]) == 0
        f = float(two["f"][b])
        assert abs(f - ref["f"]) <= RTOL_F * abs(ref["f"]), (f, ref["f"])
        x = two["x_mode"][b].cpu().numpy()
        assert np.abs(x - ref["x"]).max() <= RTOL_X * np.abs(ref["x"]).max()
        v = two["marg_var"][b].cpu().numpy()
        assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= RTOL_V
        g = two["grad"][b].cpu().numpy()
        assert np.abs(g - ref["grad"]).max() <= RTOL_G * max(1.0, np.abs(ref["grad"]).max()), (g, ref["grad"])
        # against the one-chain order on the same GPU
        assert abs(f - float(one["f"][b])) <= 1e-12 * abs(f)
        x1 = one["x_mode"][b].cpu().numpy()
        assert np.abs(x - x1).max() <= 1e-11 * np.abs(x1).max()
        v1 = one["marg_var"][b].cpu().numpy()
        assert np.max(np.abs(v - v1) / v1) <= 1e-11
        g1 = one["grad"][b].cpu().numpy()
        assert np.abs(g - g1).max() <= 1e-10 * max(1.0, np.abs(g1).max())


@pytest.mark.parametrize("lik", ["poisson", "binomial", "negbinomial"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_newton_iterations_on_split_chains_match_oracle(pkg, lik, use_graph):
    # every Newton iteration factorises and solves on the two chains, and the adjoint's
    # selected inversion and solve at the mode follow; in a graph the loop body (a
    # conditional while-node) forks the second chain from streams of its own
    mdl = build("tpn", 5, 6, 2, 500, lik, seed=21)
    th = thetas(mdl, 4, seed=6, counts=True)
    model = pkg.Model(mdl)
    refs = [bta.evaluate(mdl, t, want_grad=True, want_var=True) for t in th]
    for rep in range(2 if use_graph else 1):   # capture, then replay
        r = model.eval(cuda(th), grad="adjoint", want_mode=True, want_marg_var=True, use_graph=use_graph)
        torch.cuda.synchronize()
        for b, ref in enumerate(refs):
            assert int(r["status"][b]) == 0, (lik, b)
            assert abs(float(r["f"][b]) - ref["f"]) <= RTOL_F * abs(ref["f"])
            x = r["x_mode"][b].cpu().numpy()
            assert np.abs(x - ref["x"]).max() <= RTOL_X * np.abs(ref["x"]).max()
            v = r["marg_var"][b].cpu().numpy()
            assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= RTOL_V
            g = r["grad"][b].cpu().numpy()
            assert np.abs(g - ref["grad"]).max() <= RTOL_G * max(1.0, np.abs(ref["grad"]).max())
            assert abs(int(r["newton_iters"][b]) - ref["iters"]) <= 1


def test_fd_stencil_on_split_chains_matches_oracle(pkg):
    mdl = build("tpf", 6, 9, 2, 800, "gaussian", seed=4)
    th = thetas(mdl, 2, seed=8)
    model = pkg.Model(mdl)
    one, two = both(model, th, grad="fd")
    for b in range(th.shape[0]):
        fs = [bta.gaussian(mdl, p)["f"] for p in fd_stencil(th[b])]
        assert abs(float(two["f"][b]) - fs[0]) <= RTOL_F * abs(fs[0])
        # differences of f values that agree to 1e-10 relative, divided by 2 eps
        g = two["grad"][b].cpu().numpy()
        assert np.abs(g - fd.gradient_from_stencil(fs)).max() <= 2 * RTOL_F * abs(fs[0]) / 1e-3
        assert np.abs(g - one["grad"][b].cpu().numpy()).max() <= 2e-12 * abs(fs[0]) / 1e-3


@pytest.mark.parametrize("blocked", [False, True])
def test_mixed_precision_split_chain(pkg, blocked):
    # FP32 blocks on both chains (block sweep, or the blocked inversion with 3xTF32
    # products on the tensor cores), the mode refined with FP64 residuals of the split solve
    mdl = build("tpm", 7, 25, 2, 2500, "gaussian", seed=17)
    th = thetas(mdl, 2, seed=9)
    model = pkg.Model(mdl)
    if blocked:
        model.set_tiles(32, pkg.capi.INLA_INV_BLOCKED, pkg.capi.INLA_GEMM_TF32X3)
    one, two = both(model, th, grad="none", want_mode=True, precision="mixed")
    for b in range(th.shape[0]):
        ref = bta.gaussian(mdl, th[b])
        assert int(two["status"][b]) == 0
        assert abs(float(two["f"][b]) - ref["f"]) <= MIX_F * abs(ref["f"])
        x = two["x_mode"][b].cpu().numpy()
        assert np.abs(x - ref["x"]).max() <= MIX_X * np.abs(ref["x"]).max()


def test_prior_factorisation_on_split_chains(pkg):
    # log|Q| by the block factorisation of the prior (no selected inversion after it)
    mdl = build("tpq", 5, 9, 2, 500, "gaussian", seed=5)
    th = thetas(mdl, 2, seed=3)
    model = pkg.Model(mdl)
    k = model.eval(cuda(th), grad="fd", prior="kronecker")
    b = model.eval(cuda(th), grad="fd", prior="bta")
    torch.cuda.synchronize()
    fk, fb = k["f"].cpu().numpy(), b["f"].cpu().numpy()
    assert np.all(np.abs(fk - fb) <= RTOL_F * np.abs(fk))


def test_mixed_adjoint_on_split_chains(pkg):
    # FP32 selected inversion with 3xTF32 products on the tensor cores on both chains
    mdl = build("tpa", 5, 25, 2, 2500, "gaussian", seed=19)
    th = thetas(mdl, 2, seed=2)
    model = pkg.Model(mdl)
    one, two = both(model, th, grad="adjoint", want_marg_var=True, precision="mixed")
    for b in range(th.shape[0]):
        ref = bta.gaussian(mdl, th[b], want_grad=True, want_var=True)
        assert int(two["status"][b]) == 0
        assert abs(float(two["f"][b]) - ref["f"]) <= MIX_F * abs(ref["f"])
        g = two["grad"][b].cpu().numpy()
        assert np.abs(g - ref["grad"]).max() <= 1e-5 * max(1.0, np.abs(ref["grad"]).max())
        v = two["marg_var"][b].cpu().numpy()
        assert np.max(np.abs(v - ref["var"]) / ref["var"]) <= 5e-5


def test_workspace_holds_a_second_chain(pkg):
    mdl = build("tpw", 4, 9, 2, 500, "gaussian", seed=2)
    model = pkg.Model(mdl)
    model.set_time_partition(1)
    w1 = [model.workspace_bytes(2, grad=g) for g in ("fd", "adjoint")]
    model.set_time_partition(2)
    w2 = [model.workspace_bytes(2, grad=g) for g in ("fd", "adjoint")]
    assert all(b > a for a, b in zip(w1, w2))
    with pytest.raises(Exception):
        model.set_time_partition(3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_point_groups_are_bit_identical(pkg, precision):
    # two point groups (first and second half of the wave) factorised concurrently on two
    # stream pairs: every point's arithmetic is the one-group arithmetic, eager and in a graph
    mdl = build("tpg", 6, 9, 2, 800, "gaussian", seed=8)
    th = thetas(mdl, 3, seed=4)
    model = pkg.Model(mdl)
    # the groups run inside CUDA graphs; eager calls keep one group
    for kw in (dict(grad="fd", use_graph=True), dict(grad="none", want_mode=True, use_graph=True),
               dict(grad="adjoint", want_marg_var=True, use_graph=True)):
        model.set_point_groups(1)
        a = model.eval(cuda(th), precision=precision, **kw)
        model.set_point_groups(2)
        b = model.eval(cuda(th), precision=precision, **kw)
        torch.cuda.synchronize()
        for key in ("f", "grad", "x_mode", "marg_var", "status"):
            if key in a:
                assert torch.equal(a[key], b[key]), (kw, key)
    with pytest.raises(Exception):
        model.set_point_groups(3)

