"""The 3xTF32 tensor-core GEMM (tcgen05, kind::tf32) of the mixed selected
inversion: the product itself against an FP64 product of the same FP32
inputs, and the mixed evaluation with it against the oracle."""
import numpy as np
import pytest

from synth import Stream, build, config_model, fd_stencil, theta_batch
from oracle import bta

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX_F, MIX_G, MIX_X, MIX_V = 1e-6, 1e-5, 1e-9, 5e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def _tf32_rna(a):
    """Round FP32 values to TF32 (10 explicit mantissa bits), to nearest with
    ties away from zero, by integer arithmetic on the bit patterns."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("n,batch", [(128, 1), (256, 3), (1024, 2)])
def test_product_against_fp64(pkg, n, batch):
    s = Stream(21 + n, 0)
    X = s.normal(batch * n * n).reshape(batch, n, n).astype(np.float32)
    Y = s.normal(batch * n * n).reshape(batch, n, n).astype(np.float32)
    C, st = pkg.gemm_tf32x3(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    ref = np.einsum("bik,bjk->bij", X.astype(np.float64), Y.astype(np.float64))
    err = np.abs(C.cpu().numpy().astype(np.float64) - ref).max()
    scale = np.sqrt(n)                              # |C_ij| ~ sqrt(n) for unit normals
    # FP32 level: the split leaves ~2^-22 per product, the stage sums ~2^-24
    # each; sqrt(n) random terms of either kind stay below 1e-6 sqrt(n) |C_ij|
    assert err <= 1e-6 * scale * scale, err
    # a single TF32 product (no lo terms) is ~2^-11 relative: the split must beat it by far
    one = np.einsum("bik,bjk->bij", _tf32_rna(X).astype(np.float64), _tf32_rna(Y).astype(np.float64))
    assert err < np.abs(one - ref).max() / 50


def test_identity_times_transpose_is_exact_layout(pkg):
    """X = I gives C = Y^T: every entry lands in its own place (swizzle and
    TMEM lane/column mapping), equal to Y_hi + Y_lo (error <= 2^-21 |y|)."""
    n = 256
    s = Stream(5, 0)
    Y = s.normal(n * n).reshape(n, n).astype(np.float32)
    X = np.eye(n, dtype=np.float32)
    C, st = pkg.gemm_tf32x3(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    c = C.cpu().numpy()
    assert np.all(np.abs(c - Y.T) <= 2.0 ** -21 * np.abs(Y.T) + 1e-30)


def test_invalid_sizes_rejected(pkg):
    from paper_2204_04678_gb300 import capi
    X = torch.zeros(2, 100, 100, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.InlaError):
        pkg.gemm_tf32x3(X, X)


def _mixed_vs_oracle(pkg, mdl, th, gemm, sweep=64):
    model = pkg.Model(mdl)
    try:
        model.set_tiles(32, sweep, gemm)
        r = model.eval(torch.tensor(th, dtype=torch.float64, device="cuda"), grad="adjoint", precision="mixed",
                       want_mode=True, want_marg_var=True)
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
    finally:
        model.close()


@pytest.mark.parametrize("lik", ["gaussian", "poisson"])
def test_mixed_with_tensor_gemm_matches_oracle(pkg, lik):
    from paper_2204_04678_gb300 import capi
    mdl = build("tc", 3, 16, 2, 1500, lik, seed=3)        # n_s = 256: two 128-wide tiles per block side
    th = mdl.theta_true[None, :] + np.array([[0.0, 0.0, 0.0, 0.0], [0.1, -0.1, 0.05, -0.2]])
    _mixed_vs_oracle(pkg, mdl, th, capi.INLA_GEMM_TF32X3)


@pytest.mark.parametrize("lik,nx", [("gaussian", 16), ("poisson", 16), ("gaussian", 23)])
def test_mixed_blocked_inverse_matches_oracle(pkg, lik, nx):
    # n_s = 256 and 529 (padded to 256 and 640): D_t^-1 by the block recursion with
    # 3xTF32 tensor-core products (one and two levels above the 128 x 128 base blocks)
    from paper_2204_04678_gb300 import capi
    mdl = build("tb", 3, nx, 2, 1500, lik, seed=5)
    th = mdl.theta_true[None, :] + np.array([[0.0, 0.0, 0.0, 0.0], [0.1, -0.1, 0.05, -0.2]])
    _mixed_vs_oracle(pkg, mdl, th, capi.INLA_GEMM_TF32X3, sweep=capi.INLA_INV_BLOCKED)


def test_mixed_tensor_gemm_full_size_config2(pkg):
    """n_t = 50, 32 x 32 grid, m = 100 000: the stencil batch with the tensor-core
    GEMM against the FP64 path (which matches the oracle to 1e-10)."""
    from paper_2204_04678_gb300 import capi
    mdl = config_model(2)
    model = pkg.Model(mdl)
    try:
        th = torch.tensor(fd_stencil(theta_batch(2, mdl)[0]), dtype=torch.float64, device="cuda")
        d = model.eval(th, grad="adjoint", precision="fp64")
        model.set_tiles(32, 64, capi.INLA_GEMM_TF32X3)
        m = model.eval(th, grad="adjoint", precision="mixed")
        torch.cuda.synchronize()
        assert int(m["status"].abs().sum()) == 0
        fd, fm = d["f"].cpu().numpy(), m["f"].cpu().numpy()
        assert np.all(np.abs(fm - fd) <= MIX_F * np.abs(fd))
        gd, gm = d["grad"].cpu().numpy(), m["grad"].cpu().numpy()
        assert np.abs(gm - gd).max() <= MIX_G * max(1.0, np.abs(gd).max())
    finally:
        model.close()


@pytest.mark.parametrize("lik,nx", [("gaussian", 16), ("poisson", 16), ("binomial", 16), ("gaussian", 23)])
def test_mixed_with_tensor_sweep_matches_oracle(pkg, lik, nx):
    """The rank-64 updates of the FP32 block sweep on the tensor cores: n_s = 256
    gives four 64-wide pivots and two 128-wide tensor tiles per block side (the
    masks for the pivot row and column and the next pivot cross tile borders);
    n_s = 529 (n_p = 576, not a multiple of 128) takes the CUDA-core sweep."""
    from paper_2204_04678_gb300 import capi
    mdl = build("tcs", 3, nx, 2, 1500, lik, seed=4)
    th = mdl.theta_true[None, :] + np.array([[0.0, 0.0, 0.0, 0.0], [0.1, -0.1, 0.05, -0.2]])
    _mixed_vs_oracle(pkg, mdl, th, capi.INLA_GEMM_TF32X3, sweep=capi.INLA_SWEEP_TF32X3)


def test_tensor_sweep_full_size_config2(pkg):
    """n_t = 50, 32 x 32 grid: the mixed path with the tensor-core sweep against
    the FP64 path and against the mixed path with the CUDA-core sweep."""
    from paper_2204_04678_gb300 import capi
    mdl = config_model(2)
    model = pkg.Model(mdl)
    try:
        th = torch.tensor(fd_stencil(theta_batch(2, mdl)[0]), dtype=torch.float64, device="cuda")
        d = model.eval(th, grad="adjoint", precision="fp64", want_marg_var=True)
        model.set_tiles(32, capi.INLA_SWEEP_TF32X3, capi.INLA_GEMM_TF32X3)
        t = model.eval(th, grad="adjoint", precision="mixed", want_marg_var=True)
        model.set_tiles(32, 64, capi.INLA_GEMM_TF32X3)
        c = model.eval(th, grad="adjoint", precision="mixed", want_marg_var=True)
        torch.cuda.synchronize()
        fd_, ft, fc = (o["f"].cpu().numpy() for o in (d, t, c))
        assert np.all(t["status"].cpu().numpy() == 0)
        assert np.all(np.abs(ft - fd_) <= MIX_F * np.abs(fd_))
        assert np.all(np.abs(ft - fc) <= MIX_F * np.abs(fd_))
        gd, gt = d["grad"].cpu().numpy(), t["grad"].cpu().numpy()
        assert np.abs(gt - gd).max() <= MIX_G * max(1.0, np.abs(gd).max())
        vd, vt = d["marg_var"].cpu().numpy(), t["marg_var"].cpu().numpy()
        assert np.max(np.abs(vt - vd) / vd) <= MIX_V
    finally:
        model.close()


def test_split_product_matches_the_oracle_emulation(pkg):
    """Against the oracle's emulation of the 3xTF32 split (oracle.tf32): bit for
    bit on integer matrices (TF32 values whose partial sums stay below 2^24, so
    no step of the product rounds), and within FP32 accumulation error of the
    emulated split product on random FP32 matrices."""
    from oracle import tf32
    s = Stream(77, 0)
    n, batch = 256, 2
    Xi = (s.integers(batch * n * n, 65) - 32).reshape(batch, n, n).astype(np.float32)
    Yi = (s.integers(batch * n * n, 65) - 32).reshape(batch, n, n).astype(np.float32)
    C, st = pkg.gemm_tf32x3(torch.tensor(Xi, device="cuda"), torch.tensor(Yi, device="cuda"))
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    emu = tf32.product_3xtf32(Xi, Yi)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), emu)
    X = s.normal(batch * n * n).reshape(batch, n, n).astype(np.float32)
    Y = s.normal(batch * n * n).reshape(batch, n, n).astype(np.float32)
    C, st = pkg.gemm_tf32x3(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    torch.cuda.synchronize()
    absprod = np.einsum("bik,bjk->bij", np.abs(X.astype(np.float64)), np.abs(Y.astype(np.float64)))
    err = np.abs(C.cpu().numpy().astype(np.float64) - tf32.product_3xtf32(X, Y))
    assert np.all(err <= 2.0 ** -18 * absprod)
