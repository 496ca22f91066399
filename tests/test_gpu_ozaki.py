"""The FP64 product on the BF16 tensor cores (inla_gemm_f64, error-free digit
splitting) against exact products.

* Integer matrices whose products fit 53 bits are multiplied exactly (every
  digit product and every partial sum of the leading levels is an exact
  integer in the tensor cores' FP32 accumulators).
* Random FP64 matrices, with row and column magnitudes spread over 2^+-20:
  every entry within the stated bound K 2^(e_r + e_c - 50) + 2^-52 |C| of the
  product computed in extended precision on the host.
* A wait limit below 1 us makes every CTA give up at its first copy: status
  INLA_ERR_TIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2204_04678_gb300 as p
    p.build()
    return p


def exact_product(X, Y):
    """X Y^T in the host's extended precision (binary128 on aarch64, x87 80-bit on x86)."""
    return (X.astype(np.longdouble) @ Y.astype(np.longdouble).T)


def row_exponents(A):
    m = np.max(np.abs(A), axis=-1)
    return np.where(m > 0, np.frexp(m)[1], -1021)


@pytest.mark.parametrize("n,batch", [(128, 1), (256, 2), (384, 1)])
def test_integer_products_are_exact(pkg, n, batch):
    rng = np.random.default_rng(n)
    X = rng.integers(-1000, 1001, size=(batch, n, n)).astype(np.float64)
    Y = rng.integers(-1000, 1001, size=(batch, n, n)).astype(np.float64)
    X[:, 3, :] = 0.0                       # a zero row
    C, st = pkg.gemm_f64(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    ref = np.einsum("bik,bjk->bij", X.astype(np.int64), Y.astype(np.int64))
    assert np.array_equal(C.cpu().numpy(), ref.astype(np.float64))


@pytest.mark.parametrize("n,batch,spread", [(128, 2, 0), (256, 1, 20), (512, 1, 8)])
def test_random_products_within_the_stated_bound(pkg, n, batch, spread):
    rng = np.random.default_rng(7 + n)
    X = rng.standard_normal((batch, n, n))
    Y = rng.standard_normal((batch, n, n))
    if spread:
        X *= 2.0 ** rng.integers(-spread, spread + 1, size=(batch, n, 1))
        Y *= 2.0 ** rng.integers(-spread, spread + 1, size=(batch, n, 1))
        X *= 2.0 ** rng.integers(-spread, spread + 1, size=(batch, 1, n))   # magnitudes vary along K too
    C, st = pkg.gemm_f64(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"))
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    C = C.cpu().numpy()
    for b in range(batch):
        ref = exact_product(X[b], Y[b])
        er, ec = row_exponents(X[b]), row_exponents(Y[b])
        bound = n * 2.0 ** (er[:, None] + ec[None, :] - 50) + 2.0 ** -52 * np.abs(ref).astype(np.float64)
        err = np.abs((C[b] - ref).astype(np.float64))
        assert np.all(err <= bound), float(np.max(err / bound))
        if spread:
            continue
        # with row magnitudes of one order the error is of the order of an FP64 product's
        d = torch.tensor(X[b], device="cuda") @ torch.tensor(Y[b], device="cuda").T
        e64 = np.abs((d.cpu().numpy() - ref).astype(np.float64))
        scale = np.abs(X[b]) @ np.abs(Y[b]).T
        assert np.max(err / scale) <= 64 * max(np.max(e64 / scale), 2.0 ** -53)


def test_wait_limit_times_out_every_product(pkg):
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.standard_normal((2, 256, 256)), device="cuda")
    lib = pkg.capi.load()
    try:
        pkg.capi.check(lib.inla_set_wait_limit(1e-9))
        C, st = pkg.gemm_f64(X, X)
        torch.cuda.synchronize()
    finally:
        pkg.capi.check(lib.inla_set_wait_limit(2.0))
    assert np.all(st.cpu().numpy() == pkg.capi.INLA_ERR_TIMEOUT)
    C, st = pkg.gemm_f64(X, X)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    ref = (X.double() @ X.double().transpose(1, 2)).cpu().numpy()
    assert np.allclose(C.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
