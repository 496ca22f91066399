"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, brute force, textbook identities, library routines, invariants and
the worked example the paper prints (Fig. arrowhead_matrices).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from scipy import stats

from synth import build, config_model, fd_stencil
from oracle import bta, dense, fd, scalar
from oracle import model as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(n_t=3, nx=4, n_b=2, m=150, lik="gaussian", seed=0):
    return build("small", n_t, nx, n_b, m, lik, seed=seed)


def read_patterns(path):
    pats, name, rows = {}, None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if set(line) <= set("x."):
            rows.append([c == "x" for c in line])
        else:
            if name:
                pats[name] = np.array(rows)
            name, rows = line, []
    pats[name] = np.array(rows)
    return pats


def random_spd_with_pattern(pattern, rng):
    n = pattern.shape[0]
    Q = np.where(pattern, rng.uniform(-1, 1, (n, n)), 0.0)
    Q = np.tril(Q) + np.tril(Q, -1).T
    np.fill_diagonal(Q, 0.0)
    Q += np.diag(np.abs(Q).sum(1) + 1.0)       # strictly diagonally dominant
    return Q


# ---------------------------------------------------------------- Fig. arrowhead

def test_arrowhead_fill_matches_paper_figure():
    pats = read_patterns(os.path.join(GOLDEN, "arrowhead_fill.txt"))
    rng = np.random.default_rng(1)
    for q, l in (("Q1", "L1"), ("Q2", "L2")):
        Q = random_spd_with_pattern(pats[q], rng)
        assert np.array_equal(Q != 0, pats[q])
        assert np.array_equal(scalar.fill_pattern(Q), pats[l])
        assert np.array_equal(np.linalg.cholesky(Q) != 0, pats[l])


def test_bta_pattern_has_no_fill_with_arrow_last():
    mdl = small(n_t=3, nx=3, n_b=2, m=80)
    A = M.obs_matrix(mdl)
    Qc = (M.prior_Q(mdl, mdl.theta_true) + math.exp(1.0) * (A.T @ A)).toarray()
    blocks, outside = bta.from_sparse(sp.csr_matrix(Qc), mdl.n_t, mdl.n_s, mdl.n_b)
    assert outside == 0
    L = np.linalg.cholesky(Qc)
    Lb, out_L = bta.from_sparse(sp.csr_matrix(np.where(np.abs(L) > 0, L, 0.0) + np.tril(L, -1).T),
                                mdl.n_t, mdl.n_s, mdl.n_b)
    assert out_L == 0
    # arrow first: the fixed effects couple every block, the factor fills in
    n, nb = mdl.n, mdl.n_b
    perm = np.r_[np.arange(n - nb, n), np.arange(n - nb)]
    Lf = np.linalg.cholesky(Qc[np.ix_(perm, perm)])
    lower = np.tril(np.ones((n, n), bool))
    assert np.count_nonzero(Lf[lower] == 0.0) < 0.01 * lower.sum()


# ---------------------------------------------------------------- model pieces

def test_ar1_precision_inverts_to_geometric_correlation():
    for n_t, rho in ((1, 0.3), (2, 0.5), (7, 0.82)):
        Qt = M.temporal_Q(n_t, rho).toarray()
        i = np.arange(n_t)
        R = rho ** np.abs(i[:, None] - i[None, :])
        assert np.allclose(np.linalg.inv(Qt), R, rtol=1e-12, atol=1e-12)
        assert np.isclose(np.linalg.slogdet(Qt)[1], -(n_t - 1) * math.log(1 - rho * rho), atol=1e-12)


def test_spatial_precision_coefficients():
    mdl = small(nx=6)
    th = np.array([0.0, -0.7, 0.3, 0.0])
    h = M.hyper(th)
    Qs = M.spatial_Q(mdl, th).toarray()
    C, G = (x.toarray() for x in M.fem_matrices(mdl))
    # G 1 = 0, so Q_s 1 = tau^2 kappa^4 C 1 and the total is kappa^2 / (4 pi sigma^2)
    assert np.isclose(Qs.sum(), h["kappa"] ** 2 / (4 * math.pi * h["sigma"] ** 2), rtol=1e-11)
    # factored form (kappa^2 C + G) C^-1 (kappa^2 C + G) of the alpha = 2 operator
    K = h["kappa"] ** 2 * C + G
    assert np.allclose(Qs, h["tau2"] * K @ np.linalg.inv(C) @ K, rtol=1e-11, atol=1e-9)


def test_spde_marginal_variance_is_sigma_squared_in_interior():
    # Matern nu = 1 in 2-D: marginal variance 1/(4 pi kappa^2 tau^2) = sigma^2
    mdl = build("fine", 1, 41, 0, 10)
    sigma = 1.3
    th = np.array([0.0, math.log(0.25), math.log(sigma), 0.0])
    v = np.diag(np.linalg.inv(M.spatial_Q(mdl, th).toarray())).reshape(41, 41)
    assert abs(v[20, 20] / sigma ** 2 - 1.0) < 0.12


def test_log_prior_and_poisson_loglik_match_scipy():
    mdl = small(lik="poisson")
    th = np.array([-6.0, -1.2, 0.4, 2.0])
    ref = stats.norm.logpdf(th, mdl.prior_mean, mdl.prior_sd).sum()
    assert np.isclose(M.log_prior(mdl, th), ref, rtol=1e-14)
    eta = np.linspace(-1, 1, mdl.m)
    ref = stats.poisson.logpmf(mdl.y, mdl.E * np.exp(eta)).sum()
    assert np.isclose(M.poisson_loglik(mdl, eta), ref, rtol=1e-12)


def test_binomial_loglik_matches_scipy_and_its_derivatives_are_b_prime():
    mdl = small(lik="binomial")
    eta = np.linspace(-3, 3, mdl.m)
    ref = stats.binom.logpmf(mdl.y, mdl.E, 1.0 / (1.0 + np.exp(-eta))).sum()
    assert np.isclose(M.binomial_loglik(mdl, eta), ref, rtol=1e-12)
    # b(eta) = N log(1 + e^eta): mean, weight and third derivative by central differences
    for lik in ("binomial", "poisson"):
        mdl = small(lik=lik)
        b = (lambda e: mdl.E * np.logaddexp(0.0, e)) if lik == "binomial" else (lambda e: mdl.E * np.exp(e))
        h = 1e-4
        mean, wgt, third = M.glm_terms(mdl, eta)
        assert np.allclose(mean, (b(eta + h) - b(eta - h)) / (2 * h), rtol=1e-7)
        assert np.allclose(wgt, (M.glm_terms(mdl, eta + h)[0] - M.glm_terms(mdl, eta - h)[0]) / (2 * h),
                           rtol=1e-6, atol=1e-9)
        assert np.allclose(third, (M.glm_terms(mdl, eta + h)[1] - M.glm_terms(mdl, eta - h)[1]) / (2 * h),
                           rtol=1e-6, atol=1e-9)


def test_negbinomial_loglik_matches_scipy_and_its_terms_are_derivatives():
    mdl = small(lik="negbinomial")
    eta = np.linspace(-2, 2, mdl.m)
    r = mdl.nb_size
    mu = mdl.E * np.exp(eta)
    ref = stats.nbinom.logpmf(mdl.y, r, r / (r + mu)).sum()
    assert np.isclose(M.negbinomial_loglik(mdl, eta), ref, rtol=1e-12)
    # (y - score, D, dD/deta) against central differences of the log-likelihood, observation by observation
    ll = lambda e: (stats.nbinom.logpmf(mdl.y, r, r / (r + mdl.E * np.exp(e))))
    h = 1e-4
    score = (ll(eta + h) - ll(eta - h)) / (2 * h)
    ymm, wgt, third = M.glm_terms(mdl, eta)
    assert np.allclose(mdl.y - ymm, score, rtol=1e-6, atol=1e-8)
    d2 = (ll(eta + h) - 2 * ll(eta) + ll(eta - h)) / h ** 2
    assert np.allclose(wgt, -d2, rtol=1e-4, atol=1e-6)
    assert np.all(wgt > 0)
    assert np.allclose(third, (M.glm_terms(mdl, eta + h)[1] - M.glm_terms(mdl, eta - h)[1]) / (2 * h),
                       rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("lik", ["gaussian", "poisson", "binomial", "negbinomial"])
def test_dQ_matches_finite_difference_of_Q(lik):
    mdl = small(lik=lik)
    th = mdl.theta_true + np.array([0.1, 0.05, -0.1, 0.2])
    eps = 1e-5
    for j in range(4):
        e = np.zeros(4); e[j] = eps
        num = (M.prior_Q(mdl, th + e) - M.prior_Q(mdl, th - e)).toarray() / (2 * eps)
        ana = M.dQ_dtheta(mdl, th, j).toarray()
        assert np.allclose(ana, num, rtol=1e-7, atol=1e-7 * np.abs(num).max() + 1e-12)


# ---------------------------------------------------------------- Sec. 2.4 log-det, solves

def test_logdet_three_ways_on_tiny_matrix():
    mdl = small(n_t=2, nx=3, n_b=1, m=40)
    A = M.obs_matrix(mdl)
    Qc = (M.prior_Q(mdl, mdl.theta_true) + 2.0 * (A.T @ A)).toarray()
    _, ld_chol = dense.chol_logdet(Qc)
    lu, piv = sla.lu_factor(Qc)
    ld_lu = float(np.sum(np.log(np.abs(np.diag(lu)))))
    ld_eig = float(np.sum(np.log(np.linalg.eigvalsh(Qc))))
    ld_el = 2 * float(np.sum(np.log(np.diag(scalar.cholesky(Qc)))))
    for v in (ld_lu, ld_eig, ld_el):
        assert np.isclose(ld_chol, v, rtol=1e-12, atol=1e-10)


def test_bta_factor_equals_dense_factor():
    mdl = small(n_t=3, nx=3, n_b=2, m=90)
    A = M.obs_matrix(mdl)
    Qc = (M.prior_Q(mdl, mdl.theta_true) + 3.0 * (A.T @ A)).tocsr()
    blocks, _ = bta.from_sparse(Qc, mdl.n_t, mdl.n_s, mdl.n_b)
    Lb, ld = bta.cholesky(blocks)
    L = scalar.cholesky(Qc.toarray())
    n_s, N = mdl.n_s, mdl.n_t * mdl.n_s
    for t in range(mdl.n_t):
        assert np.allclose(Lb.D[t], L[t * n_s:(t + 1) * n_s, t * n_s:(t + 1) * n_s], atol=1e-12)
        assert np.allclose(Lb.R[t], L[N:, t * n_s:(t + 1) * n_s], atol=1e-12)
        if t < mdl.n_t - 1:
            assert np.allclose(Lb.B[t], L[(t + 1) * n_s:(t + 2) * n_s, t * n_s:(t + 1) * n_s], atol=1e-12)
    assert np.allclose(Lb.T, L[N:, N:], atol=1e-12)
    assert np.isclose(ld, 2 * np.sum(np.log(np.diag(L))), rtol=1e-13)
    b = np.random.default_rng(0).normal(size=mdl.n)
    assert np.allclose(bta.solve(Lb, b), np.linalg.solve(Qc.toarray(), b), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n_t,k,n_b", [(3, 1, 2), (5, 2, 2), (6, 3, 1), (6, 1, 0), (7, 5, 2)])
def test_split_order_factor_is_the_dense_factor_of_the_permuted_matrix(n_t, k, n_b):
    # one level of nested dissection of the time chain (Sec. 3.3): the block algorithm
    # in the split order equals the dense Cholesky factor of Q_c with its time blocks
    # permuted into that order (no fill outside the pattern), and its log-determinant,
    # solve and selected inverse equal the dense definitions
    mdl = small(n_t=n_t, nx=3, n_b=n_b, m=40 * n_t, seed=n_t + k)
    A = M.obs_matrix(mdl)
    Qc = (M.prior_Q(mdl, mdl.theta_true) + 2.3 * (A.T @ A)).tocsr()
    blocks, _ = bta.from_sparse(Qc, mdl.n_t, mdl.n_s, mdl.n_b)
    F, ld = bta.cholesky_split(blocks, k)
    n_s, N = mdl.n_s, mdl.n_t * mdl.n_s
    order, nxt = bta.split_order(n_t, k)
    assert sorted(order) == list(range(n_t)) and order[-1] == k
    perm = np.concatenate([np.arange(t * n_s, (t + 1) * n_s) for t in order] + [np.arange(N, N + n_b)])
    Qd = Qc.toarray()
    Lp = np.linalg.cholesky(Qd[np.ix_(perm, perm)])
    pos = {t: i for i, t in enumerate(order)}
    blk = lambda i, j: Lp[i * n_s:(i + 1) * n_s, j * n_s:(j + 1) * n_s]
    for t in range(n_t):
        assert np.allclose(F.D[t], blk(pos[t], pos[t]), atol=1e-12)
        assert np.allclose(F.R[t], Lp[N:, pos[t] * n_s:(pos[t] + 1) * n_s], atol=1e-12)
        later = [u for u in range(n_t) if pos[u] > pos[t]]
        for u in later:
            want = F.C[t] if nxt[t] == u else 0.0
            assert np.allclose(blk(pos[u], pos[t]), want, atol=1e-12), (t, u)   # no fill
    if n_b:
        assert np.allclose(F.T, Lp[N:, N:], atol=1e-12)
    assert np.isclose(ld, np.linalg.slogdet(Qd)[1], rtol=1e-13)
    b = np.random.default_rng(1).normal(size=mdl.n)
    assert np.allclose(bta.solve_split(F, b), np.linalg.solve(Qd, b), rtol=1e-11, atol=1e-11)
    S = bta.selinv_split(F)
    Sinv, _ = bta.from_sparse(sp.csr_matrix(np.linalg.inv(Qd)), mdl.n_t, mdl.n_s, mdl.n_b)
    for t in range(n_t):
        assert np.allclose(S.D[t], Sinv.D[t], rtol=1e-10, atol=1e-12)
        assert np.allclose(S.R[t], Sinv.R[t], rtol=1e-10, atol=1e-12)
        if t < n_t - 1:
            assert np.allclose(S.B[t], Sinv.B[t], rtol=1e-10, atol=1e-12)
    if n_b:
        assert np.allclose(S.T, Sinv.T, rtol=1e-10, atol=1e-12)


def test_kronecker_logdet_identity():
    for n_t, nx, n_b in ((1, 4, 0), (5, 5, 3), (8, 6, 2)):
        mdl = build("k", n_t, nx, n_b, 20)
        th = np.array([0.5, -0.8, 0.2, 0.7])
        h = M.hyper(th)
        blocks, _ = bta.from_sparse(M.prior_Q(mdl, th), n_t, mdl.n_s, n_b)
        _, ld = bta.cholesky(blocks)
        ld_t = -(n_t - 1) * math.log(1 - h["rho"] ** 2)
        ld_s = np.linalg.slogdet(M.spatial_Q(mdl, th).toarray())[1]
        assert np.isclose(ld, mdl.n_s * ld_t + n_t * ld_s + n_b * math.log(h["tau_b"]), rtol=1e-12)


def test_backward_solve_samples_have_covariance_q_inverse():
    # Eq. backward_solve: x = L^-T z with Cov(z) = I has Cov(x) = L^-T L^-1 = Q^-1
    rng = np.random.default_rng(3)
    Q = random_spd_with_pattern(np.ones((6, 6), bool), rng)
    L = scalar.cholesky(Q)
    X = np.column_stack([scalar.backward_solve(L, e) for e in np.eye(6)])
    assert np.allclose(X @ X.T, np.linalg.inv(Q), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- Sec. 2.4.2 selected inversion

def test_scalar_recursions_equal_dense_inverse_and_each_other():
    mdl = small(n_t=2, nx=3, n_b=1, m=30)
    A = M.obs_matrix(mdl)
    Q = (M.prior_Q(mdl, mdl.theta_true) + (A.T @ A)).toarray()
    L = scalar.cholesky(Q)
    inv = np.linalg.inv(Q)
    S1, S2 = scalar.sel_inv_cov(L), scalar.takahashi(L)
    assert np.allclose(S1, inv, rtol=1e-11, atol=1e-13)
    assert np.allclose(S2, inv, rtol=1e-11, atol=1e-13)
    # selected: only the pattern of L is computed, and it equals the same entries of the inverse
    P1, P2 = scalar.sel_inv_cov(L, selected=True), scalar.takahashi(L, selected=True)
    need = np.isfinite(P1)
    assert np.array_equal(need, np.isfinite(P2))
    assert np.array_equal(need, (L != 0) | (L.T != 0))
    assert need.sum() < need.size
    assert np.allclose(P1[need], inv[need], rtol=1e-11, atol=1e-13)
    assert np.allclose(P2[need], inv[need], rtol=1e-11, atol=1e-13)


def test_block_selinv_equals_dense_inverse_on_pattern():
    mdl = small(n_t=4, nx=3, n_b=2, m=100)
    A = M.obs_matrix(mdl)
    Qc = (M.prior_Q(mdl, mdl.theta_true) + 2.7 * (A.T @ A)).tocsr()
    blocks, _ = bta.from_sparse(Qc, mdl.n_t, mdl.n_s, mdl.n_b)
    Lb, _ = bta.cholesky(blocks)
    S = bta.selinv(Lb)
    inv = np.linalg.inv(Qc.toarray())
    Sinv, _ = bta.from_sparse(sp.csr_matrix(inv), mdl.n_t, mdl.n_s, mdl.n_b)
    for t in range(mdl.n_t):
        assert np.allclose(S.D[t], Sinv.D[t], rtol=1e-11, atol=1e-14)
        assert np.allclose(S.R[t], Sinv.R[t], rtol=1e-11, atol=1e-14)
        if t < mdl.n_t - 1:
            assert np.allclose(S.B[t], Sinv.B[t], rtol=1e-11, atol=1e-14)
    assert np.allclose(S.T, Sinv.T, rtol=1e-11)
    # Q Sigma = I read on the pattern: (Q_c Sigma_full)_ij = delta_ij there, and the
    # selected values are those of Sigma_full
    QS = Qc.toarray() @ inv
    pat = np.abs(Qc.toarray()) > 0
    assert np.allclose(QS[pat], np.eye(mdl.n)[pat], atol=1e-10)
    # tip: inverse of the Schur complement of the latent block
    N = mdl.n_t * mdl.n_s
    Qd = Qc.toarray()
    schur = Qd[N:, N:] - Qd[N:, :N] @ np.linalg.solve(Qd[:N, :N], Qd[:N, N:])
    assert np.allclose(S.T, np.linalg.inv(schur), rtol=1e-10)


def test_prior_marginal_variances_are_kronecker():
    mdl = build("k", 4, 4, 2, 20)
    th = np.array([0.0, -0.5, 0.1, 0.4])
    h = M.hyper(th)
    blocks, _ = bta.from_sparse(M.prior_Q(mdl, th), 4, mdl.n_s, 2)
    Lb, _ = bta.cholesky(blocks)
    v = bta.diag_of(bta.selinv(Lb))
    vt = np.diag(np.linalg.inv(M.temporal_Q(4, h["rho"]).toarray()))
    vs = np.diag(np.linalg.inv(M.spatial_Q(mdl, th).toarray()))
    assert np.allclose(v[:-2], np.kron(vt, vs), rtol=1e-11)
    assert np.allclose(v[-2:], 1.0 / h["tau_b"], rtol=1e-12)


def test_prior_trace_closed_forms():
    mdl = build("k", 5, 4, 2, 20)
    th = np.array([0.0, -0.5, 0.1, 0.9])
    h = M.hyper(th)
    rho = h["rho"]
    blocks, _ = bta.from_sparse(M.prior_Q(mdl, th), 5, mdl.n_s, 2)
    Lb, _ = bta.cholesky(blocks)
    S = bta.selinv(Lb)
    tr = lambda j: bta.contract(S, bta.from_sparse(M.dQ_dtheta(mdl, th, j), 5, mdl.n_s, 2)[0])
    assert np.isclose(tr(2), -2.0 * mdl.n_t * mdl.n_s, rtol=1e-11)
    expect = mdl.n_s * rho * (1 - rho) * 2 * (mdl.n_t - 1) * rho / (1 - rho * rho)
    assert np.isclose(tr(3), expect, rtol=1e-11)


# ---------------------------------------------------------------- f(theta), Eq. post_theta_approx

def test_gaussian_f_equals_closed_form_marginal_likelihood_config1():
    mdl = config_model(1)
    th = mdl.theta_true
    cf = dense.gaussian_closed_form(mdl, th)
    d = dense.gaussian_eval(mdl, th, want_var=False)
    b = bta.gaussian(mdl, th)
    assert abs(d["f"] - cf) / abs(cf) < 1e-11
    assert abs(b["f"] - cf) / abs(cf) < 1e-11
    A = M.obs_matrix(mdl)
    tau_y = math.exp(th[0])
    Qc = M.prior_Q(mdl, th) + tau_y * (A.T @ A)
    rhs = tau_y * (A.T @ mdl.y)
    assert np.linalg.norm(Qc @ b["x"] - rhs) / np.linalg.norm(rhs) < 1e-13


def test_gaussian_bta_matches_dense_definition():
    mdl = small(n_t=4, nx=4, n_b=3, m=300)
    th = mdl.theta_true + np.array([-0.2, 0.1, 0.05, -0.3])
    d = dense.gaussian_eval(mdl, th)
    b = bta.gaussian(mdl, th, want_var=True)
    assert abs(d["f"] - b["f"]) < 1e-11 * abs(d["f"])
    assert np.allclose(d["x"], b["x"], rtol=1e-11, atol=1e-12 * np.abs(d["x"]).max())
    assert np.allclose(d["var"], b["var"], rtol=1e-11)


@pytest.mark.parametrize("lik", ["gaussian", "poisson", "binomial", "negbinomial"])
def test_adjoint_gradient_matches_central_differences(lik):
    mdl = small(n_t=3, nx=4, n_b=2, m=200, lik=lik)
    th = mdl.theta_true + np.array([0.1, -0.1, 0.05, 0.2])
    g = bta.evaluate(mdl, th, want_grad=True)["grad"]
    f = lambda t: bta.evaluate(mdl, t)["f"]
    errs = []
    for eps in (1e-2, 1e-3):
        errs.append(np.abs(fd.central_gradient(f, th, eps) - g).max())
    assert errs[-1] < 1e-5 * max(1.0, np.abs(g).max())
    assert errs[1] < errs[0] / 20.0          # O(eps^2) until round-off


def test_forward_differences_are_first_order():
    f = lambda t: float(np.exp(t[0]) * np.sin(t[1]) + t[2] ** 3 - t[3] * t[0])
    th = np.array([0.3, 0.7, -0.4, 1.2])
    exact = np.array([np.exp(th[0]) * np.sin(th[1]) - th[3], np.exp(th[0]) * np.cos(th[1]), 3 * th[2] ** 2, -th[0]])
    e1 = np.abs(fd.forward_gradient(f, th, 1e-3) - exact).max()
    e2 = np.abs(fd.forward_gradient(f, th, 1e-4) - exact).max()
    assert 5.0 < e1 / e2 < 20.0          # O(eps)
    assert np.abs(fd.central_gradient(f, th, 1e-3) - exact).max() < e2   # central is O(eps^2)


def test_fd_stencil_layout_and_gradient():
    th = np.array([0.3, -0.2, 0.1, 1.0])
    pts = fd_stencil(th, 1e-3)
    quad = lambda t: float(t @ np.diag([1.0, 2.0, 3.0, 4.0]) @ t + t.sum())
    g = fd.gradient_from_stencil([quad(p) for p in pts], 1e-3)
    assert np.allclose(g, 2 * np.array([1.0, 2.0, 3.0, 4.0]) * th + 1.0, rtol=1e-9)


# ---------------------------------------------------------------- Poisson (Laplace, Sec. 2.2)

@pytest.mark.parametrize("lik", ["poisson", "binomial", "negbinomial"])
def test_poisson_mode_is_stationary_and_matches_dense_newton(lik):
    mdl = small(n_t=3, nx=4, n_b=2, m=250, lik=lik)
    th = mdl.theta_true + np.array([0.5, 0.0, 0.1, 0.0])
    b = bta.poisson(mdl, th, want_var=True)
    d = dense.poisson_eval(mdl, th)
    A = M.obs_matrix(mdl)
    Q = M.prior_Q(mdl, th)
    eta = A @ b["x"]
    if lik == "poisson":
        score = mdl.y - mdl.E * np.exp(eta)
    elif lik == "binomial":
        score = mdl.y - mdl.E / (1.0 + np.exp(-eta))
    else:   # d/deta of log NB(y; E e^eta, r), written out independently of glm_terms
        mu = mdl.E * np.exp(eta)
        score = mdl.y * mdl.nb_size / (mdl.nb_size + mu) - mdl.nb_size * mu / (mdl.nb_size + mu)
    grad = Q @ b["x"] - A.T @ score
    assert np.abs(grad).max() < 1e-8 * max(1.0, np.abs(A.T @ mdl.y).max())
    assert b["converged"] and d["converged"]
    assert abs(b["f"] - d["f"]) < 1e-11 * abs(d["f"])
    assert np.allclose(b["x"], d["x"], atol=1e-10)
    assert np.allclose(b["var"], d["var"], rtol=1e-10)


@pytest.mark.parametrize("lik", ["poisson", "binomial", "negbinomial"])
def test_poisson_laplace_matches_generic_laplace_formula(lik):
    # log p(y|theta) ~ h(x*) + (n/2) log 2 pi - 1/2 log|-h''(x*)|, with
    # h(x) = log pi(x|theta) + log p(y|x, theta), mode from a generic optimiser
    from scipy.optimize import minimize
    mdl = small(n_t=2, nx=3, n_b=1, m=60, lik=lik)
    th = mdl.theta_true + np.array([1.0, 0.0, 0.0, 0.0])
    Q = M.prior_Q(mdl, th).toarray()
    A = M.obs_matrix(mdl).toarray()
    n = mdl.n
    logdetQ = np.linalg.slogdet(Q)[1]

    r = mdl.nb_size

    def logp(eta):
        if lik == "poisson":
            return stats.poisson.logpmf(mdl.y, mdl.E * np.exp(eta)).sum()
        if lik == "negbinomial":
            return stats.nbinom.logpmf(mdl.y, r, r / (r + mdl.E * np.exp(eta))).sum()
        return stats.binom.logpmf(mdl.y, mdl.E, 1.0 / (1.0 + np.exp(-eta))).sum()

    def mean_and_weight(eta):
        """(y - d logp / d eta, -d^2 logp / d eta^2) per observation."""
        if lik == "poisson":
            mu = mdl.E * np.exp(eta)
            return mu, mu
        if lik == "negbinomial":
            mu = mdl.E * np.exp(eta)
            return mdl.y - r * (mdl.y - mu) / (r + mu), r * mu * (mdl.y + r) / (r + mu) ** 2
        pr = 1.0 / (1.0 + np.exp(-eta))
        return mdl.E * pr, mdl.E * pr * (1.0 - pr)

    def h(x):
        return (-0.5 * n * math.log(2 * math.pi) + 0.5 * logdetQ - 0.5 * x @ Q @ x + logp(A @ x))

    def dh(x):
        return -Q @ x + A.T @ (mdl.y - mean_and_weight(A @ x)[0])

    res = minimize(lambda x: -h(x), np.zeros(n), jac=lambda x: -dh(x), method="BFGS",
                   options=dict(gtol=1e-11, maxiter=10000))
    xs = res.x
    Hn = Q + A.T @ np.diag(mean_and_weight(A @ xs)[1]) @ A
    laplace = h(xs) + 0.5 * n * math.log(2 * math.pi) - 0.5 * np.linalg.slogdet(Hn)[1]
    expect_f = -M.log_prior(mdl, th) - laplace
    assert abs(bta.poisson(mdl, th)["f"] - expect_f) < 1e-7 * abs(expect_f)


def test_capped_newton_reaches_the_plain_newton_mode_in_fewer_steps():
    # the full step from x = 0 overshoots exp(eta) on counts; capping |d eta| at 2 per step
    # reaches the same mode (the stationary point does not depend on the step length)
    from synth import CONFIGS, theta_batch
    c = dict(CONFIGS[5]); c["n_t"] = 2; c["m"] = 6000; c["nx"] = 24
    mdl = build(**c)
    th = theta_batch(5, mdl)[0]
    x_cap, it_cap, ok_cap = bta.poisson_mode(mdl, th, max_iter=60)
    A = M.obs_matrix(mdl)
    Q = M.prior_Q(mdl, th)
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    x = np.zeros(mdl.n)
    for it_plain in range(1, 80):
        eta = A @ x
        mean, w, _ = M.glm_terms(mdl, eta)
        xn = spla.spsolve((Q + A.T @ sp.diags(w) @ A).tocsc(), A.T @ (mdl.y - mean + w * eta))
        done = np.linalg.norm(xn - x) < 1e-8
        x = xn
        if done:
            break
    assert ok_cap and it_cap < it_plain
    np.testing.assert_allclose(x_cap, x, atol=1e-8)


# ---------------------------------------------------------------- TF32 split product (mixed path)

def test_tf32_rounding_is_nearest_ties_away():
    from oracle import tf32
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -10)                  # TF32 unit in the last place at 1
    exact = np.array([0.0, 1.0, -0.75, 1.5, 2047.0, -1024.0, 2.0 ** -20, 3.0 * 2 ** 40], dtype=np.float32)
    assert np.array_equal(tf32.tf32_rna(exact), exact)
    half = np.float32(one + ulp / 2)              # halfway between 1 and 1 + 2^-10
    assert tf32.tf32_rna(half) == one + ulp and tf32.tf32_rna(-half) == -(one + ulp)
    assert tf32.tf32_rna(np.float32(one + ulp / 4)) == one
    assert tf32.tf32_rna(np.float32(one + 3 * ulp / 4)) == one + ulp
    x = np.random.default_rng(0).standard_normal(100000).astype(np.float32)
    r = tf32.tf32_rna(x)
    assert np.all(r.view(np.uint32) & 0x1FFF == 0)                      # 10 explicit mantissa bits
    assert np.all(np.abs(r.astype(np.float64) - x) <= 2.0 ** -11 * np.abs(x.astype(np.float64)))


def test_tf32_split_recovers_fp32_value():
    from oracle import tf32
    x = (np.random.default_rng(1).standard_normal(100000) * 10.0 ** np.random.default_rng(2).integers(
        -6, 6, 100000)).astype(np.float32)
    hi, lo = tf32.split(x)
    assert np.all(hi.view(np.uint32) & 0x1FFF == 0) and np.all(lo.view(np.uint32) & 0x1FFF == 0)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(x.astype(np.float64)))


def test_tf32_split_product_error_model():
    from oracle import tf32
    rng = np.random.default_rng(3)
    # integers of at most 11 significant bits are TF32 values: the split product is exact
    Xi = rng.integers(-32, 33, (64, 256)).astype(np.float32)
    Yi = rng.integers(-32, 33, (48, 256)).astype(np.float32)
    assert np.array_equal(tf32.product_3xtf32(Xi, Yi), Xi.astype(np.float64) @ Yi.astype(np.float64).T)
    # FP32 inputs: the three kept terms miss lo*lo and the rounding of lo, each below 2^-22 |x||y|
    X = rng.standard_normal((64, 256)).astype(np.float32)
    Y = rng.standard_normal((48, 256)).astype(np.float32)
    exact = X.astype(np.float64) @ Y.astype(np.float64).T
    bound = 3 * 2.0 ** -22 * (np.abs(X.astype(np.float64)) @ np.abs(Y.astype(np.float64)).T)
    err = np.abs(tf32.product_3xtf32(X, Y) - exact)
    assert np.all(err <= bound)
    single = np.abs(tf32.tf32_rna(X).astype(np.float64) @ tf32.tf32_rna(Y).astype(np.float64).T - exact)
    assert err.max() < single.max() / 100
