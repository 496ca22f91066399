"""The definition of f(theta), x*(theta) and diag(Q_c^-1), with dense matrices.

For small n only (every matrix is a dense n x n array).  This is the plain
reading of Eq. post_theta_approx: the Laplace approximation of pi(theta|y),

  pi~(theta|y) = pi(theta) pi(x|theta) pi(y|x,theta) / pi_G(x|theta,y)  at x = x*(theta),

with f(theta) = -log pi~(theta|y) (Sec. 3.1).  Log-determinants come from a
Cholesky factor, log|Q| = sum_i 2 log L_ii (Sec. 2.4); the mode solves
Q_c x* = b (Sec. 2.2); the marginal variances are the diagonal of the full
inverse of Q_c (Sec. 2.3).  For a Gaussian likelihood pi_G is exact
(Sec. 2.3) and there is also the closed form -log pi(theta) - log p(y|theta)
with y ~ N(0, A Q^-1 A^T + tau_y^-1 I), used as a pin.
"""
import math
import numpy as np
import scipy.linalg as sla

from . import model as M

LOG2PI = math.log(2.0 * math.pi)


def chol_logdet(Q):
    L = np.linalg.cholesky(Q)
    return L, 2.0 * float(np.sum(np.log(np.diag(L))))


def gaussian_eval(model, theta, want_var=True):
    """f, x*, diag(Q_c^-1), log|Q|, log|Q_c| for a Gaussian likelihood."""
    h = M.hyper(theta, "gaussian", model.tau_b)
    tau_y = h["tau_y"]
    Q = M.prior_Q(model, theta).toarray()
    A = M.obs_matrix(model)
    Qc = Q + tau_y * (A.T @ A).toarray()
    _, logdetQ = chol_logdet(Q)
    Lc, logdetQc = chol_logdet(Qc)
    b = tau_y * (A.T @ model.y)
    x = sla.cho_solve((Lc, True), b)
    r = model.y - A @ x
    f = (-M.log_prior(model, theta) - 0.5 * logdetQ + 0.5 * x @ Q @ x
         - 0.5 * model.m * float(theta[0]) + 0.5 * model.m * LOG2PI
         + 0.5 * tau_y * float(r @ r) + 0.5 * logdetQc)
    out = dict(f=float(f), x=x, logdetQ=logdetQ, logdetQc=logdetQc)
    if want_var:
        out["var"] = np.diag(sla.cho_solve((Lc, True), np.eye(model.n))).copy()
    return out


def gaussian_closed_form(model, theta):
    """-log pi(theta) - log N(y; 0, S),  S = A Q^-1 A^T + tau_y^-1 I_m (dense m x m)."""
    h = M.hyper(theta, "gaussian", model.tau_b)
    Q = M.prior_Q(model, theta).toarray()
    A = M.obs_matrix(model).toarray()
    S = A @ np.linalg.solve(Q, A.T) + np.eye(model.m) / h["tau_y"]
    L, logdetS = chol_logdet(S)
    z = sla.solve_triangular(L, model.y, lower=True)
    return float(-M.log_prior(model, theta) + 0.5 * model.m * LOG2PI + 0.5 * logdetS + 0.5 * z @ z)


def capped_step(A, x, xn):
    return M.capped_step(A, x, xn)


def poisson_mode(model, theta, tol=1e-8, max_iter=50, x0=None):
    """Newton iteration for the mode of pi(x | theta, y), non-Gaussian likelihood.

    x^{k+1} solves (Q + A^T D A) x = A^T (y - b1 + D eta) with eta = A x^k,
    b1 = the mean and D = diag(weight) from glm_terms (Poisson: both E e^eta),
    the step capped so that no linear predictor moves by more than 2
    (capped_step); stop when ||x^{k+1} - x^k||_2 < tol.  Returns (x*,
    iterations, converged).
    """
    Q = M.prior_Q(model, theta).toarray()
    A = M.obs_matrix(model)
    x = np.zeros(model.n) if x0 is None else np.array(x0, dtype=float)
    for k in range(1, max_iter + 1):
        eta = A @ x
        mean, wgt, _ = M.glm_terms(model, eta)
        Qc = Q + (A.T @ (A.multiply(wgt[:, None]))).toarray()
        rhs = A.T @ (model.y - mean + wgt * eta)
        xn = sla.cho_solve((np.linalg.cholesky(Qc), True), rhs)
        xn = capped_step(A, x, xn)
        step = float(np.linalg.norm(xn - x))
        x = xn
        if step < tol:
            return x, k, True
    return x, max_iter, False


def poisson_eval(model, theta, want_var=True, tol=1e-8, max_iter=50):
    """Laplace f(theta) for a non-Gaussian likelihood, Q_c refactorised at x*."""
    Q = M.prior_Q(model, theta).toarray()
    A = M.obs_matrix(model)
    x, iters, ok = poisson_mode(model, theta, tol, max_iter)
    eta = A @ x
    _, wgt, _ = M.glm_terms(model, eta)
    Qc = Q + (A.T @ (A.multiply(wgt[:, None]))).toarray()
    _, logdetQ = chol_logdet(Q)
    Lc, logdetQc = chol_logdet(Qc)
    f = (-M.log_prior(model, theta) - 0.5 * logdetQ + 0.5 * x @ Q @ x
         - M.glm_loglik(model, eta) + 0.5 * logdetQc)
    out = dict(f=float(f), x=x, logdetQ=logdetQ, logdetQc=logdetQc, iters=iters, converged=ok)
    if want_var:
        out["var"] = np.diag(sla.cho_solve((Lc, True), np.eye(model.n))).copy()
    return out


def evaluate(model, theta, want_var=True):
    if model.lik == "gaussian":
        return gaussian_eval(model, theta, want_var)
    return poisson_eval(model, theta, want_var)
