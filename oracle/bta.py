"""Block-tridiagonal-arrowhead (BTA) Cholesky, solves and selected inversion.

With the latent vector ordered time-major and the fixed effects last, Q and
Q_c = Q + A^T D A are block tridiagonal with an arrowhead: n_t diagonal
blocks D_t (n_s x n_s), sub-diagonal blocks B_t = block (t+1, t), arrow
blocks R_t = block (a, t) (n_b x n_s) and a tip (n_b x n_b).  Placing the
dense arrow last means the Cholesky factor has no fill outside this block
pattern (the arrowhead example of Fig. arrowhead_matrices, Sec. 2.4.1).

The algorithms are the paper's, written per block with numpy/scipy dense
kernels as the steps:
  * Cholesky Q = L L^T and log|Q| = sum_i 2 log L_ii (Sec. 2.4): per time
    step L_t = chol(D_t), L_{t+1,t} = B_t L_t^-T, L_{a,t} = R_t L_t^-T, then the
    Schur updates D_{t+1} -= L_{t+1,t} L_{t+1,t}^T, R_{t+1} -= L_{a,t} L_{t+1,t}^T,
    T -= L_{a,t} L_{a,t}^T; finally L_a = chol(T).
  * forward and backward substitution for Q x = b (Sec. 2.4).
  * selected inversion: the block form of Eq. sel_inv_cov,
      Sigma_IJ = delta_IJ L_II^-T L_II^-1 - L_II^-T sum_{K > I, L_KI != 0} L_KI^T Sigma_KJ,
    run from the bottom-right block to the top-left, computing only the
    blocks on the pattern of L (Sec. 2.4.2).
  * one level of nested dissection of the time chain (Sec. 3.3): the same
    factorisation, substitution and selected inversion in the split order
    (cholesky_split, solve_split, selinv_split).
Then f(theta), x*, diag(Q_c^-1) and the gradient for both likelihoods.

The gradient is the adjoint form: for a Gaussian likelihood
  d_j f = -d_j log pi(theta) - 1/2 tr(Q^-1 d_jQ) + 1/2 x*^T d_jQ x*
          + 1/2 tr(Q_c^-1 d_jQ_c) + [j = 1](-m/2 + tau_y/2 ||y - A x*||^2)
(the quadratic in x is minimised at x*, so dx*/dtheta drops out); for the
Poisson likelihood the log|Q_c(x*)| term adds -lambda^T d_jQ x* with
Q_c lambda = A^T w, w_i = 1/2 (a_i^T Q_c^-1 a_i) E_i exp(eta_i).  The
paper only discusses (and sets aside) automatic differentiation (Sec. 3.1);
these formulas are this library's own derivation and are pinned against
central differences (Eq. central_diff) in the tests.
"""
import math
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import model as M

LOG2PI = math.log(2.0 * math.pi)


class Blocks:
    """A symmetric BTA matrix (or its factor, or its selected inverse) by blocks."""

    def __init__(self, n_t, n_s, n_b):
        self.n_t, self.n_s, self.n_b = n_t, n_s, n_b
        self.D = [None] * n_t          # diagonal blocks (t, t)
        self.B = [None] * (n_t - 1)    # sub-diagonal blocks (t+1, t)
        self.R = [None] * n_t          # arrow blocks (a, t)
        self.T = None                  # tip (a, a)


def from_sparse(Q, n_t, n_s, n_b):
    """Cut a sparse symmetric matrix into BTA blocks.

    Returns (blocks, outside) where outside counts the nonzeros of the lower
    triangle that fall outside the BTA pattern (0 for the model's Q and Q_c).
    """
    Q = sp.csr_matrix(Q)
    b = Blocks(n_t, n_s, n_b)
    N = n_t * n_s
    for t in range(n_t):
        s = slice(t * n_s, (t + 1) * n_s)
        b.D[t] = Q[s, s].toarray()
        if t < n_t - 1:
            b.B[t] = Q[(t + 1) * n_s:(t + 2) * n_s, s].toarray()
        b.R[t] = Q[N:N + n_b, s].toarray()
    b.T = Q[N:, N:].toarray()
    L = sp.tril(Q, format="coo")
    ti, tj = L.row // n_s, L.col // n_s
    ti = np.where(L.row >= N, n_t, ti)
    tj = np.where(L.col >= N, n_t, tj)
    inside = (ti == tj) | (ti == tj + 1) | (ti == n_t)
    outside = int(np.count_nonzero((L.data != 0) & ~inside))
    return b, outside


def cholesky(Qb):
    """BTA Cholesky.  Returns (L blocks, log|Q|).  Raises LinAlgError if not SPD."""
    n_t, n_b = Qb.n_t, Qb.n_b
    L = Blocks(n_t, Qb.n_s, n_b)
    D = [d.copy() for d in Qb.D]
    R = [r.copy() for r in Qb.R]
    T = Qb.T.copy()
    logdet = 0.0
    for t in range(n_t):
        Lt = np.linalg.cholesky(D[t])
        L.D[t] = Lt
        logdet += 2.0 * float(np.sum(np.log(np.diag(Lt))))
        if t < n_t - 1:
            L.B[t] = sla.solve_triangular(Lt, Qb.B[t].T, lower=True).T
            D[t + 1] = D[t + 1] - L.B[t] @ L.B[t].T
        L.R[t] = sla.solve_triangular(Lt, R[t].T, lower=True).T if n_b else np.zeros((0, Qb.n_s))
        if t < n_t - 1 and n_b:
            R[t + 1] = R[t + 1] - L.R[t] @ L.B[t].T
        if n_b:
            T = T - L.R[t] @ L.R[t].T
    if n_b:
        L.T = np.linalg.cholesky(T)
        logdet += 2.0 * float(np.sum(np.log(np.diag(L.T))))
    else:
        L.T = np.zeros((0, 0))
    return L, logdet


def solve(L, b):
    """x with (L L^T) x = b by forward then backward block substitution."""
    n_t, n_s, n_b = L.n_t, L.n_s, L.n_b
    N = n_t * n_s
    z = [None] * n_t
    for t in range(n_t):
        rhs = b[t * n_s:(t + 1) * n_s].copy()
        if t > 0:
            rhs -= L.B[t - 1] @ z[t - 1]
        z[t] = sla.solve_triangular(L.D[t], rhs, lower=True)
    x = np.empty(N + n_b)
    if n_b:
        za = b[N:].copy()
        for t in range(n_t):
            za -= L.R[t] @ z[t]
        za = sla.solve_triangular(L.T, za, lower=True)
        xa = sla.solve_triangular(L.T, za, lower=True, trans="T")
        x[N:] = xa
    else:
        xa = np.zeros(0)
    for t in reversed(range(n_t)):
        rhs = z[t].copy()
        if t < n_t - 1:
            rhs -= L.B[t].T @ x[(t + 1) * n_s:(t + 2) * n_s]
        if n_b:
            rhs -= L.R[t].T @ xa
        x[t * n_s:(t + 1) * n_s] = sla.solve_triangular(L.D[t], rhs, lower=True, trans="T")
    return x


def selinv(L):
    """Selected inverse on the BTA pattern by the block form of Eq. sel_inv_cov."""
    n_t, n_s, n_b = L.n_t, L.n_s, L.n_b
    S = Blocks(n_t, n_s, n_b)
    if n_b:
        Ti = sla.solve_triangular(L.T, np.eye(n_b), lower=True)
        S.T = Ti.T @ Ti
    else:
        S.T = np.zeros((0, 0))
    I = np.eye(n_s)
    for t in reversed(range(n_t)):
        Lt = L.D[t]
        # sum over K > t with L_{K,t} != 0, i.e. K in {t+1, a}, of L_{K,t}^T Sigma_{K,J}
        acc_a = L.R[t].T @ S.T if n_b else np.zeros((n_s, 0))           # J = a
        acc_t1 = None
        if t < n_t - 1:
            acc_t1 = L.B[t].T @ S.D[t + 1]                                # J = t+1
            if n_b:
                acc_t1 = acc_t1 + L.R[t].T @ S.R[t + 1]
                acc_a = acc_a + L.B[t].T @ S.R[t + 1].T
        S_ta = -sla.solve_triangular(Lt, acc_a, lower=True, trans="T")   # Sigma_{t,a}
        S.R[t] = S_ta.T
        acc_tt = L.R[t].T @ S.R[t] if n_b else np.zeros((n_s, n_s))
        if acc_t1 is not None:
            S_t_t1 = -sla.solve_triangular(Lt, acc_t1, lower=True, trans="T")  # Sigma_{t,t+1}
            S.B[t] = S_t_t1.T
            acc_tt = acc_tt + L.B[t].T @ S.B[t]
        Linv = sla.solve_triangular(Lt, I, lower=True)
        Stt = Linv.T @ Linv - sla.solve_triangular(Lt, acc_tt, lower=True, trans="T")
        S.D[t] = 0.5 * (Stt + Stt.T)
    return S


# ---------------------------------------------------------------- one level of nested dissection
#
# Sec. 3.3: a nested-dissection order splits a matrix into two independent parts joined
# by a separator; the parts are factorised independently, then the separator, and the
# partial inverse runs the other way (the separator's entries first).  On the time chain
# one level of it takes block k as the separator: blocks 0..k-1 are eliminated in order
# towards k, blocks n_t-1..k+1 in reverse order towards k, then block k, then the tip.
# Every block keeps one neighbour that is eliminated after it (t + 1 on the first part,
# t - 1 on the second, none for k), so the factor has no fill outside the BTA pattern; it
# is the Cholesky factor of the matrix with its time blocks permuted into that order.


def split_order(n_t, k):
    """The elimination order of the split chain and, per block, the neighbour eliminated
    after it (None for the separator)."""
    order = list(range(k)) + list(range(n_t - 1, k, -1)) + [k]
    nxt = {t: (t + 1 if t < k else t - 1) for t in range(n_t) if t != k}
    nxt[k] = None
    return order, nxt


def _coupling(Qb, t, s):
    """Block (s, t) of the BTA matrix for neighbours s = t +- 1."""
    return Qb.B[t] if s == t + 1 else Qb.B[s].T


def cholesky_split(Qb, k):
    """Block Cholesky in the split order.  Returns (factor, log|Q|); the factor holds
    L_t (F.D[t]), L_{nxt(t), t} (F.C[t]), L_{a,t} (F.R[t]) and L_a (F.T)."""
    n_t, n_s, n_b = Qb.n_t, Qb.n_s, Qb.n_b
    order, nxt = split_order(n_t, k)
    F = Blocks(n_t, n_s, n_b)
    F.C = [None] * n_t
    D = [d.copy() for d in Qb.D]
    R = [r.copy() for r in Qb.R]
    T = Qb.T.copy()
    logdet = 0.0
    for t in order:
        Lt = np.linalg.cholesky(D[t])
        F.D[t] = Lt
        logdet += 2.0 * float(np.sum(np.log(np.diag(Lt))))
        s = nxt[t]
        if s is not None:
            F.C[t] = sla.solve_triangular(Lt, _coupling(Qb, t, s).T, lower=True).T
            D[s] = D[s] - F.C[t] @ F.C[t].T
        F.R[t] = sla.solve_triangular(Lt, R[t].T, lower=True).T if n_b else np.zeros((0, n_s))
        if n_b:
            if s is not None:
                R[s] = R[s] - F.R[t] @ F.C[t].T
            T = T - F.R[t] @ F.R[t].T
    F.T = np.linalg.cholesky(T) if n_b else np.zeros((0, 0))
    if n_b:
        logdet += 2.0 * float(np.sum(np.log(np.diag(F.T))))
    F.order, F.nxt = order, nxt
    return F, logdet


def solve_split(F, b):
    """x with (L L^T) x = b for the split factor: forward substitution in the split
    order, the tip, then backward substitution in the reverse order."""
    n_t, n_s, n_b = F.n_t, F.n_s, F.n_b
    N = n_t * n_s
    blk = lambda v, t: v[t * n_s:(t + 1) * n_s]
    r = b.astype(float).copy()
    z = [None] * n_t
    for t in F.order:
        z[t] = sla.solve_triangular(F.D[t], blk(r, t), lower=True)
        s = F.nxt[t]
        if s is not None:
            r[s * n_s:(s + 1) * n_s] -= F.C[t] @ z[t]
        if n_b:
            r[N:] -= F.R[t] @ z[t]
    x = np.empty(N + n_b)
    if n_b:
        za = sla.solve_triangular(F.T, r[N:], lower=True)
        x[N:] = sla.solve_triangular(F.T, za, lower=True, trans="T")
    for t in reversed(F.order):
        rhs = z[t].copy()
        s = F.nxt[t]
        if s is not None:
            rhs -= F.C[t].T @ blk(x, s)
        if n_b:
            rhs -= F.R[t].T @ x[N:]
        x[t * n_s:(t + 1) * n_s] = sla.solve_triangular(F.D[t], rhs, lower=True, trans="T")
    return x


def selinv_split(F):
    """Selected inverse (Eq. sel_inv_cov in block form) in the reverse split order: the
    tip, the separator, then both parts outwards.  Returns BTA blocks (S.B[t] = block
    (t+1, t))."""
    n_t, n_s, n_b = F.n_t, F.n_s, F.n_b
    S = Blocks(n_t, n_s, n_b)
    off = {}                       # Sigma_{nxt(t), t}
    if n_b:
        Ti = sla.solve_triangular(F.T, np.eye(n_b), lower=True)
        S.T = Ti.T @ Ti
    else:
        S.T = np.zeros((0, 0))
    I = np.eye(n_s)
    for t in reversed(F.order):
        Lt, s = F.D[t], F.nxt[t]
        # sum over the blocks K eliminated after t with L_{K,t} != 0: K in {nxt(t), a}
        acc_a = F.R[t].T @ S.T if n_b else np.zeros((n_s, 0))
        acc_s = None
        if s is not None:
            acc_s = F.C[t].T @ S.D[s]
            if n_b:
                acc_s = acc_s + F.R[t].T @ S.R[s]
                acc_a = acc_a + F.C[t].T @ S.R[s].T
        S.R[t] = (-sla.solve_triangular(Lt, acc_a, lower=True, trans="T")).T
        acc_tt = F.R[t].T @ S.R[t] if n_b else np.zeros((n_s, n_s))
        if acc_s is not None:
            off[t] = (-sla.solve_triangular(Lt, acc_s, lower=True, trans="T")).T     # Sigma_{s,t}
            acc_tt = acc_tt + F.C[t].T @ off[t]
        Linv = sla.solve_triangular(Lt, I, lower=True)
        Stt = Linv.T @ Linv - sla.solve_triangular(Lt, acc_tt, lower=True, trans="T")
        S.D[t] = 0.5 * (Stt + Stt.T)
    for t in range(n_t - 1):       # block (t+1, t) from whichever of the pair was eliminated first
        S.B[t] = off[t] if F.nxt[t] == t + 1 else off[t + 1].T
    return S


def diag_of(S):
    parts = [np.diag(d) for d in S.D]
    if S.n_b:
        parts.append(np.diag(S.T))
    return np.concatenate(parts)


def contract(S, Mb):
    """tr(Sigma M) = sum_ij Sigma_ij M_ij for symmetric Sigma and M, M on the pattern."""
    s = sum(float(np.sum(S.D[t] * Mb.D[t])) for t in range(S.n_t))
    s += 2.0 * sum(float(np.sum(S.B[t] * Mb.B[t])) for t in range(S.n_t - 1))
    if S.n_b:
        s += 2.0 * sum(float(np.sum(S.R[t] * Mb.R[t])) for t in range(S.n_t))
        s += float(np.sum(S.T * Mb.T))
    return s


def quad_forms_on_pattern(S, model, A):
    """a_i^T Sigma a_i for every observation row, using only pattern entries of Sigma."""
    n_t, n_s, n_b = model.n_t, model.n_s, model.n_b
    N = n_t * n_s
    A = sp.csr_matrix(A)
    out = np.zeros(model.m)
    for i in range(model.m):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        acc = 0.0
        for p, vp in zip(cols, vals):
            for q, vq in zip(cols, vals):
                acc += vp * vq * _entry(S, p, q, n_s, N)
        out[i] = acc
    return out


def _entry(S, p, q, n_s, N):
    if p >= N and q >= N:
        return S.T[p - N, q - N]
    if p >= N:
        return S.R[q // n_s][p - N, q % n_s]
    if q >= N:
        return S.R[p // n_s][q - N, p % n_s]
    tp, tq = p // n_s, q // n_s
    if tp == tq:
        return S.D[tp][p % n_s, q % n_s]
    if tp == tq + 1:
        return S.B[tq][p % n_s, q % n_s]
    if tq == tp + 1:
        return S.B[tp][q % n_s, p % n_s]
    raise KeyError("entry outside the BTA pattern")


def _blocks(model, Qsp):
    b, _ = from_sparse(Qsp, model.n_t, model.n_s, model.n_b)
    return b


def gaussian(model, theta, want_grad=False, want_var=False):
    """f, x*, log|Q|, log|Q_c| (and diag(Q_c^-1), gradient) for a Gaussian likelihood."""
    h = M.hyper(theta, "gaussian", model.tau_b)
    tau_y = h["tau_y"]
    A = M.obs_matrix(model)
    Q = M.prior_Q(model, theta)
    AtA = (A.T @ A).tocsr()
    Qc = (Q + tau_y * AtA).tocsr()
    LQ, logdetQ = cholesky(_blocks(model, Q))
    LQc, logdetQc = cholesky(_blocks(model, Qc))
    x = solve(LQc, tau_y * (A.T @ model.y))
    r = model.y - A @ x
    f = (-M.log_prior(model, theta) - 0.5 * logdetQ + 0.5 * float(x @ (Q @ x))
         - 0.5 * model.m * float(theta[0]) + 0.5 * model.m * LOG2PI
         + 0.5 * tau_y * float(r @ r) + 0.5 * logdetQc)
    out = dict(f=float(f), x=x, logdetQ=logdetQ, logdetQc=logdetQc)
    if want_var or want_grad:
        SQc = selinv(LQc)
        out["var"] = diag_of(SQc)
    if want_grad:
        SQ = selinv(LQ)
        dlp = M.dlog_prior(model, theta)
        g = np.zeros(4)
        for j in range(4):
            dQ = M.dQ_dtheta(model, theta, j)
            dQb = _blocks(model, dQ)
            g[j] = (-dlp[j] - 0.5 * contract(SQ, dQb) + 0.5 * float(x @ (dQ @ x))
                    + 0.5 * contract(SQc, dQb))
        g[0] += 0.5 * tau_y * contract(SQc, _blocks(model, AtA)) - 0.5 * model.m + 0.5 * tau_y * float(r @ r)
        out["grad"] = g
    return out


def poisson_mode(model, theta, tol=1e-8, max_iter=50):
    """Newton iteration for x*(theta) (Sec. 2.2) with BTA factorisations, for a
    non-Gaussian likelihood (D = diag(weight), right-hand side
    A^T (y - mean + D eta), both from glm_terms)."""
    A = M.obs_matrix(model)
    Q = M.prior_Q(model, theta)
    x = np.zeros(model.n)
    for k in range(1, max_iter + 1):
        eta = A @ x
        mean, wgt, _ = M.glm_terms(model, eta)
        Qc = (Q + A.T @ sp.diags(wgt) @ A).tocsr()
        L, _ = cholesky(_blocks(model, Qc))
        xn = M.capped_step(A, x, solve(L, A.T @ (model.y - mean + wgt * eta)))
        step = float(np.linalg.norm(xn - x))
        x = xn
        if step < tol:
            return x, k, True
    return x, max_iter, False


def poisson(model, theta, want_grad=False, want_var=False, tol=1e-8, max_iter=50):
    """Laplace f for a non-Gaussian likelihood; Q_c is refactorised at the mode.
    The adjoint gradient adds -lambda^T dQ x* with Q_c lambda = A^T w,
    w_i = 1/2 (a_i^T Sigma_c a_i) times the derivative of the weight at eta_i."""
    A = M.obs_matrix(model)
    Q = M.prior_Q(model, theta)
    x, iters, ok = poisson_mode(model, theta, tol, max_iter)
    eta = A @ x
    _, wgt, third = M.glm_terms(model, eta)
    Qc = (Q + A.T @ sp.diags(wgt) @ A).tocsr()
    LQ, logdetQ = cholesky(_blocks(model, Q))
    LQc, logdetQc = cholesky(_blocks(model, Qc))
    f = (-M.log_prior(model, theta) - 0.5 * logdetQ + 0.5 * float(x @ (Q @ x))
         - M.glm_loglik(model, eta) + 0.5 * logdetQc)
    out = dict(f=float(f), x=x, logdetQ=logdetQ, logdetQc=logdetQc, iters=iters, converged=ok)
    if want_var or want_grad:
        SQc = selinv(LQc)
        out["var"] = diag_of(SQc)
    if want_grad:
        SQ = selinv(LQ)
        w = 0.5 * quad_forms_on_pattern(SQc, model, A) * third
        lam = solve(LQc, A.T @ w)
        dlp = M.dlog_prior(model, theta)
        g = np.zeros(4)
        for j in range(4):
            dQ = M.dQ_dtheta(model, theta, j)
            dQb = _blocks(model, dQ)
            g[j] = (-dlp[j] - 0.5 * contract(SQ, dQb) + 0.5 * float(x @ (dQ @ x))
                    + 0.5 * contract(SQc, dQb) - float(lam @ (dQ @ x)))
        out["grad"] = g
    return out


def evaluate(model, theta, want_grad=False, want_var=False):
    if model.lik == "gaussian":
        return gaussian(model, theta, want_grad, want_var)
    return poisson(model, theta, want_grad, want_var)
