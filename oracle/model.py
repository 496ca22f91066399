"""Model pieces of the spatio-temporal latent Gaussian model (oracle side).

The paper defines the latent Gaussian model generically (Sec. 2.1): a GMRF
x ~ N(0, Q(theta)^-1), observations conditionally independent given the
linear predictor eta = A x, and a prior pi(theta).  The concrete model used
here is the workload's reading of it:

  Q_s(theta) = tau^2 (kappa^4 C + 2 kappa^2 G + G C^-1 G)        (SPDE, alpha = 2)
  kappa = sqrt(8) / r,  r = exp(theta_2)
  tau^2 = 1 / (4 pi kappa^2 sigma^2),  sigma = exp(theta_3)
  Q_t(rho) = AR(1) precision with unit marginal variance, rho = logistic(theta_4)
  Q(theta) = Q_t (x) Q_s  (+)  tau_b I_{n_b}       (time-major, fixed effects last)
  Gaussian: theta_1 = log tau_y, y | x ~ N(A x, tau_y^-1 I), tau_b fixed
  Poisson:  theta_1 = log tau_b, y_i | x ~ Poisson(E_i exp(eta_i))
  binomial: theta_1 = log tau_b, y_i | x ~ Bin(N_i, logistic(eta_i))
  negative binomial: theta_1 = log tau_b, y_i | x ~ NB(mean E_i exp(eta_i), size r), r fixed
  log pi(theta) = sum_j log N(theta_j; mu_j, s_j^2)

Everything is float64 and built with scipy.sparse exactly as written above.
"""
import math
import numpy as np
import scipy.sparse as sp


def hyper(theta, lik="gaussian", tau_b_fixed=1e-3):
    """Map theta (internal scale) to the model's scalars."""
    th = np.asarray(theta, dtype=float)
    r = math.exp(th[1])
    sigma = math.exp(th[2])
    rho = 1.0 / (1.0 + math.exp(-th[3]))
    kappa = math.sqrt(8.0) / r
    tau2 = 1.0 / (4.0 * math.pi * kappa ** 2 * sigma ** 2)
    if lik == "gaussian":
        tau_y, tau_b = math.exp(th[0]), tau_b_fixed
    else:
        tau_y, tau_b = None, math.exp(th[0])
    return dict(r=r, sigma=sigma, rho=rho, kappa=kappa, tau2=tau2, tau_y=tau_y, tau_b=tau_b)


def fem_matrices(model):
    """C (diagonal, sparse) and G (sparse) from the model inputs."""
    n_s = model.n_s
    C = sp.diags(model.C_diag).tocsr()
    G = sp.csr_matrix((model.G_val, model.G_col, model.G_rowptr), shape=(n_s, n_s))
    return C, G


def spatial_Q(model, theta):
    """Q_s(theta) = tau^2 (kappa^4 C + 2 kappa^2 G + G C^-1 G)."""
    h = hyper(theta, model.lik, model.tau_b)
    C, G = fem_matrices(model)
    Cinv = sp.diags(1.0 / model.C_diag)
    k2 = h["kappa"] ** 2
    return (h["tau2"] * (k2 * k2 * C + 2.0 * k2 * G + G @ Cinv @ G)).tocsr()


def temporal_Q(n_t, rho):
    """Stationary AR(1) precision with unit marginal variance:
    (1 - rho^2)^-1 tridiag(-rho; 1, 1 + rho^2, ..., 1 + rho^2, 1; -rho)."""
    if n_t == 1:
        return sp.csr_matrix(np.ones((1, 1)))
    d = np.full(n_t, 1.0 + rho * rho)
    d[0] = d[-1] = 1.0
    off = np.full(n_t - 1, -rho)
    return (sp.diags([off, d, off], [-1, 0, 1]) / (1.0 - rho * rho)).tocsr()


def prior_Q(model, theta):
    """Q(theta) = Q_t (x) Q_s (+) tau_b I, time-major with the fixed effects last."""
    h = hyper(theta, model.lik, model.tau_b)
    Qst = sp.kron(temporal_Q(model.n_t, h["rho"]), spatial_Q(model, theta))
    if model.n_b == 0:
        return Qst.tocsr()
    return sp.block_diag([Qst, h["tau_b"] * sp.identity(model.n_b)]).tocsr()


def obs_matrix(model):
    """A as an m x n sparse matrix."""
    return sp.csr_matrix((model.A_val, model.A_col, model.A_rowptr), shape=(model.m, model.n))


def log_prior(model, theta):
    """log pi(theta) = sum_j log N(theta_j; mu_j, s_j^2), full normalising constant."""
    th = np.asarray(theta, dtype=float)
    mu, s = model.prior_mean, model.prior_sd
    return float(np.sum(-0.5 * math.log(2.0 * math.pi) - np.log(s) - 0.5 * ((th - mu) / s) ** 2))


def dlog_prior(model, theta):
    th = np.asarray(theta, dtype=float)
    return -(th - model.prior_mean) / model.prior_sd ** 2


def poisson_loglik(model, eta):
    """sum_i [y_i log(E_i exp(eta_i)) - E_i exp(eta_i) - log y_i!]."""
    from scipy.special import gammaln
    y, E = model.y, model.E
    return float(np.sum(y * (np.log(E) + eta) - E * np.exp(eta) - gammaln(y + 1.0)))


def binomial_loglik(model, eta):
    """sum_i [log C(N_i, y_i) + y_i log p_i + (N_i - y_i) log(1 - p_i)], p = logistic(eta),
    N = the numbers of trials (held in model.E)."""
    from scipy.special import gammaln
    y, N = model.y, model.E
    logC = gammaln(N + 1.0) - gammaln(y + 1.0) - gammaln(N - y + 1.0)
    # log p = -log(1 + e^-eta), log(1 - p) = -log(1 + e^eta)
    return float(np.sum(logC - y * np.logaddexp(0.0, -eta) - (N - y) * np.logaddexp(0.0, eta)))


def negbinomial_loglik(model, eta):
    """sum_i log NB(y_i; mean mu_i = E_i e^eta_i, size r):
    lgamma(y + r) - lgamma(r) - lgamma(y + 1) + r log(r / (r + mu)) + y log(mu / (r + mu))."""
    from scipy.special import gammaln
    y, r = model.y, float(model.nb_size)
    mu = model.E * np.exp(eta)
    return float(np.sum(gammaln(y + r) - gammaln(r) - gammaln(y + 1.0) + r * np.log(r / (r + mu))
                        + y * np.log(mu / (r + mu))))


def glm_loglik(model, eta):
    """log p(y | eta) of a non-Gaussian likelihood (Poisson, binomial or negative binomial)."""
    if model.lik == "poisson":
        return poisson_loglik(model, eta)
    if model.lik == "negbinomial":
        return negbinomial_loglik(model, eta)
    return binomial_loglik(model, eta)


NEWTON_DETA = 2.0


def capped_step(A, x, xn, deta=NEWTON_DETA):
    """Safeguarded Newton update: x + a (xn - x) with a = min(1, deta / max_i |(A (xn - x))_i|),
    so that no linear predictor moves by more than deta in one step (the full
    step from x = 0 overshoots exp(eta) by orders of magnitude on Poisson data)."""
    d = xn - x
    m = float(np.abs(A @ d).max()) if d.size else 0.0
    a = deta / m if m > deta else 1.0
    return x + a * d


def glm_terms(model, eta):
    """(y - score, D, dD/deta) per observation, with score = d log p(y | eta) / d eta
    and D = -d^2 log p / d eta^2, the Newton weight.  For the canonical links
    (log p = y eta - b(eta) + const: Poisson b = E e^eta, binomial
    b = N log(1 + e^eta)) these are the first three derivatives of b: the mean,
    the Newton weight and its derivative.  The negative binomial with the log
    link (mean mu = E e^eta, size r) is not canonical: score = y - (y + r) mu / (r + mu)
    and D = (y + r) r mu / (r + mu)^2, the observed information, which the
    Laplace approximation's Hessian at the mode uses (Sec. 2.2)."""
    eta = np.asarray(eta, dtype=float)
    if model.lik == "poisson":
        mu = model.E * np.exp(eta)
        return mu, mu, mu
    if model.lik == "negbinomial":
        y, r = model.y, float(model.nb_size)
        mu = model.E * np.exp(eta)
        s = r + mu
        return (y + r) * mu / s, (y + r) * r * mu / s ** 2, (y + r) * r * mu * (r - mu) / s ** 3
    p = 1.0 / (1.0 + np.exp(-eta))
    q = 1.0 / (1.0 + np.exp(eta))
    N = model.E
    return N * p, N * p * q, N * p * q * (q - p)


def dQ_dtheta(model, theta, j):
    """dQ/dtheta_j as a sparse matrix, differentiating the formulas above.

    j = 0: zero (Gaussian) or tau_b I on the fixed effects (Poisson).
    j = 1: log range;  j = 2: log sigma;  j = 3: logit rho.
    """
    h = hyper(theta, model.lik, model.tau_b)
    n_t, n_s, n_b = model.n_t, model.n_s, model.n_b
    C, G = fem_matrices(model)
    H = G @ sp.diags(1.0 / model.C_diag) @ G
    k2, tau2 = h["kappa"] ** 2, h["tau2"]
    Qt = temporal_Q(n_t, h["rho"])
    zero_tip = sp.csr_matrix((n_b, n_b))
    if j == 0:
        blk = sp.csr_matrix((n_t * n_s, n_t * n_s))
        tip = zero_tip if model.lik == "gaussian" else h["tau_b"] * sp.identity(n_b)
    elif j == 1:
        # kappa = sqrt(8) e^{-theta_2}: tau^2 kappa^4 scales as kappa^2, tau^2 kappa^2 is
        # constant, tau^2 as kappa^-2, so d/dtheta_2 gives -2, 0 and +2 times each term.
        dQs = tau2 * (-2.0 * k2 * k2 * C + 2.0 * H)
        blk = sp.kron(Qt, dQs)
        tip = zero_tip
    elif j == 2:
        blk = sp.kron(Qt, -2.0 * spatial_Q(model, theta))
        tip = zero_tip
    elif j == 3:
        rho = h["rho"]
        if n_t == 1:
            dQt = sp.csr_matrix((1, 1))
        else:
            d = np.full(n_t, 1.0 + rho * rho); d[0] = d[-1] = 1.0
            off = np.full(n_t - 1, -rho)
            T = sp.diags([off, d, off], [-1, 0, 1])
            dd = np.full(n_t, 2.0 * rho); dd[0] = dd[-1] = 0.0
            dT = sp.diags([np.full(n_t - 1, -1.0), dd, np.full(n_t - 1, -1.0)], [-1, 0, 1])
            dQt = (2.0 * rho / (1.0 - rho * rho) ** 2) * T + dT / (1.0 - rho * rho)
            dQt = dQt * (rho * (1.0 - rho))
        blk = sp.kron(dQt, spatial_Q(model, theta))
        tip = zero_tip
    else:
        raise ValueError(j)
    if n_b == 0:
        return sp.csr_matrix(blk)
    return sp.block_diag([blk, tip]).tocsr()
