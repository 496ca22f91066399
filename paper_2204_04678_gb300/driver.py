"""Host drivers over the batched evaluation (no device code here).

* ``bfgs``: the mode search of the hyperparameter phase.  BFGS on f(theta)
  (Eq. bfgs_update) with the parallel line search of Sec. 3.2: the points of
  the search interval are evaluated in ONE batch, a quadratic is fitted to
  them by robust regression with bisquare weights, and its minimiser on the
  interval is the next iterate.
* ``integrate``: the integration stage (Sec. 2.2-2.3, Eq. LatParam): a finite-
  difference Hessian of f at the mode from a batch of gradients, a 25-point
  central composite design in the Hessian's eigenbasis evaluated in one batch
  with modes and marginal variances, and the mixture moments of pi(x_i | y).

The callables passed in evaluate batches (the GPU library through
``Model.eval`` in production; any evaluator in tests).
"""
import numpy as np

BISQUARE_C = 4.685          # Tukey bisquare tuning constant (95% efficiency at the normal)


def bisquare_quadratic(a, f, max_iter=50):
    """Fit q(a) = c0 + c1 a + c2 a^2 by iteratively reweighted least squares
    with bisquare weights w = (1 - (r / (c s))^2)^2 (0 beyond c s), where r are
    the residuals and s = MAD(r) / 0.6745.  Iterates until the weights repeat;
    returns (coefficients, the weights of the last fit)."""
    a = np.asarray(a, dtype=float)
    f = np.asarray(f, dtype=float)
    X = np.stack([np.ones_like(a), a, a * a], 1)
    w = np.ones_like(a)
    coef = np.zeros(3)
    for _ in range(max_iter):
        sw = np.sqrt(w)
        coef = np.linalg.lstsq(X * sw[:, None], f * sw, rcond=None)[0]
        r = f - X @ coef
        s = np.median(np.abs(r - np.median(r))) / 0.6745
        if not s > 1e-12 * max(1.0, np.abs(f).max()):
            break                       # (near) exact fit: nothing to down-weight
        u = r / (BISQUARE_C * s)
        w_new = np.where(np.abs(u) < 1.0, (1.0 - u * u) ** 2, 0.0)
        if np.abs(w_new - w).max() < 1e-12:
            break
        w = w_new
    return coef, w


def line_search_steps(gamma=1.0, n_inside=14, behind=(0.05, 0.1)):
    """Step lengths along the descent direction: n_inside uniform on (0, gamma]
    plus two just behind the current point (Sec. 3.2)."""
    return np.concatenate([gamma * np.arange(1, n_inside + 1) / n_inside, -np.asarray(behind, dtype=float)])


def parallel_line_search(eval_f_batch, theta, f0, d, gamma=1.0, max_shrink=6):
    """One parallel line search from theta along d on I = (theta, theta + gamma d].

    The 16 points of ``line_search_steps`` are evaluated in one batch.  If none
    on I improves on f0 the interval is shrunk tenfold and the batch repeated
    (at most max_shrink times).  Otherwise the bisquare quadratic through
    (0, f0) and the 16 points is minimised on I; where it has no interior
    minimum the best evaluated point is taken.  Returns (step, the interval's
    gamma, the last batch's points, their f); step = 0 when nothing improved.
    """
    for _ in range(max_shrink + 1):
        alphas = line_search_steps(gamma)
        pts = theta[None, :] + alphas[:, None] * d[None, :]
        fv = np.asarray(eval_f_batch(pts), dtype=float)
        inside = np.where(np.isfinite(fv) & (alphas > 0), fv, np.inf)
        if inside.min() < f0:
            break
        gamma *= 0.1
    else:
        return 0.0, gamma, pts, fv
    a = np.concatenate([[0.0], alphas])
    fa = np.concatenate([[f0], fv])
    ok = np.isfinite(fa)
    coef, _ = bisquare_quadratic(a[ok], fa[ok])
    best = float(alphas[int(np.argmin(inside))])
    step = best
    if coef[2] > 0:
        vertex = -coef[1] / (2.0 * coef[2])
        if 0.0 < vertex:
            step = float(min(vertex, gamma))
    return step, gamma, pts, fv


def bfgs(eval_f_grad, eval_f_batch, theta0, max_iter=50, gtol=1e-3, gamma=1.0, max_step=2.0, ftol=0.0,
         state=None, on_iteration=None):
    """Minimise f with BFGS (inverse-Hessian update, Eq. bfgs_update) and the
    parallel line search.

    eval_f_grad(theta) -> (f, grad) at one point (central differences or the
    adjoint); eval_f_batch(points [k, d]) -> f at k points (NaN where the
    evaluation failed, e.g. a precision matrix that is not positive definite).
    The search direction is capped at Euclidean length max_step (the first one
    at 1) and the initial inverse Hessian is the identity.  The interval
    length gamma_l adapts: it doubles (up to 8 gamma) after a step to its end
    and falls back towards gamma otherwise.  The step is accepted if it lowers
    f, else the best point of the batch is taken.  Stops when max |grad| <
    gtol, or when an iteration lowers f by less than ftol |f| (for evaluations
    whose rounding error exceeds what gtol asks).  Returns a dict with the
    final point, f, gradient, iteration count and the history of f.

    Checkpointing: on_iteration(state) is called after every iteration with the
    optimiser state (theta, f, grad, inverse Hessian, interval length,
    iteration, history); passing such a state back as `state` resumes the run
    exactly where it stopped (theta0 is then ignored).  save_state/load_state
    write and read it as JSON.
    """
    if state is not None:
        theta = np.asarray(state["theta"], dtype=float).copy()
        f, g = float(state["f"]), np.asarray(state["grad"], dtype=float).copy()
        Hinv = np.asarray(state["Hinv"], dtype=float).copy()
        gam = float(state["gamma"])
        start = int(state["iteration"])
        hist = list(state["history"])
        dim = theta.size
    else:
        theta = np.asarray(theta0, dtype=float).copy()
        dim = theta.size
        Hinv = np.eye(dim)
        f, g = eval_f_grad(theta)
        hist = [f]
        gam = gamma
        start = 0
    it = start
    for it in range(start + 1, max_iter + 1):
        if np.abs(g).max() < gtol:
            it -= 1
            break
        d = -Hinv @ g
        if g @ d >= 0:                                  # not a descent direction: restart
            Hinv = np.eye(dim)
            d = -g
        cap = 1.0 if it == 1 else max_step
        d = d * min(1.0, cap / np.linalg.norm(d))
        step, used, pts, fv = parallel_line_search(eval_f_batch, theta, f, d, gam)
        # next interval: twice as long after a step to its end, back towards gamma otherwise
        gam = min(8.0 * gamma, 2.0 * used) if step >= used else max(gamma, 0.5 * used)
        if step <= 0.0:
            it -= 1
            break
        theta_new = theta + step * d
        f_new, g_new = eval_f_grad(theta_new)
        if not np.isfinite(f_new) or f_new > f:         # take the best evaluated point instead
            k = int(np.argmin(np.where(np.isfinite(fv), fv, np.inf)))
            theta_new = pts[k]
            f_new, g_new = eval_f_grad(theta_new)
        s, y = theta_new - theta, g_new - g
        sy = float(s @ y)
        if sy > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            rho = 1.0 / sy
            V = np.eye(dim) - rho * np.outer(s, y)
            Hinv = V @ Hinv @ V.T + rho * np.outer(s, s)
        done = f - f_new < ftol * abs(f)
        theta, f, g = theta_new, f_new, g_new
        hist.append(f)
        if on_iteration is not None:
            on_iteration(dict(theta=theta.copy(), f=f, grad=g.copy(), Hinv=Hinv.copy(), gamma=gam, iteration=it,
                              history=list(hist)))
        if done:
            break
    return dict(theta=theta, f=f, grad=g, iterations=it, history=np.array(hist))


def save_state(path, state):
    """Write a BFGS state (from on_iteration) as JSON."""
    import json
    plain = {k: (np.asarray(v).tolist() if isinstance(v, (np.ndarray, list)) else v) for k, v in state.items()}
    with open(path, "w") as fh:
        json.dump(plain, fh)


def load_state(path):
    """Read a BFGS state written by save_state."""
    import json
    with open(path) as fh:
        return json.load(fh)


def ccd_unit_design(dim=4):
    """Rotatable central composite design in `dim` = 4 dimensions: the centre, the
    axial points +/- 2 e_j and the 2^4 corners (radius 2 = sqrt(dim))."""
    pts = [np.zeros(dim)]
    for j in range(dim):
        for s in (2.0, -2.0):
            v = np.zeros(dim)
            v[j] = s
            pts.append(v)
    for k in range(2 ** dim):
        pts.append(np.array([1.0 if (k >> j) & 1 else -1.0 for j in range(dim)]))
    return np.array(pts)


def integrate(eval_grad_batch, eval_full_batch, theta_mode, h=1e-3, scale=1.0):
    """Integration stage around the mode.

    eval_grad_batch(points) -> gradients [k, d]; eval_full_batch(points) ->
    (f [k], x_mode [k, n], marg_var [k, n]).  The Hessian of f at the mode is
    the central difference of gradients; the design points are
    theta_mode + V diag(lambda)^-1/2 (scale z_k) for the unit CCD z_k; the
    weights are proportional to exp(f(mode) - f(theta_k)) (equal design
    weights); pi(x_i | y) is the mixture sum_k w_k N(x*_k, v_k) (Eq. LatParam).
    """
    theta_mode = np.asarray(theta_mode, dtype=float)
    dim = theta_mode.size
    E = np.eye(dim) * h
    pts = np.concatenate([theta_mode[None, :] + E, theta_mode[None, :] - E])
    G = np.asarray(eval_grad_batch(pts), dtype=float)
    H = (G[:dim] - G[dim:]).T / (2.0 * h)
    H = 0.5 * (H + H.T)
    lam, V = np.linalg.eigh(H)
    V = V * np.where(V[np.abs(V).argmax(0), np.arange(dim)] < 0, -1.0, 1.0)   # canonical signs
    if np.any(lam <= 0):
        raise ValueError("Hessian at the mode is not positive definite")
    Z = ccd_unit_design(dim) * scale
    design = theta_mode[None, :] + (Z / np.sqrt(lam)[None, :]) @ V.T
    f, xm, mv = eval_full_batch(design)
    f = np.asarray(f, dtype=float)
    lw = -(f - f.min())
    w = np.exp(lw)
    w /= w.sum()
    mean = w @ xm
    var = w @ (mv + xm * xm) - mean * mean
    theta_mean = w @ design
    theta_cov = (design - theta_mean).T @ (w[:, None] * (design - theta_mean))
    return dict(hessian=H, design=design, f=f, weights=w, x_mean=mean, x_var=var,
                theta_mean=theta_mean, theta_cov=theta_cov)


def model_evaluators(model, grad="adjoint", precision="fp64", fd_eps=1e-3):
    """The four batch callables of ``bfgs`` and ``integrate`` over a ``Model``
    (every evaluation is one ``inla_eval_batch`` call on the device).

    grad = "fd": the gradient of each point comes from its 2d + 1 central-
    difference stencil in the same batch; "adjoint": from the selected inverse.
    """
    import torch

    def _theta(points):
        return torch.as_tensor(np.atleast_2d(np.asarray(points, dtype=float)), dtype=torch.float64,
                               device=f"cuda:{model.device}")

    def _checked(r):
        st = r["status"].cpu().numpy()
        if np.any(st != 0):
            raise RuntimeError(f"evaluation failed with status {st.tolist()}")
        return r

    def f_grad(theta):
        r = _checked(model.eval(_theta(theta), grad=grad, precision=precision, fd_eps=fd_eps))
        return float(r["f"][0]), r["grad"][0].cpu().numpy()

    def f_batch(points):
        r = model.eval(_theta(points), grad="none", precision=precision)
        f = r["f"].cpu().numpy().copy()
        f[r["status"].cpu().numpy() != 0] = np.nan
        return f

    def grad_batch(points):
        r = _checked(model.eval(_theta(points), grad=grad, precision=precision, fd_eps=fd_eps))
        return r["grad"].cpu().numpy()

    def full_batch(points):
        r = _checked(model.eval(_theta(points), grad="none", precision=precision, want_mode=True,
                                want_marg_var=True))
        return r["f"].cpu().numpy(), r["x_mode"].cpu().numpy(), r["marg_var"].cpu().numpy()

    return f_grad, f_batch, grad_batch, full_batch
