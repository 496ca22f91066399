"""Seeded synthetic spatio-temporal workloads (inputs only).

A workload is the data of a latent Gaussian model (Sec. 2.1): a regular
triangulated grid on the unit square with its P1 finite-element matrices
(lumped mass C, stiffness G), an observation matrix A whose rows hold the
three barycentric weights of a random location in one time slice plus n_b
covariates, and observations y simulated from a smooth spatio-temporal
field.  The latent vector is ordered time-major with the fixed effects
last: x = (u_0, ..., u_{n_t-1}, beta), n = n_t * n_s + n_b.

Both the CPU oracle and the GPU library consume these arrays; neither
imports the other.  Nothing here evaluates the INLA posterior: the
simulated field is drawn from a continuous Matern(nu = 1) field with
random Fourier features and an AR(1) recursion in time, not from any
precision matrix the method assembles.

Substream ids (seed 0 unless stated): 0 observation times, 1 observation
locations, 2 covariates, 3 field, 4 beta, 5 noise / Poisson / binomial /
negative-binomial draws, 6 exposure / numbers of trials (1..10), 7
hyperparameter batch.
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import Stream

THETA_TRUE_GAUSSIAN = np.array([1.0, -1.0, 0.0, 1.5])
THETA_TRUE_POISSON = np.array([np.log(1e-3), -1.0, 0.0, 1.5])
FD_EPS = 1e-3
NB_SIZE = 4   # size (overdispersion) r of the negative-binomial workloads, a fixed model constant


@dataclass
class GridModel:
    """Inputs of one workload.  Arrays are float64 / int32 / int64, C order."""
    name: str
    n_t: int
    nx: int
    n_b: int
    m: int
    lik: str                      # "gaussian", "poisson" or "binomial"
    tau_b: float                  # fixed-effect prior precision (Gaussian)
    C_diag: np.ndarray            # [n_s] lumped mass
    G_rowptr: np.ndarray          # CSR of the n_s x n_s stiffness matrix,
    G_col: np.ndarray             #   every triangle edge stored (some values
    G_val: np.ndarray             #   are exactly zero on right triangles)
    A_rowptr: np.ndarray          # CSR of the m x n observation matrix (int64)
    A_col: np.ndarray             # int32 column indices
    A_val: np.ndarray
    y: np.ndarray                 # [m]
    E: np.ndarray = None          # [m] exposure (Poisson, negative binomial) / number of trials (binomial)
    nb_size: float = 0.0          # negative binomial size r (0 for the other likelihoods)
    prior_mean: np.ndarray = field(default_factory=lambda: np.zeros(4))
    prior_sd: np.ndarray = field(default_factory=lambda: np.full(4, 10.0))
    obs_t: np.ndarray = None      # [m] time slice of each observation
    theta_true: np.ndarray = None

    @property
    def n_s(self):
        return self.nx * self.nx

    @property
    def n(self):
        return self.n_t * self.n_s + self.n_b

    @property
    def d(self):
        return 4


def grid_fem(nx: int):
    """P1 finite elements on an nx-by-nx vertex grid of [0,1]^2.

    Vertex k = i + nx*j sits at (i*h, j*h), h = 1/(nx-1).  Cell (i, j) is cut
    along its diagonal (i,j)-(i+1,j+1) into T1 = {(i,j),(i+1,j),(i+1,j+1)} and
    T2 = {(i,j),(i+1,j+1),(i,j+1)}.  Returns the lumped mass diagonal
    C_kk = sum over triangles T containing k of |T|/3, and the stiffness
    G_kl = sum_T integral_T grad(phi_k).grad(phi_l) in CSR with every
    triangle edge stored, sorted columns.
    """
    if nx < 2:
        raise ValueError("nx must be >= 2")
    h = 1.0 / (nx - 1)
    n_s = nx * nx
    area = 0.5 * h * h
    C = np.zeros(n_s)
    rows, cols, vals = [], [], []
    # reference gradients (times h) of the three hat functions on each triangle
    grads_T1 = np.array([[-1.0, 0.0], [1.0, -1.0], [0.0, 1.0]]) / h
    grads_T2 = np.array([[0.0, -1.0], [1.0, 0.0], [-1.0, 1.0]]) / h
    KT1 = area * grads_T1 @ grads_T1.T
    KT2 = area * grads_T2 @ grads_T2.T
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(nx - 1), indexing="ij")
    i = i.ravel(); j = j.ravel()
    v00 = i + nx * j
    v10 = (i + 1) + nx * j
    v11 = (i + 1) + nx * (j + 1)
    v01 = i + nx * (j + 1)
    for tri, K in (((v00, v10, v11), KT1), ((v00, v11, v01), KT2)):
        for a in range(3):
            np.add.at(C, tri[a], area / 3.0)
            for b in range(3):
                rows.append(tri[a]); cols.append(tri[b])
                vals.append(np.full(tri[a].shape, K[a, b]))
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    key = rows.astype(np.int64) * n_s + cols
    order = np.argsort(key, kind="stable")
    key = key[order]; vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start)
    r = (uniq // n_s).astype(np.int64)
    c = (uniq % n_s).astype(np.int32)
    rowptr = np.zeros(n_s + 1, dtype=np.int32)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    # stiffness rows sum to zero; clean the rounding of that identity
    return C, rowptr, c, summed


def locate(nx: int, px: np.ndarray, py: np.ndarray):
    """Triangle vertices and barycentric weights of points in [0,1]^2.

    The cell is (floor(x/h), floor(y/h)) clamped to nx-2; within it the point
    belongs to T1 when (x - x_i) >= (y - y_j), else to T2 (points on the
    diagonal go to T1).
    """
    h = 1.0 / (nx - 1)
    ci = np.minimum(np.floor(px / h).astype(np.int64), nx - 2)
    cj = np.minimum(np.floor(py / h).astype(np.int64), nx - 2)
    dx = (px - ci * h) / h
    dy = (py - cj * h) / h
    t1 = dx >= dy
    v00 = ci + nx * cj
    v10 = (ci + 1) + nx * cj
    v11 = (ci + 1) + nx * (cj + 1)
    v01 = ci + nx * (cj + 1)
    verts = np.where(t1[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1))
    w = np.where(t1[:, None],
                 np.stack([1.0 - dx, dx - dy, dy], 1),
                 np.stack([1.0 - dy, dx, dy - dx], 1))
    return verts, w


def matern_field(stream: Stream, nx: int, n_t: int, range_: float, sigma: float, rho: float,
                 n_features: int = 128):
    """A smooth space-time field on the grid vertices, shape [n_t, n_s].

    Space: a stationary Matern(nu = 1) field on R^2 with range r
    (kappa = sqrt(8)/r) and marginal sd sigma, by random Fourier features.
    Its spectral density is proportional to (kappa^2 + |w|^2)^-2, so
    |w| = kappa * sqrt(U / (1 - U)) by inversion and the direction is
    uniform.  Time: u_t = rho u_{t-1} + sqrt(1 - rho^2) e_t with
    independent spatial innovations e_t and a stationary start.
    """
    h = 1.0 / (nx - 1)
    g = np.arange(nx) * h
    X = np.tile(g, nx)            # vertex k = i + nx*j -> x = i*h
    Y = np.repeat(g, nx)          #                     -> y = j*h
    kappa = np.sqrt(8.0) / range_
    out = np.empty((n_t, nx * nx))
    prev = None
    for t in range(n_t):
        u = stream.uniform_open(n_features)
        ang = 2.0 * np.pi * stream.uniform(n_features)
        phase = 2.0 * np.pi * stream.uniform(n_features)
        r = kappa * np.sqrt(u / (1.0 - u))
        wx = r * np.cos(ang); wy = r * np.sin(ang)
        e = sigma * np.sqrt(2.0 / n_features) * np.cos(np.outer(X, wx) + np.outer(Y, wy) + phase).sum(1)
        cur = e if prev is None else rho * prev + np.sqrt(1.0 - rho * rho) * e
        out[t] = cur
        prev = cur
    return out


def build(name: str, n_t: int, nx: int, n_b: int, m: int, lik: str = "gaussian", seed: int = 0,
          theta_true=None, tau_b: float = 1e-3) -> GridModel:
    """Build one workload.  See the module docstring for the recipe."""
    if lik not in ("gaussian", "poisson", "binomial", "negbinomial"):
        raise ValueError(lik)
    theta_true = np.array(theta_true if theta_true is not None else
                          (THETA_TRUE_GAUSSIAN if lik == "gaussian" else THETA_TRUE_POISSON), dtype=float)
    n_s = nx * nx
    C, G_rowptr, G_col, G_val = grid_fem(nx)
    s_time, s_loc, s_cov = Stream(seed, 0), Stream(seed, 1), Stream(seed, 2)
    s_field, s_beta, s_noise, s_exp = Stream(seed, 3), Stream(seed, 4), Stream(seed, 5), Stream(seed, 6)
    obs_t = s_time.integers(m, n_t)
    loc = s_loc.uniform(2 * m).reshape(m, 2)
    Z = s_cov.normal(m * n_b).reshape(m, n_b) if n_b else np.zeros((m, 0))
    verts, w = locate(nx, loc[:, 0], loc[:, 1])
    # A in CSR: 3 spatial entries (sorted by column) then the n_b covariates
    order = np.argsort(verts, axis=1, kind="stable")
    verts = np.take_along_axis(verts, order, 1)
    w = np.take_along_axis(w, order, 1)
    nnz_row = 3 + n_b
    A_col = np.empty((m, nnz_row), dtype=np.int32)
    A_val = np.empty((m, nnz_row))
    A_col[:, :3] = obs_t[:, None] * n_s + verts
    A_val[:, :3] = w
    A_col[:, 3:] = n_t * n_s + np.arange(n_b)[None, :]
    A_val[:, 3:] = Z
    A_rowptr = np.arange(m + 1, dtype=np.int64) * nnz_row
    # truth
    range_ = np.exp(theta_true[1]); sigma = np.exp(theta_true[2])
    rho = 1.0 / (1.0 + np.exp(-theta_true[3]))
    u = matern_field(s_field, nx, n_t, range_, sigma, rho)
    beta = s_beta.normal(n_b) * (1.0 if lik == "gaussian" else 0.1)
    eta = (w * u[obs_t[:, None], verts]).sum(1) + Z @ beta
    E = None
    if lik == "gaussian":
        tau_y = np.exp(theta_true[0])
        y = eta + s_noise.normal(m) / np.sqrt(tau_y)
        prior_mean = np.zeros(4)
    elif lik == "poisson":
        E = 0.5 + 1.5 * s_exp.uniform(m)
        y = s_noise.poisson(E * np.exp(eta)).astype(np.float64)
        prior_mean = np.array([np.log(1e-3), 0.0, 0.0, 0.0])
    elif lik == "negbinomial":
        E = 0.5 + 1.5 * s_exp.uniform(m)
        y = s_noise.negbinomial(NB_SIZE, E * np.exp(eta)).astype(np.float64)
        prior_mean = np.array([np.log(1e-3), 0.0, 0.0, 0.0])
    else:
        trials = 1 + s_exp.integers(m, 10)
        E = trials.astype(np.float64)
        y = s_noise.binomial(trials, 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
        prior_mean = np.array([np.log(1e-3), 0.0, 0.0, 0.0])
    return GridModel(name=name, n_t=n_t, nx=nx, n_b=n_b, m=m, lik=lik, tau_b=tau_b,
                     nb_size=float(NB_SIZE) if lik == "negbinomial" else 0.0,
                     C_diag=C, G_rowptr=G_rowptr, G_col=G_col, G_val=G_val,
                     A_rowptr=A_rowptr, A_col=A_col.ravel(), A_val=A_val.ravel(), y=y, E=E,
                     prior_mean=prior_mean, prior_sd=np.full(4, 10.0), obs_t=obs_t,
                     theta_true=theta_true)


# The five workloads: (n_t, nx, n_b, m, likelihood).
CONFIGS = {
    1: dict(name="st-spde-ar1 nt8 8x8 nb2 m2000 gaussian", n_t=8, nx=8, n_b=2, m=2000, lik="gaussian"),
    2: dict(name="st-spde-ar1 nt50 32x32 nb4 m100k gaussian", n_t=50, nx=32, n_b=4, m=100_000, lik="gaussian"),
    3: dict(name="st-spde-ar1 nt100 45x45 nb6 m400k gaussian", n_t=100, nx=45, n_b=6, m=400_000, lik="gaussian"),
    4: dict(name="st-spde-ar1 nt200 50x50 nb6 m1M gaussian", n_t=200, nx=50, n_b=6, m=1_000_000, lik="gaussian"),
    5: dict(name="st-spde-ar1 nt100 64x64 nb8 m500k poisson", n_t=100, nx=64, n_b=8, m=500_000, lik="poisson"),
}


def config_model(cfg: int, seed: int = 0) -> GridModel:
    return build(seed=seed, **CONFIGS[cfg])


def fd_stencil(center: np.ndarray, eps: float = FD_EPS) -> np.ndarray:
    """The 2d+1 points of the central-difference gradient (Eq. central_diff):
    row 0 is the centre, rows 1+2j and 2+2j are centre +/- eps e_j."""
    center = np.asarray(center, dtype=float)
    d = center.size
    pts = np.repeat(center[None, :], 2 * d + 1, 0)
    for j in range(d):
        pts[1 + 2 * j, j] += eps
        pts[2 + 2 * j, j] -= eps
    return pts


def ccd_design(center: np.ndarray, step: float = 0.1) -> np.ndarray:
    """25-point rotatable central composite design in d = 4 around center:
    the centre, the 8 axial points +/-2 e_j and the 16 corners {+/-1}^4."""
    center = np.asarray(center, dtype=float)
    d = center.size
    pts = [np.zeros(d)]
    for j in range(d):
        for s in (2.0, -2.0):
            v = np.zeros(d); v[j] = s; pts.append(v)
    for k in range(2 ** d):
        pts.append(np.array([1.0 if (k >> j) & 1 else -1.0 for j in range(d)]))
    return center[None, :] + step * np.array(pts)


def line_points(center: np.ndarray, direction: np.ndarray, gamma: float = 0.5) -> np.ndarray:
    """16 line-search points: 14 uniform on (centre, centre + gamma p] plus two
    just behind the centre at -0.05 p and -0.1 p (Sec. 3.2)."""
    p = np.asarray(direction, dtype=float)
    p = p / np.linalg.norm(p)
    a = np.concatenate([gamma * np.arange(1, 15) / 14.0, [-0.05, -0.1]])
    return np.asarray(center, dtype=float)[None, :] + a[:, None] * p[None, :]


def theta_batch(cfg: int, model: GridModel, seed: int = 0) -> np.ndarray:
    """The hyperparameter batch of a workload, [B, 4]."""
    s = Stream(seed, 7)
    if cfg == 1:
        return fd_stencil(model.theta_true)
    center = model.theta_true + 0.1 * s.normal(4)
    if cfg in (2, 4):
        return fd_stencil(center)
    if cfg == 3:
        return line_points(center, s.normal(4))
    return ccd_design(center)
