"""Element-wise recursions of Sec. 2.4 on tiny dense matrices (pure Python loops).

  cholesky          L_jj = sqrt(Q_jj - sum_{k<j} L_jk^2),
                    L_ij = (Q_ij - sum_{k<j} L_ik L_jk) / L_jj      (i > j)
  backward_solve    Eq. backward_solve: x_i = z_i / L_ii - (1/L_ii) sum_{k>i, L_ki != 0} L_ki x_k
  sel_inv_cov       Eq. sel_inv_cov: Sigma_ij = delta_ij / L_ii^2 - (1/L_ii) sum_{k>i, L_ki != 0} L_ki Sigma_kj
  takahashi         Eq. takahashi_recursion with Q = V D V^T, V unit lower, D diagonal:
                    Sigma_ij = delta_ij / D_ii - sum_{k>i, V_ki != 0} V_ki Sigma_kj     (i <= j)

The two inverse recursions run from Sigma_nn upwards.  ``selected=True``
computes only entries (i, j), i <= j, with L_ji != 0 (plus the diagonal):
the entries the selected inverse needs (Sec. 2.4.2).
"""
import math
import numpy as np


def cholesky(Q):
    Q = np.asarray(Q, dtype=float)
    n = Q.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        s = Q[j, j] - sum(L[j, k] ** 2 for k in range(j))
        if not s > 0.0:
            raise ValueError("matrix is not positive definite")
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (Q[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    return L


def backward_solve(L, z):
    n = L.shape[0]
    x = np.zeros(n)
    for i in reversed(range(n)):
        acc = sum(L[k, i] * x[k] for k in range(i + 1, n) if L[k, i] != 0.0)
        x[i] = z[i] / L[i, i] - acc / L[i, i]
    return x


def _needed(L, selected):
    n = L.shape[0]
    if not selected:
        return [[True] * n for _ in range(n)]
    # entry (i, j), i <= j, is needed when L_ji != 0 (the pattern of L, mirrored)
    return [[(i == j) or (j > i and L[j, i] != 0.0) for j in range(n)] for i in range(n)]


def sel_inv_cov(L, selected=False):
    """Eq. sel_inv_cov.  Returns a dense array with NaN where not computed."""
    n = L.shape[0]
    need = _needed(L, selected)
    S = np.full((n, n), np.nan)
    for i in reversed(range(n)):
        for j in reversed(range(i, n)):
            if not need[i][j]:
                continue
            acc = 0.0
            for k in range(i + 1, n):
                if L[k, i] != 0.0:
                    skj = S[k, j] if k <= j else S[j, k]
                    acc += L[k, i] * skj
            S[i, j] = (1.0 if i == j else 0.0) / L[i, i] ** 2 - acc / L[i, i]
            S[j, i] = S[i, j]
    return S


def takahashi(L, selected=False):
    """Eq. takahashi_recursion with V = L diag(L)^-1 and D = diag(L)^2."""
    n = L.shape[0]
    d = np.diag(L).copy()
    V = L / d[None, :]
    D = d * d
    need = _needed(L, selected)
    S = np.full((n, n), np.nan)
    for i in reversed(range(n)):
        for j in reversed(range(i, n)):
            if not need[i][j]:
                continue
            acc = 0.0
            for k in range(i + 1, n):
                if V[k, i] != 0.0:
                    skj = S[k, j] if k <= j else S[j, k]
                    acc += V[k, i] * skj
            S[i, j] = (1.0 if i == j else 0.0) / D[i] - acc
            S[j, i] = S[i, j]
    return S


def fill_pattern(Q):
    """Boolean nonzero pattern of the element-wise Cholesky factor of Q."""
    return cholesky(Q) != 0.0
