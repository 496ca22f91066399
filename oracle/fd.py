"""Central-difference gradient (Eq. central_diff), and the forward-difference
variant the paper mixes in (d + 1 evaluations, first-order accurate).

d f / d theta_i ~ (f(theta + eps_i) - f(theta - eps_i)) / (2 ||eps_i||), with eps_i
= eps e_i.  The 2d + 1 evaluations (centre included) are independent, which
is what the paper parallelises (Sec. 3.1).
"""
import numpy as np


def central_gradient(f, theta, eps=1e-3):
    theta = np.asarray(theta, dtype=float)
    g = np.zeros(theta.size)
    for i in range(theta.size):
        e = np.zeros(theta.size)
        e[i] = eps
        g[i] = (f(theta + e) - f(theta - e)) / (2.0 * eps)
    return g


def gradient_from_stencil(f_values, eps=1e-3):
    """Gradient from f at the 2d+1 stencil points ordered centre, +e_0, -e_0, +e_1, ..."""
    f_values = np.asarray(f_values, dtype=float)
    d = (f_values.size - 1) // 2
    return np.array([(f_values[1 + 2 * j] - f_values[2 + 2 * j]) / (2.0 * eps) for j in range(d)])


def forward_gradient(f, theta, eps=1e-3):
    """d f / d theta_i ~ (f(theta + eps e_i) - f(theta)) / eps."""
    theta = np.asarray(theta, dtype=float)
    f0 = f(theta)
    g = np.zeros(theta.size)
    for i in range(theta.size):
        e = np.zeros(theta.size)
        e[i] = eps
        g[i] = (f(theta + e) - f0) / eps
    return g
