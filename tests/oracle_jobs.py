"""Oracle jobs for the full-size parity tests, run in spawn worker processes.

Kept apart from the test modules so that the workers import only numpy,
scipy, ``synth`` and ``oracle`` (no torch, no CUDA).
"""
import os

import numpy as np

from synth import CONFIGS, build, theta_batch


def shortened(cfg, n_t):
    """A benchmark workload with fewer time steps (same mesh, n_b, likelihood and
    observations per time step)."""
    c = dict(CONFIGS[cfg])
    c["m"] = c["m"] * n_t // c["n_t"]
    c["n_t"] = n_t
    c["name"] = c["name"] + f" shortened to n_t={n_t}"
    return c


CASES = {"c2": dict(CONFIGS[2]), "c3s": shortened(3, 20), "c4s": shortened(4, 12), "c5s": shortened(5, 2)}


def model(key):
    return build(**CASES[key])


def centre(key):
    mdl = model(key)
    if key.startswith("c5"):
        return mdl.theta_true + np.array([0.05, -0.05, 0.05, -0.05])
    return theta_batch(2, mdl)[0]


BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def set_threads(threads):
    """BLAS threads of worker processes started after this call (set in the parent)."""
    for v in BLAS_ENV:
        os.environ[v] = str(threads)


def evaluate(key, theta, want):
    from oracle import bta
    r = bta.evaluate(model(key), np.asarray(theta), want_grad=want, want_var=want)
    return {k: r[k] for k in ("f", "x", "var", "grad", "iters") if k in r}
