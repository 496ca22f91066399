"""GB300 library for the hyperparameter phase of INLA (Gaedke-Merzhaeuser et al.).

Batched evaluation of f(theta) = -log pi~(theta|y) (Eq. post_theta_approx),
its gradient, the latent mode and the marginal variances for a
spatio-temporal SPDE x AR(1) latent Gaussian model, by block-tridiagonal-
arrowhead factorisation and block Takahashi selected inversion in CUDA.
"""
from .build import LIB, build
from .api import (Model, gemm_f64, gemm_tf32x3, log_posterior, make_opts, measure_fp32_peak, measure_fp64_peak,
                  synth_build)
from . import capi

__all__ = ["LIB", "build", "Model", "gemm_f64", "gemm_tf32x3", "log_posterior", "make_opts", "measure_fp32_peak", "measure_fp64_peak", "synth_build", "capi"]
