"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds random-number generation and the construction of model inputs (mesh,
finite-element matrices, observation matrix, simulated data, hyperparameter
batches).  It contains none of the posterior computation.
"""
from .grid_model import (GridModel, build, config_model, theta_batch, fd_stencil, ccd_design,
                         line_points, grid_fem, locate, CONFIGS, FD_EPS,
                         THETA_TRUE_GAUSSIAN, THETA_TRUE_POISSON)
from .rng import Stream
