"""ctypes declarations of the C ABI in include/inla_gpu.h (same names).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  Loading fails loudly if the library has not been built.
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

from .build import LIB, PROBE_LIB

INLA_OK = 0
INLA_ERR_ARG = 1
INLA_ERR_CUDA = 2
INLA_ERR_OOM = 3
INLA_ERR_NOT_SPD = 4
INLA_ERR_NO_CONVERGENCE = 5
INLA_ERR_TIMEOUT = 6
INLA_ERR_UNSUPPORTED = 7
INLA_LIK_GAUSSIAN = 0
INLA_LIK_POISSON = 1
INLA_LIK_BINOMIAL = 2
INLA_LIK_NEGBINOMIAL = 3
INLA_GRAD_NONE = 0
INLA_GRAD_FD_CENTRAL = 1
INLA_GRAD_ADJOINT = 2
INLA_GRAD_FD_FORWARD = 3
INLA_PRIOR_KRONECKER = 0
INLA_PRIOR_BTA = 1
INLA_FP64 = 0
INLA_MIXED = 1
INLA_GEMM_TF32X3 = 3
INLA_SWEEP_TF32X3 = 3
INLA_INV_BLOCKED = 4
KERNEL_GJ_UPDATE = 0
KERNEL_GEMM = 1
KERNEL_GJ_PIVOT = 2
KERNEL_GJ_PANEL = 3
KERNEL_GJ_UPDATE32 = 4

STATIC_SCRATCH_BYTES = 64 << 20

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_SPD",
                5: "ERR_NO_CONVERGENCE", 6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class inla_model_desc(ctypes.Structure):
    _fields_ = [("n_t", c_int32), ("n_s", c_int32), ("n_b", c_int32), ("lik", c_int32), ("m", c_int64),
                ("C_diag", POINTER(c_double)),
                ("G_rowptr", POINTER(c_int32)), ("G_col", POINTER(c_int32)), ("G_val", POINTER(c_double)),
                ("A_rowptr", POINTER(c_int64)), ("A_col", POINTER(c_int32)), ("A_val", POINTER(c_double)),
                ("y", POINTER(c_double)), ("E", POINTER(c_double)),
                ("tau_b", c_double), ("prior_mean", c_double * 4), ("prior_sd", c_double * 4),
                ("nb_size", c_double)]


class inla_eval_opts(ctypes.Structure):
    _fields_ = [("grad", c_int32), ("prior_mode", c_int32), ("precision", c_int32), ("want_mode", c_int32),
                ("want_marg_var", c_int32), ("max_newton", c_int32), ("newton_tol", c_double),
                ("fd_eps", c_double), ("use_graph", c_int32)]


class inla_eval_out(ctypes.Structure):
    _fields_ = [("f_dev", c_void_p), ("grad_dev", c_void_p), ("x_mode_dev", c_void_p),
                ("marg_var_dev", c_void_p), ("status_dev", c_void_p), ("newton_iters_dev", c_void_p)]


class inla_eval_out_host(ctypes.Structure):
    _fields_ = [("f", c_void_p), ("grad", c_void_p), ("x_mode", c_void_p), ("marg_var", c_void_p),
                ("status", c_void_p), ("newton_iters", c_void_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "inla_model_create": (c_int, [POINTER(inla_model_desc), c_int, POINTER(c_void_p)]),
    "inla_workspace_bytes": (c_int, [c_void_p, c_int, POINTER(inla_eval_opts), POINTER(c_size_t)]),
    "inla_eval_batch": (c_int, [c_void_p, c_int, c_void_p, POINTER(inla_eval_opts), POINTER(inla_eval_out),
                                c_void_p]),
    "inla_eval_batch_static": (c_int, [c_void_p, c_int, c_void_p, POINTER(inla_eval_opts), POINTER(inla_eval_out),
                                       c_void_p]),
    "inla_eval_batch_host": (c_int, [c_void_p, c_int, c_void_p, POINTER(inla_eval_opts),
                                     POINTER(inla_eval_out_host)]),
    "inla_autotune": (c_int, [c_void_p, c_int, c_void_p, POINTER(inla_eval_opts), POINTER(c_int32)]),
    "inla_set_tiles": (c_int, [c_void_p, c_int, c_int, c_int]),
    "inla_set_wait_limit": (c_int, [c_double]),
    "inla_set_fp64_products": (c_int, [c_void_p, c_int]),
    "inla_set_time_partition": (c_int, [c_void_p, c_int]),
    "inla_set_point_groups": (c_int, [c_void_p, c_int]),
    "inla_model_latent_dim": (c_int64, [c_void_p]),
    "inla_last_launch_count": (c_int64, [c_void_p]),
    "inla_model_destroy": (None, [c_void_p]),
    "inla_last_error": (c_char_p, []),
    "inla_gemm_tf32x3": (c_int, [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "inla_gemm_f64": (c_int, [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "inla_gemm_f64_workspace_bytes": (c_size_t, [c_int, c_int]),
    "inla_synth_build": (c_int, [c_int32, c_int32, c_int32, c_int64, c_int32, c_uint64, c_void_p,
                                 POINTER(inla_model_desc), POINTER(c_void_p)]),
    "inla_synth_grid_model": (c_int, [c_int32, c_uint64, POINTER(inla_model_desc), POINTER(c_void_p)]),
    "inla_synth_free": (None, [c_void_p]),
    "inla_profile_enable": (c_int, [c_void_p, c_int]),
    "inla_profile_read": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_int64), POINTER(c_double)]),
}

# include/inla_probe.h (libinla_probe.so, the benchmark's throughput probes)
PROBE_SIGNATURES = {
    "inla_measure_fp64_peak": (c_int, [c_int, c_int, POINTER(c_double)]),
    "inla_measure_fp32_peak": (c_int, [c_int, POINTER(c_double)]),
    "inla_probe_last_error": (c_char_p, []),
}

_lib = None
_probe = None


def load_probe(path: str = PROBE_LIB):
    """Load the probe library (measurement utilities, not the evaluation path)."""
    global _probe
    if _probe is not None:
        return _probe
    if not os.path.exists(path):
        raise RuntimeError(f"libinla_probe.so not found at {path}: build it first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROBE_SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _probe = lib
    return lib


def load(path: str = LIB):
    """Load the shared library and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libinla_gpu.so not found at {path}: build it first "
                           "(python -m paper_2204_04678_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class InlaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code):
    if code != INLA_OK:
        msg = load().inla_last_error()
        raise InlaError(code, msg.decode() if msg else "")
