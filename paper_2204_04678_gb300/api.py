"""Python binding of the C ABI: model construction, batched evaluation and a
``torch.autograd.Function`` for f(theta).

PyTorch only provides device memory and the stream; the arithmetic runs in
libinla_gpu.so.  There is no CPU fallback: without the library (or without
a CUDA device) every call raises.
"""
import ctypes
from ctypes import byref, c_double, c_size_t, c_void_p

import numpy as np

from . import capi as C

_GRAD = {"none": C.INLA_GRAD_NONE, "fd": C.INLA_GRAD_FD_CENTRAL, "adjoint": C.INLA_GRAD_ADJOINT,
         "fd_forward": C.INLA_GRAD_FD_FORWARD}
_PRIOR = {"kronecker": C.INLA_PRIOR_KRONECKER, "bta": C.INLA_PRIOR_BTA}


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


_PREC = {"fp64": C.INLA_FP64, "mixed": C.INLA_MIXED}


def make_opts(grad="none", prior="kronecker", want_mode=False, want_marg_var=False, max_newton=50,
              newton_tol=1e-8, fd_eps=1e-3, precision="fp64", use_graph=False):
    o = C.inla_eval_opts()
    o.grad = _GRAD[grad]
    o.prior_mode = _PRIOR[prior]
    o.precision = _PREC[precision]
    o.want_mode = int(bool(want_mode))
    o.want_marg_var = int(bool(want_marg_var))
    o.max_newton = int(max_newton)
    o.newton_tol = float(newton_tol)
    o.fd_eps = float(fd_eps)
    o.use_graph = int(bool(use_graph))
    return o


class Model:
    """A spatio-temporal latent Gaussian model resident on one GPU.

    ``data`` provides n_t, n_s, n_b, m, lik ('gaussian' / 'poisson'), C_diag,
    G (CSR: G_rowptr, G_col, G_val), A (CSR: A_rowptr int64, A_col, A_val),
    y, E (Poisson / negative-binomial exposures, binomial trials), tau_b,
    prior_mean[4], prior_sd[4], nb_size (negative binomial) (e.g. ``synth.GridModel``);
    lik is "gaussian", "poisson", "binomial" or "negbinomial".
    """

    def __init__(self, data, device: int = 0):
        self.lib = C.load()
        arr = lambda x, dt: np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep = dict(C=arr(data.C_diag, np.float64), Gr=arr(data.G_rowptr, np.int32), Gc=arr(data.G_col, np.int32),
                    Gv=arr(data.G_val, np.float64), Ar=arr(data.A_rowptr, np.int64), Ac=arr(data.A_col, np.int32),
                    Av=arr(data.A_val, np.float64), y=arr(data.y, np.float64))
        d = C.inla_model_desc()
        d.n_t, d.n_s, d.n_b, d.m = int(data.n_t), int(data.n_s), int(data.n_b), int(data.m)
        d.lik = {"gaussian": C.INLA_LIK_GAUSSIAN, "poisson": C.INLA_LIK_POISSON,
                 "binomial": C.INLA_LIK_BINOMIAL, "negbinomial": C.INLA_LIK_NEGBINOMIAL}[data.lik]
        d.nb_size = float(getattr(data, "nb_size", 0.0) or 0.0)
        d.C_diag = _ptr(keep["C"], c_double)
        d.G_rowptr = _ptr(keep["Gr"], ctypes.c_int32)
        d.G_col = _ptr(keep["Gc"], ctypes.c_int32)
        d.G_val = _ptr(keep["Gv"], c_double)
        d.A_rowptr = _ptr(keep["Ar"], ctypes.c_int64)
        d.A_col = _ptr(keep["Ac"], ctypes.c_int32)
        d.A_val = _ptr(keep["Av"], c_double)
        d.y = _ptr(keep["y"], c_double)
        if getattr(data, "E", None) is not None:
            keep["E"] = arr(data.E, np.float64)
            d.E = _ptr(keep["E"], c_double)
        d.tau_b = float(data.tau_b)
        for j in range(4):
            d.prior_mean[j] = float(data.prior_mean[j])
            d.prior_sd[j] = float(data.prior_sd[j])
        h = c_void_p()
        C.check(self.lib.inla_model_create(byref(d), int(device), byref(h)))
        self.handle = h
        self.device = int(device)
        self.n = int(self.lib.inla_model_latent_dim(h))
        self.n_t, self.n_s, self.n_b, self.m = d.n_t, d.n_s, d.n_b, d.m
        self.lik = data.lik

    def close(self):
        if getattr(self, "handle", None):
            self.lib.inla_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, B, **kw):
        out = c_size_t()
        o = make_opts(**kw)
        C.check(self.lib.inla_workspace_bytes(self.handle, int(B), byref(o), byref(out)))
        return out.value

    def autotune(self, theta, grad="none", precision="fp64", **kw):
        """Pick the fastest block-tile shapes for this batch; returns the chosen
        (FP64 sweep width, FP32 sweep width, FP32 GEMM tile)."""
        theta = theta.contiguous()
        o = make_opts(grad=grad, precision=precision, **kw)
        ch = (ctypes.c_int32 * 3)()
        C.check(self.lib.inla_autotune(self.handle, int(theta.shape[0]), c_void_p(theta.data_ptr()), byref(o), ch))
        return tuple(ch)

    def set_tiles(self, sweep_fp64=32, sweep_fp32=64, gemm_fp32=128):
        C.check(self.lib.inla_set_tiles(self.handle, int(sweep_fp64), int(sweep_fp32), int(gemm_fp32)))

    def set_fp64_products(self, tensor=True):
        """FP64 selected-inversion products on the BF16 tensor cores (digit
        splitting; the default) or with FP64 FMA on the CUDA cores."""
        C.check(self.lib.inla_set_fp64_products(self.handle, int(bool(tensor))))

    def set_time_partition(self, parts=2):
        """Split the time chain at its middle block into two independent
        elimination chains (parts = 2, the default; nested dissection, Sec. 3.3)
        for factorisations that no selected inversion follows, or keep one
        chain (parts = 1)."""
        C.check(self.lib.inla_set_time_partition(self.handle, int(parts)))

    def set_point_groups(self, groups=2):
        """Factorise a Gaussian call's points as two concurrent groups (groups = 2,
        the default) or as one batch (groups = 1)."""
        C.check(self.lib.inla_set_point_groups(self.handle, int(groups)))

    def last_launch_count(self):
        return int(self.lib.inla_last_launch_count(self.handle))

    def profile_enable(self, every=1):
        """Time every `every`-th launch of the instrumented kernels (0 = off)."""
        C.check(self.lib.inla_profile_enable(self.handle, int(every)))

    def profile_read(self, kernel):
        """(total_ms, launches, units) of one kernel since profiling was enabled."""
        ms, n, u = c_double(), ctypes.c_int64(), c_double()
        C.check(self.lib.inla_profile_read(self.handle, int(kernel), byref(ms), byref(n), byref(u)))
        return ms.value, n.value, u.value

    def eval(self, theta, grad="none", prior="kronecker", want_mode=False, want_marg_var=False, max_newton=50,
             newton_tol=1e-8, fd_eps=1e-3, stream=None, out=None, precision="fp64", use_graph=False):
        """Evaluate a batch on the GPU.  theta: CUDA float64 tensor [B, 4].

        Returns a dict of CUDA tensors: f [B], grad [B, 4] (if requested),
        x_mode [B, n], marg_var [B, n], status [B] (int32), newton_iters [B].
        Work is enqueued on ``stream`` (default: torch's current stream).
        """
        import torch
        if not (isinstance(theta, torch.Tensor) and theta.is_cuda and theta.dtype == torch.float64):
            raise TypeError("theta must be a CUDA float64 tensor")
        theta = theta.contiguous()
        B = theta.shape[0]
        if theta.dim() != 2 or theta.shape[1] != 4:
            raise ValueError("theta must have shape [B, 4]")
        dev = theta.device
        if out is None:
            out = dict(f=torch.empty(B, dtype=torch.float64, device=dev),
                       status=torch.empty(B, dtype=torch.int32, device=dev),
                       newton_iters=torch.empty(B, dtype=torch.int32, device=dev))
            if grad != "none":
                out["grad"] = torch.empty(B, 4, dtype=torch.float64, device=dev)
            if want_mode:
                out["x_mode"] = torch.empty(B, self.n, dtype=torch.float64, device=dev)
            if want_marg_var:
                out["marg_var"] = torch.empty(B, self.n, dtype=torch.float64, device=dev)
        o = make_opts(grad, prior, want_mode, want_marg_var, max_newton, newton_tol, fd_eps, precision, use_graph)
        so = C.inla_eval_out()
        so.f_dev = out["f"].data_ptr()
        so.status_dev = out["status"].data_ptr()
        so.newton_iters_dev = out["newton_iters"].data_ptr()
        so.grad_dev = out["grad"].data_ptr() if "grad" in out else None
        so.x_mode_dev = out["x_mode"].data_ptr() if "x_mode" in out else None
        so.marg_var_dev = out["marg_var"].data_ptr() if "marg_var" in out else None
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        C.check(self.lib.inla_eval_batch(self.handle, int(B), c_void_p(theta.data_ptr()), byref(o), byref(so),
                                         c_void_p(stream.cuda_stream)))
        return out

    def eval_static(self, theta, grad="none", prior="kronecker", want_mode=False, want_marg_var=False,
                    max_newton=50, newton_tol=1e-8, fd_eps=1e-3, stream=None, out=None, precision="fp64"):
        """Same as eval() through inla_eval_batch_static: the library's fixed
        device array serves as the workspace, so the call allocates no device
        memory.  Pass ``out`` (the dict eval() returns) to reuse output tensors;
        otherwise they are allocated here, by torch."""
        import torch
        theta = theta.contiguous()
        B = theta.shape[0]
        dev = theta.device
        if out is None:
            out = dict(f=torch.empty(B, dtype=torch.float64, device=dev),
                       status=torch.empty(B, dtype=torch.int32, device=dev),
                       newton_iters=torch.empty(B, dtype=torch.int32, device=dev))
            if grad != "none":
                out["grad"] = torch.empty(B, 4, dtype=torch.float64, device=dev)
            if want_mode:
                out["x_mode"] = torch.empty(B, self.n, dtype=torch.float64, device=dev)
            if want_marg_var:
                out["marg_var"] = torch.empty(B, self.n, dtype=torch.float64, device=dev)
        o = make_opts(grad, prior, want_mode, want_marg_var, max_newton, newton_tol, fd_eps, precision)
        so = C.inla_eval_out()
        so.f_dev = out["f"].data_ptr()
        so.status_dev = out["status"].data_ptr()
        so.newton_iters_dev = out["newton_iters"].data_ptr()
        so.grad_dev = out["grad"].data_ptr() if "grad" in out else None
        so.x_mode_dev = out["x_mode"].data_ptr() if "x_mode" in out else None
        so.marg_var_dev = out["marg_var"].data_ptr() if "marg_var" in out else None
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        C.check(self.lib.inla_eval_batch_static(self.handle, int(B), c_void_p(theta.data_ptr()), byref(o),
                                                byref(so), c_void_p(stream.cuda_stream)))
        return out

    def eval_host(self, theta, grad="none", prior="kronecker", want_mode=False, want_marg_var=False,
                  max_newton=50, newton_tol=1e-8, fd_eps=1e-3, precision="fp64", use_graph=False):
        """Evaluate with HOST numpy buffers (copies in and out inside the call)."""
        theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 4))
        B = theta.shape[0]
        res = dict(f=np.empty(B), status=np.empty(B, np.int32), newton_iters=np.empty(B, np.int32))
        if grad != "none":
            res["grad"] = np.empty((B, 4))
        if want_mode:
            res["x_mode"] = np.empty((B, self.n))
        if want_marg_var:
            res["marg_var"] = np.empty((B, self.n))
        o = make_opts(grad, prior, want_mode, want_marg_var, max_newton, newton_tol, fd_eps, precision, use_graph)
        so = C.inla_eval_out_host()
        so.f = res["f"].ctypes.data
        so.status = res["status"].ctypes.data
        so.newton_iters = res["newton_iters"].ctypes.data
        so.grad = res["grad"].ctypes.data if "grad" in res else None
        so.x_mode = res["x_mode"].ctypes.data if "x_mode" in res else None
        so.marg_var = res["marg_var"].ctypes.data if "marg_var" in res else None
        C.check(self.lib.inla_eval_batch_host(self.handle, int(B), theta.ctypes.data, byref(o), byref(so)))
        return res


def _probe_check(code):
    if code != C.INLA_OK:
        raise C.InlaError(code, C.load_probe().inla_probe_last_error().decode())


def measure_fp64_peak(device=0, tensor=False):
    """Measured FP64 throughput (TFLOP/s) of scalar FMA or the DMMA instruction
    (libinla_probe.so, a benchmark utility)."""
    lib = C.load_probe()
    v = c_double()
    _probe_check(lib.inla_measure_fp64_peak(int(device), int(bool(tensor)), byref(v)))
    return v.value


def measure_fp32_peak(device=0):
    """Measured FP32 scalar FMA throughput (TFLOP/s) (libinla_probe.so)."""
    lib = C.load_probe()
    v = c_double()
    _probe_check(lib.inla_measure_fp32_peak(int(device), byref(v)))
    return v.value


class SynthModel:
    """A synthetic workload built by the library's C generator (inla_synth_build):
    the model arrays as numpy copies, with the attributes Model() reads."""

    def __init__(self, desc, theta_true, name):
        n_s, m = desc.n_s, desc.m
        nnz_g = None
        self.name = name
        self.n_t, self.n_b, self.m = desc.n_t, desc.n_b, m
        self.nx = int(round(n_s ** 0.5))
        self.lik = {C.INLA_LIK_GAUSSIAN: "gaussian", C.INLA_LIK_POISSON: "poisson",
                    C.INLA_LIK_BINOMIAL: "binomial"}[desc.lik]
        self.tau_b = desc.tau_b
        arr = np.ctypeslib.as_array
        self.C_diag = arr(desc.C_diag, (n_s,)).copy()
        self.G_rowptr = arr(desc.G_rowptr, (n_s + 1,)).copy()
        nnz_g = int(self.G_rowptr[-1])
        self.G_col = arr(desc.G_col, (nnz_g,)).copy()
        self.G_val = arr(desc.G_val, (nnz_g,)).copy()
        self.A_rowptr = arr(desc.A_rowptr, (m + 1,)).copy()
        nnz_a = int(self.A_rowptr[-1])
        self.A_col = arr(desc.A_col, (nnz_a,)).copy()
        self.A_val = arr(desc.A_val, (nnz_a,)).copy()
        self.y = arr(desc.y, (m,)).copy()
        self.E = arr(desc.E, (m,)).copy() if desc.E else None
        self.prior_mean = np.array(desc.prior_mean[:])
        self.prior_sd = np.array(desc.prior_sd[:])
        self.theta_true = np.asarray(theta_true, dtype=float)

    @property
    def n_s(self):
        return self.nx * self.nx

    @property
    def n(self):
        return self.n_t * self.n_s + self.n_b


def synth_build(n_t, nx, n_b, m, lik="gaussian", seed=0, theta_true=None):
    """Build a synthetic workload with the library's C generator (host code)."""
    lib = C.load()
    desc = C.inla_model_desc()
    owner = c_void_p()
    liki = {"gaussian": C.INLA_LIK_GAUSSIAN, "poisson": C.INLA_LIK_POISSON, "binomial": C.INLA_LIK_BINOMIAL}[lik]
    if theta_true is None:
        theta_true = [1.0, -1.0, 0.0, 1.5] if lik == "gaussian" else [float(np.log(1e-3)), -1.0, 0.0, 1.5]
    th = (ctypes.c_double * 4)(*theta_true)
    C.check(lib.inla_synth_build(int(n_t), int(nx), int(n_b), int(m), liki, int(seed),
                                 ctypes.cast(th, c_void_p), byref(desc), byref(owner)))
    try:
        return SynthModel(desc, theta_true, f"synthetic n_t={n_t} {nx}x{nx} n_b={n_b} m={m} {lik}")
    finally:
        lib.inla_synth_free(owner)


def gemm_tf32x3(X, Y, stream=None):
    """C[b] = X[b] @ Y[b].T on the tensor cores (3xTF32 split product) for CUDA
    float32 tensors X, Y of shape [batch, n, n] (or [n, n]), n a multiple of 128.
    Returns (C, status) with status [batch] int32 (0, or ERR_TIMEOUT)."""
    import torch
    lib = C.load()
    squeeze = X.dim() == 2
    X = (X[None] if squeeze else X).contiguous()
    Y = (Y[None] if squeeze else Y).contiguous()
    if X.dtype != torch.float32 or Y.dtype != torch.float32 or not X.is_cuda or X.shape != Y.shape:
        raise TypeError("X and Y must be CUDA float32 tensors of the same shape")
    batch, n = X.shape[0], X.shape[1]
    Cm = torch.empty_like(X)
    status = torch.empty(batch, dtype=torch.int32, device=X.device)
    if stream is None:
        stream = torch.cuda.current_stream(X.device)
    C.check(lib.inla_gemm_tf32x3(int(n), int(batch), c_void_p(X.data_ptr()), c_void_p(Y.data_ptr()),
                                 c_void_p(Cm.data_ptr()), c_void_p(status.data_ptr()), c_void_p(stream.cuda_stream)))
    return (Cm[0] if squeeze else Cm), status


def gemm_f64(X, Y, stream=None):
    """C[b] = X[b] @ Y[b].T in FP64 on the BF16 tensor cores (error-free digit
    splitting) for CUDA float64 tensors of shape [batch, n, n] (or [n, n]), n a
    multiple of 128.  Returns (C, status) with status [batch] int32."""
    import torch
    lib = C.load()
    squeeze = X.dim() == 2
    X = (X[None] if squeeze else X).contiguous()
    Y = (Y[None] if squeeze else Y).contiguous()
    if X.dtype != torch.float64 or Y.dtype != torch.float64 or not X.is_cuda or X.shape != Y.shape:
        raise TypeError("X and Y must be CUDA float64 tensors of the same shape")
    batch, n = X.shape[0], X.shape[1]
    Cm = torch.empty_like(X)
    status = torch.empty(batch, dtype=torch.int32, device=X.device)
    nbytes = int(lib.inla_gemm_f64_workspace_bytes(int(n), int(batch)))
    work = torch.empty(nbytes + 256, dtype=torch.uint8, device=X.device)
    wptr = (work.data_ptr() + 255) // 256 * 256
    if stream is None:
        stream = torch.cuda.current_stream(X.device)
    C.check(lib.inla_gemm_f64(int(n), int(batch), c_void_p(X.data_ptr()), c_void_p(Y.data_ptr()),
                              c_void_p(Cm.data_ptr()), c_void_p(wptr), nbytes, c_void_p(status.data_ptr()),
                              c_void_p(stream.cuda_stream)))
    return (Cm[0] if squeeze else Cm), status


def _make_function():
    import torch

    class LogPosterior(torch.autograd.Function):
        """f(theta) = -log pi~(theta|y) for a batch; backward uses the adjoint gradient."""

        @staticmethod
        def forward(ctx, theta, model, prior="kronecker"):
            need = ctx.needs_input_grad[0]
            r = model.eval(theta.detach().contiguous(), grad="adjoint" if need else "none", prior=prior)
            if need:
                ctx.save_for_backward(r["grad"])
            ctx.mark_non_differentiable(r["status"])
            return r["f"]

        @staticmethod
        def backward(ctx, gf):
            (g,) = ctx.saved_tensors
            return gf[:, None] * g, None, None

    return LogPosterior


_LP = None


def log_posterior(theta, model, prior="kronecker"):
    """Differentiable f(theta) for a [B, 4] CUDA float64 tensor."""
    global _LP
    if _LP is None:
        _LP = _make_function()
    return _LP.apply(theta, model, prior)
