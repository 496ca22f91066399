#!/usr/bin/env python
"""Benchmark: batched f(theta) + grad f evaluations per second on GB300.

Workload (default): the spatio-temporal SPDE x AR(1) model with n_t = 50,
32 x 32 grid (n_s = 1024), n_b = 4, m = 100 000 Gaussian observations.  One
step is one ``inla_eval_batch`` call evaluating the 2d + 1 = 9 points of the
central-difference stencil (Eq. central_diff) in one batch in FP64, which
yields one f + grad f evaluation.  Inputs (the model and its ~4 GB of
factor storage) stay resident in HBM; the working set is far larger than
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead (a bounded sample per step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "theta-evals/s (f+grad f)"
PROFILE_EVERY = 8   # event-time every 8th launch of the instrumented kernels (keeps the overhead small)
UNIT = "f+grad evaluations/s"
CONFIG_WORKLOAD = {
    1: "st-spde-ar1 n_t=8 grid=8x8 (n_s=64) n_b=2 m=2000 gaussian; one step = 9-point "
       "central-difference stencil in one FP64 launch",
    2: "st-spde-ar1 n_t=50 grid=32x32 (n_s=1024) n_b=4 m=100000 gaussian; one step = 9-point "
       "central-difference stencil in one FP64 launch",
    3: "st-spde-ar1 n_t=100 grid=45x45 (n_s=2025) n_b=6 m=400000 gaussian; one step = 16 line-search "
       "points with adjoint gradients, FP64",
    4: "st-spde-ar1 n_t=200 grid=50x50 (n_s=2500) n_b=6 m=1000000 gaussian; one step = 9 stencil "
       "points with adjoint gradients, mixed precision",
    5: "st-spde-ar1 n_t=100 grid=64x64 (n_s=4096) n_b=8 m=500000 poisson; one step = 25-point CCD "
       "design with Newton modes and adjoint gradients, mixed precision",
}
# natural gradient mode and precision of each workload
MODES = {1: ("fd", "fp64"), 2: ("fd", "fp64"), 3: ("adjoint", "fp64"), 4: ("adjoint", "mixed"),
         5: ("adjoint", "mixed")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grad", default=None, choices=["fd", "adjoint"],
                    help="fd: one f+grad from the 9-point stencil per step; adjoint: every point of the "
                         "workload's batch gets f and an adjoint gradient (default: the workload's own)")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"])
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel of a step from the host (default: replay the step as one captured CUDA "
                         "graph, the library's use_graph option)")
    ap.add_argument("--gemm", default=None, choices=["cuda-core", "tensor"],
                    help="FP32 selected-inversion GEMM: 128x128 FP32 FMA tiles or tcgen05 3xTF32")
    ap.add_argument("--sweep", default=None, choices=["cuda-core", "tensor", "blocked"],
                    help="FP32 Schur-block inversion: the sweep with FP32 FMA tile updates, the sweep with tcgen05 "
                         "3xTF32 updates, or the blocked recursion with 3xTF32 products (the library picks by size)")
    ap.add_argument("--time-parts", type=int, default=2, choices=[1, 2],
                    help="2 (the library default): the time chain split at its middle block into two "
                         "independent elimination chains; 1: one chain")
    ap.add_argument("--point-groups", type=int, default=None, choices=[1, 2],
                    help="the library's point groups (default: the library's own setting)")
    ap.add_argument("--nt", type=int, default=None, help="override n_t (profiling case only)")
    ap.add_argument("--centres", type=int, default=1,
                    help="stencil centres per step (FD mode) / copies of the batch (adjoint mode); profiling only")
    ap.add_argument("--theta-iter", action="store_true",
                    help="time theta-iterations (gradient + 16-point line search) in the FD/FP64 form and "
                         "the adjoint/mixed form on the same workload, and run BFGS to the mode with both")
    ap.add_argument("--no-errors", action="store_true", help="skip the accuracy checks against the oracle")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the extra legs (mode + variances, adjoint FP64 / mixed, theta-iterations)")
    ap.add_argument("--no-bfgs", action="store_true", help="with --theta-iter: skip the runs to the mode")
    ap.add_argument("--bfgs-iters", type=int, default=30, help="with --theta-iter: BFGS iteration limit")
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle timing
#
# The oracle (numpy/scipy FP64, test infrastructure) timed on the host cores as
# a reported baseline: one theta per worker process with single-threaded BLAS,
# the paper's level-1 parallelism over the stencil points (Sec. 3.1).  The
# pool uses the spawn start method (no fork after CUDA initialisation).

_WORKER = {}
BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_init(cfg, threads):
    for v in BLAS_ENV:
        os.environ[v] = str(threads)
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from synth import config_model
    _WORKER["mdl"] = config_model(cfg)


def _oracle_eval(args):
    import numpy as np
    from oracle import bta
    theta, want = args
    t0 = time.perf_counter()
    r = bta.evaluate(_WORKER["mdl"], np.asarray(theta, dtype=float), want_grad=want, want_var=want)
    out = {"f": r["f"], "seconds": time.perf_counter() - t0}
    if want:
        out.update(grad=r["grad"].tolist(), x=r["x"], var=r["var"])
    return out


def cpu_model_name():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """Worker processes holding the workload's model, one theta per task."""

    def __init__(self, cfg, workers, threads=1):
        import multiprocessing as mp
        self.workers, self.threads = workers, threads
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(cfg, threads))

    def map(self, thetas, want=False):
        return self.pool.map(_oracle_eval, [(list(map(float, t)), want) for t in thetas], chunksize=1)

    def close(self):
        self.pool.terminate()
        self.pool.join()


def oracle_stencil_step(pool, centre):
    """One f + grad f by central differences on the oracle: the 9 stencil points
    in parallel (one per worker).  Returns (seconds, f values, oracle FD gradient)."""
    import numpy as np
    from synth import fd_stencil
    pts = fd_stencil(np.asarray(centre))
    t0 = time.perf_counter()
    res = pool.map(pts)
    sec = time.perf_counter() - t0
    f = np.array([r["f"] for r in res])
    g = np.array([(f[1 + 2 * j] - f[2 + 2 * j]) / (pts[1 + 2 * j][j] - pts[2 + 2 * j][j]) for j in range(4)])
    return sec, f, g


def one_core_f(cfg, centre):
    """Seconds for one oracle f on one core (one worker, single-threaded BLAS)."""
    pool = OraclePool(cfg, 1, 1)
    try:
        pool.map([centre])                      # warm-up: imports and model in the worker
        return pool.map([centre])[0]["seconds"]
    finally:
        pool.close()


def cpu_baseline(cfg, centre):
    """The oracle on the host cores: the workload's 9-point stencil with one theta
    per single-threaded worker (timed in full, one step), and one f on one core."""
    nproc = os.cpu_count() or 1
    workers = min(9, nproc)
    pool = OraclePool(cfg, workers, 1)
    try:
        pool.map([centre] * workers)            # warm-up: imports and model in every worker
        sec, f, g = oracle_stencil_step(pool, centre)
    finally:
        pool.close()
    sec1 = one_core_f(cfg, centre)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"one full step: the 9-point central-difference stencil, one theta per worker process "
                      f"({workers} workers, single-threaded numpy/scipy BLAS each), {sec:.2f} s",
            "nproc": nproc, "cpu_model": cpu_model_name(),
            "one_core": {"seconds_per_f": sec1, "value": 1.0 / (9 * sec1), "unit": UNIT,
                         "sample": "one oracle f on one core, 9 f per f + grad f"}}, f, g


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ reference arm (the CPU oracle)

def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, on this arm's workload: each
    step is the full 9-point central-difference stencil (one f + grad f), one
    theta per single-threaded worker process.  Warm-up steps start the workers
    and build the model in each (the oracle has no other warm-up state)."""
    if rank != 0:
        return
    cfg = args.config
    from synth import config_model, theta_batch
    if args.grad != "fd":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the central-difference "
                          "form of the workload; run it with --grad fd"}))
        return
    mdl = config_model(cfg)
    centre = theta_batch(cfg, mdl)[0]
    nproc = os.cpu_count() or 1
    workers = min(9, nproc)
    pool = OraclePool(cfg, workers, 1)
    try:
        for _ in range(args.warmup):
            pool.map([centre] * workers)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle_stencil_step(pool, centre)
        elapsed = time.perf_counter() - t0
    finally:
        pool.close()
    value = args.steps / elapsed
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(cfg, world, args.grad, args.precision,
                                  l2=L2_NOTE_FLUSH if cfg in SMALL_WORKSPACE_CONFIGS else L2_NOTE_LARGE),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"every step: the full 9-point stencil, one theta per worker process "
                                       f"({workers} workers, single-threaded BLAS each); warm-up steps start the "
                                       f"workers and build the model in each",
                             "nproc": nproc, "cpu_model": cpu_model_name()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


L2_BYTES = 129 * 2 ** 20
SMALL_WORKSPACE_CONFIGS = (1,)   # workloads whose GPU workspace is below twice the L2 (timed after a flush)
L2_NOTE_LARGE = "working set (GBs of factor storage per step) exceeds L2; no flush"
L2_NOTE_FLUSH = "working set below 2x L2: a 512 MiB buffer is rewritten before each timed step (outside its events)"


def block_cholesky_rate(mdl, points, step_s, peak_dmma):
    """The step as a block-Cholesky rate: the textbook BTA Cholesky's flops (per point and
    time step 7/3 n_s^3 for POTRF, TRSM and SYRK of the n_s x n_s blocks) over the whole step
    time, which also holds the mode solve and the rest of f: a lower bound on the
    factorisation's own rate.  The library inverts its Schur blocks instead (n_p^3 flops per
    time step), so this counts the work a Cholesky-based implementation would do."""
    flops = points * mdl.n_t * (7.0 / 3.0) * float(mdl.n_s) ** 3
    rate = flops / step_s / 1e12
    return {"textbook_equivalent": rate, "vs_fp64_dmma_peak": rate / peak_dmma if peak_dmma else None,
            "definition": "points x n_t x 7/3 n_s^3 flops per step / step time (the whole step)"}


def config_dict(cfg, world, grad=None, precision=None, points=9, l2=L2_NOTE_LARGE):
    from synth import CONFIGS
    c = CONFIGS[cfg]
    grad = grad or MODES[cfg][0]
    precision = precision or MODES[cfg][1]
    return {"workload": CONFIG_WORKLOAD[cfg], "n_t": c["n_t"], "n_s": c["nx"] ** 2, "n_b": c["n_b"], "m": c["m"],
            "theta_points_per_step": points,
            "grad": "central differences (9 points per centre)" if grad == "fd" else "adjoint",
            "precision": precision, "prior_logdet": "kronecker",
            "likelihood": c["lik"], "parallelism": f"theta-replicas x{world}",
            "l2": l2}


def measured_peaks_json():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ mixed-precision accuracy

def mixed_errors(model, theta, grad):
    """Relative errors of the mixed path against the FP64 path at the given points:
    f (|df| / |f|), the gradient (max |dg| / max |g|), the mode (max |dx| / max |x|)
    and the marginal variances (max |dv| / v)."""
    import numpy as np
    r = {}
    for prec in ("fp64", "mixed"):
        o = model.eval(theta, grad=grad, precision=prec, want_mode=True, want_marg_var=True)
        r[prec] = {k: o[k].cpu().numpy() for k in ("f", "grad", "x_mode", "marg_var", "status")}
    a, b = r["fp64"], r["mixed"]
    if np.any(a["status"] != 0) or np.any(b["status"] != 0):
        return {"error": "evaluation failed"}
    return {"points": int(theta.shape[0]),
            "f_rel": float(np.max(np.abs(b["f"] - a["f"]) / np.abs(a["f"]))),
            "grad_rel": float(np.max(np.abs(b["grad"] - a["grad"])) / np.max(np.abs(a["grad"]))),
            "x_rel": float(np.max(np.abs(b["x_mode"] - a["x_mode"])) / np.max(np.abs(a["x_mode"]))),
            "var_rel": float(np.max(np.abs(b["marg_var"] - a["marg_var"]) / a["marg_var"]))}


# ------------------------------------------------------------------ theta-iterations

def theta_iterations(args, local):
    """One theta-iteration = the gradient at the current point plus one parallel
    line search of 16 f-only points (Sec. 3.2).  FD form: the 9-point central-
    difference stencil in FP64; adjoint form: one f + adjoint gradient.  Both
    line searches are one batch each, in the form's precision."""
    import numpy as np
    import torch
    import paper_2204_04678_gb300 as pkg
    from paper_2204_04678_gb300 import capi, driver
    from synth import config_model, line_points, theta_batch

    pkg.build()
    capi.load()
    cfg = args.config
    mdl = config_model(cfg)
    model = pkg.Model(mdl, device=local)
    model.set_time_partition(args.time_parts)
    stream = torch.cuda.current_stream()
    centre = theta_batch(2, mdl)[0]          # theta_true + 0.1 N(0, I), the stencil centre of the workloads
    ref = model.eval(torch.tensor(centre[None], dtype=torch.float64, device="cuda"), grad="adjoint")
    g64 = ref["grad"][0].cpu().numpy()
    pts = line_points(centre, -g64, 0.5)
    c_t = torch.tensor(centre[None], dtype=torch.float64, device="cuda")
    l_t = torch.tensor(pts, dtype=torch.float64, device="cuda")
    forms = {"fd_fp64": ("fd", "fp64"), "adjoint_fp64": ("adjoint", "fp64"), "adjoint_mixed": ("adjoint", "mixed")}
    res = {}
    clocks = Clocks(local)
    for name, (grad, prec) in forms.items():
        def iteration():
            a = model.eval(c_t, grad=grad, precision=prec)
            n = model.last_launch_count()
            b = model.eval(l_t, grad="none", precision=prec)
            return a, b, n + model.last_launch_count()
        for _ in range(max(args.warmup, 1)):
            a, b, _ = iteration()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        e0.record(stream)
        for _ in range(args.steps):
            a, b, nl = iteration()
            launches += nl
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / args.steps
        assert int(a["status"].abs().sum()) + int(b["status"].abs().sum()) == 0, name
        res[name] = {"theta_iterations_per_s": 1.0 / sec, "ms_per_iteration": 1e3 * sec,
                     "f": np.concatenate([a["f"].cpu().numpy(), b["f"].cpu().numpy()]),
                     "grad": a["grad"][0].cpu().numpy(), "gpu_launches_per_iteration": launches / args.steps}
    clk = clocks.stop()
    base = res["adjoint_fp64"]
    for name, r in res.items():
        r["max_rel_err_f_vs_fp64"] = float(np.max(np.abs(r["f"] - base["f"]) / np.abs(base["f"])))
        r["max_rel_err_grad_vs_fp64_adjoint"] = float(np.max(np.abs(r["grad"] - base["grad"]))
                                                      / np.max(np.abs(base["grad"])))
    for r in res.values():
        del r["f"], r["grad"]
    # BFGS to the mode with each form (host driver over the same batched calls)
    to_mode = {}
    if not args.no_bfgs:
        for name, (grad, prec) in forms.items():
            fg, fb, _, _ = driver.model_evaluators(model, grad=grad, precision=prec)
            t0 = time.perf_counter()
            r = driver.bfgs(fg, fb, centre, max_iter=args.bfgs_iters, gtol=1e-2, ftol=1e-10)
            sec = time.perf_counter() - t0
            f64 = model.eval(torch.tensor(r["theta"][None], dtype=torch.float64, device="cuda"), grad="adjoint")
            to_mode[name] = {"iterations": r["iterations"], "seconds": sec, "theta": r["theta"].tolist(),
                             "f_fp64_at_end": float(f64["f"][0]),
                             "max_abs_grad_fp64_at_end": float(f64["grad"][0].abs().max())}
    fast, slow = res["adjoint_mixed"], res["fd_fp64"]
    line = {"metric": "theta-iterations/s (gradient + 16-point line search)",
            "value": fast["theta_iterations_per_s"], "unit": "theta-iterations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fast["ms_per_iteration"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": dict(config_dict(cfg, 1, "adjoint", "mixed", 17),
                                                workload=CONFIG_WORKLOAD[cfg].split(";")[0]
                                                + "; one step = gradient at the centre + 16 line-search points"),
            "clocks": clk, "forms": res, "speedup_adjoint_mixed_over_fd_fp64":
                fast["theta_iterations_per_s"] / slow["theta_iterations_per_s"],
            "bfgs_to_mode": to_mode}
    print(json.dumps(line))
    model.close()


# ------------------------------------------------------------------ our arm

def timed_calls(model, theta, kw, steps, stream, flush=None):
    """Device seconds of `steps` evaluations (CUDA events on the launch stream)
    and the kernel launches they issued.  With `flush` (a buffer larger than L2)
    each call is timed alone after the buffer has been rewritten."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches, elapsed = 0, 0.0
    if flush is not None:
        for _ in range(steps):
            flush.fill_(1)
            e0.record(stream)
            model.eval(theta, **kw)
            e1.record(stream)
            launches += model.last_launch_count()
            torch.cuda.synchronize()
            elapsed += e0.elapsed_time(e1) / 1e3
        return elapsed, launches
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        model.eval(theta, **kw)
        launches += model.last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, launches


def rel_errors(f, ref_f, grad=None, ref_grad=None, x=None, ref_x=None, v=None, ref_v=None):
    """The parity metrics: |df| / |f|, max |dg| / max(1, |g|), ||dx||_inf / ||x||_inf, max |dv| / v."""
    import numpy as np
    e = {"f_rel": float(abs(f - ref_f) / abs(ref_f))}
    if grad is not None:
        e["grad_rel"] = float(np.max(np.abs(grad - ref_grad)) / max(1.0, np.max(np.abs(ref_grad))))
    if x is not None:
        e["x_rel"] = float(np.max(np.abs(x - ref_x)) / np.max(np.abs(ref_x)))
    if v is not None:
        e["var_rel"] = float(np.max(np.abs(v - ref_v) / ref_v))
    return e


def extra_forms(model, centre, stream, steps, dist_world):
    """The workload's other forms, timed on the same model (each after one untimed
    call): FD with the mode and the marginal variances (selected inversion at the
    centre); the 9 stencil points each with an adjoint gradient in FP64 and in
    mixed precision; and theta-iterations (gradient at the centre + one 16-point
    line-search batch, Sec. 3.2) in the FD/FP64 and the adjoint/mixed forms."""
    import numpy as np
    import torch
    from synth import fd_stencil, line_points
    cen = torch.tensor(centre[None], dtype=torch.float64, device="cuda")
    st9 = torch.tensor(fd_stencil(centre), dtype=torch.float64, device="cuda")
    forms, outs = {}, {}
    legs = {"fd_fp64_mode_var": (cen, 1, dict(grad="fd", want_mode=True, want_marg_var=True)),
            "adjoint_fp64": (st9, 9, dict(grad="adjoint")),
            "adjoint_mixed": (st9, 9, dict(grad="adjoint", precision="mixed"))}
    for name, (th, per, kw) in legs.items():
        outs[name] = model.eval(th, **kw)
        sec, nl = timed_calls(model, th, kw, steps, stream)
        assert int(outs[name]["status"].abs().sum()) == 0, name
        forms[name] = {"value": per * steps / sec, "unit": UNIT, "ms_per_step": 1e3 * sec / steps,
                       "f_grad_per_step": per, "gpu_launches_per_step": nl / steps}
    outs["mixed_centre"] = model.eval(cen, grad="adjoint", want_mode=True, want_marg_var=True, precision="mixed")
    g = outs["adjoint_fp64"]["grad"][0].cpu().numpy()
    lsp = torch.tensor(line_points(centre, -g, 0.5), dtype=torch.float64, device="cuda")
    its = {}
    for name, (gk, prec) in {"fd_fp64": ("fd", "fp64"), "adjoint_mixed": ("adjoint", "mixed")}.items():
        kw_g = dict(grad=gk, precision=prec)
        kw_l = dict(grad="none", precision=prec)
        model.eval(cen, **kw_g)
        model.eval(lsp, **kw_l)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            model.eval(cen, **kw_g)
            model.eval(lsp, **kw_l)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / steps
        its[name] = {"theta_iterations_per_s": 1.0 / sec, "ms_per_iteration": 1e3 * sec}
    forms["theta_iterations"] = dict(its, speedup_adjoint_mixed_over_fd_fp64=its["adjoint_mixed"][
        "theta_iterations_per_s"] / its["fd_fp64"]["theta_iterations_per_s"],
        definition="gradient at the stencil centre + one 16-point line-search batch (f only), each form in "
                   "its own precision")
    # the FD step replayed as one captured CUDA graph (the whole call, every kernel), against eager launches
    kw = dict(grad="fd")
    model.eval(cen, use_graph=True, **kw)
    sec_g, _ = timed_calls(model, cen, dict(kw, use_graph=True), steps, stream)
    sec_e, nl = timed_calls(model, cen, kw, steps, stream)
    forms["fd_fp64_graph"] = {"value": steps / sec_g, "unit": UNIT, "ms_per_step": 1e3 * sec_g / steps,
                              "eager_ms_per_step": 1e3 * sec_e / steps, "gpu_launches_per_step": nl / steps}
    forms["config1_fd_fp64"] = small_workload_leg(steps)
    return forms, outs


def small_workload_leg(steps):
    """The 8 x 8 x 8 workload (n = 514): one FD step per call, where launch latency, not
    arithmetic, sets the time; eager launches and one graph launch, each step timed alone
    after a 512 MiB rewrite (the workspace fits in L2)."""
    import torch
    import paper_2204_04678_gb300 as pkg
    from synth import config_model, theta_batch
    mdl = config_model(1)
    model = pkg.Model(mdl)
    th = torch.tensor(theta_batch(1, mdl)[:1], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, g in (("eager", False), ("graph", True)):
        for _ in range(2):
            model.eval(th, grad="fd", use_graph=g)
        sec, nl = timed_calls(model, th, dict(grad="fd", use_graph=g), max(steps, 5), stream, flush)
        out[name] = {"ms_per_step": 1e3 * sec / max(steps, 5), "value": max(steps, 5) / sec,
                     "gpu_launches_per_step": nl / max(steps, 5)}
    model.close()
    return dict(out, unit=UNIT, workload=CONFIG_WORKLOAD[1])


def main():
    args = parse()
    if args.grad is None:
        args.grad = MODES[args.config][0]
    if args.precision is None:
        args.precision = MODES[args.config][1]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.theta_iter:
        import torch
        torch.cuda.set_device(local)
        theta_iterations(args, local)
        return

    import numpy as np
    import torch
    import paper_2204_04678_gb300 as pkg
    from paper_2204_04678_gb300 import capi
    from synth import config_model, theta_batch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        pkg.build()
    if dist:
        dist.barrier()
    capi.load()

    cfg = args.config
    peak_fp64 = pkg.measure_fp64_peak(local, tensor=False)
    peak_dmma = pkg.measure_fp64_peak(local, tensor=True)
    peak_fp32 = pkg.measure_fp32_peak(local)
    if args.nt:
        from synth import CONFIGS, build
        mdl = build(**dict(CONFIGS[cfg], n_t=args.nt, name="profiling case"))
    else:
        mdl = config_model(cfg)
    centre = theta_batch(cfg, mdl)[0] + 0.01 * rank
    model = pkg.Model(mdl, device=local)
    model.set_time_partition(args.time_parts)
    if args.point_groups:
        model.set_point_groups(args.point_groups)
    n_p = -(-mdl.n_s // 64) * 64
    tensor_sweep = n_p % 128 == 0 and args.sweep == "tensor"
    # the FP32 block inversion the model runs (the library default when no --sweep is given)
    inv_mode = args.sweep or ("blocked" if n_p % 128 == 0 and n_p >= 2048 else "cuda-core")
    inv_label = {"tensor": "block sweep, rank-64 updates on the tensor cores (tcgen05 3xTF32)",
                 "blocked": "2x2 block recursion, products on the tensor cores (tcgen05 3xTF32), "
                            "256-row base blocks swept on the CUDA cores",
                 "cuda-core": "block sweep on the CUDA cores"}[inv_mode]
    fp64_label = ("2x2 block recursion, products on the BF16 tensor cores through 8 digit slices of 7 bits "
                  "(tcgen05), 256-row base blocks swept on the CUDA cores" if n_p % 128 == 0 and n_p > 256
                  else "block sweep on the CUDA cores")
    if args.gemm or args.sweep:
        sw = {"tensor": capi.INLA_SWEEP_TF32X3, "blocked": capi.INLA_INV_BLOCKED}.get(args.sweep, 64)
        if args.sweep is None:
            sw = capi.INLA_INV_BLOCKED if (n_p % 128 == 0 and n_p >= 2048) else 64
        model.set_tiles(32, sw, capi.INLA_GEMM_TF32X3 if args.gemm != "cuda-core" else 128)
    stream = torch.cuda.current_stream()
    if args.grad == "fd":
        cen = centre[None, :] + 0.01 * np.arange(args.centres)[:, None]
        theta = torch.tensor(cen, dtype=torch.float64, device="cuda")
        per_step = args.centres
        points = 9 * args.centres
    else:
        from synth import fd_stencil
        batch = fd_stencil(centre) if cfg in (1, 2) else theta_batch(cfg, mdl) + 0.01 * rank
        if args.centres > 1:   # profiling case: the batch repeated around shifted centres
            batch = np.concatenate([batch + 0.01 * k for k in range(args.centres)])
        theta = torch.tensor(batch, dtype=torch.float64, device="cuda")
        per_step = theta.shape[0]
        points = per_step
    grad = args.grad
    prec = args.precision
    out = model.eval(theta, grad=grad, precision=prec)
    graph = not args.eager
    kw = dict(grad=grad, out=out, precision=prec, use_graph=graph)
    for _ in range(max(args.warmup, 1)):
        model.eval(theta, **kw)
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0, "evaluation failed"
    # a working set below twice the L2 would stay cache-resident from step to step: then each
    # step is timed alone, after a buffer larger than L2 has been rewritten
    flush = model.workspace_bytes(theta.shape[0], grad=grad, precision=prec) < 2 * L2_BYTES
    scratch = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda") if flush else None

    # ---- the headline: K steps, no instrumentation
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    elapsed, launches = timed_calls(model, theta, kw, args.steps, stream, scratch)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    if dist:
        from paper_2204_04678_gb300.replicas import max_over_ranks
        elapsed = max_over_ranks(elapsed)
    value = world * args.steps * per_step / elapsed

    # ---- roofline of the dominant kernel: a second pass of K steps with every
    # PROFILE_EVERY-th launch of the instrumented kernels bracketed by events
    model.profile_enable(PROFILE_EVERY)
    kwp = dict(kw, use_graph=False)
    elapsed_p, _ = timed_calls(model, theta, kwp, args.steps, stream, scratch)
    fp32 = prec == "mixed"
    tensor_gemm = fp32 and n_p % 128 == 0 and args.gemm != "cuda-core"
    upd_id = capi.KERNEL_GJ_UPDATE32 if fp32 else capi.KERNEL_GJ_UPDATE
    digit_products = (not fp32) and n_p % 128 == 0 and n_p > 128
    # the product slot covers whichever product kernel the path launches
    gemm_name = ("ozaki_gemm_kernel" if digit_products else
                 "gemm_tf32x3_tma_kernel" if tensor_gemm else "gemm_nn_kernel")
    kernels = {"gj_update_kernel": model.profile_read(upd_id), gemm_name: model.profile_read(capi.KERNEL_GEMM)}
    # the sweep's other two launches per pivot, for their event-timed durations
    sweep_aux = {"gj_pivot_kernel": model.profile_read(capi.KERNEL_GJ_PIVOT),
                 "gj_panel_kernel": model.profile_read(capi.KERNEL_GJ_PANEL)}
    model.profile_enable(0)
    flop_per_unit = 2.0 * 64 ** 3
    peaks = measured_peaks_json()
    tf32x3_peak = None
    if peaks.get("bf16_tflops_sustained"):
        # nominal dense TF32 / BF16 = 1.1 / 2.25; three TF32 products per algorithmic product
        tf32x3_peak = peaks["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0
    kname = max(kernels, key=lambda k: kernels[k][0])
    kms, knl, kunits = kernels[kname]
    avg_s = kms / 1e3 / max(knl, 1)
    achieved = kunits / max(knl, 1) * flop_per_unit / avg_s / 1e12 if knl else None
    tf32_source = ("MEASURED_PEAKS.json bf16_tflops_sustained x (1.1 / 2.25) nominal TF32/BF16 ratio / 3 "
                   "TF32 products per 3xTF32 product, of measured")
    bf16_peak = peaks.get("bf16_tflops")
    if kname == "ozaki_gemm_kernel" and bf16_peak:
        # FP64 products through 36 BF16 digit-slice products on the tensor cores: the FP64-equivalent
        # peak is the measured BF16 dense peak / 36
        peak, bound = bf16_peak / 36.0, "tensor"
        peak_source = ("MEASURED_PEAKS.json bf16_tflops (burst, the kernel timed alone) / 36 BF16 digit products "
                       "per FP64 product, of measured")
        desc = ("FP64 products of the blocked inversion on the BF16 tensor cores (tcgen05 kind::f16, 8 digit "
                "slices of 7 bits per entry, 128x64 tiles)")
    elif kname == "gj_update_kernel" and fp32 and tensor_sweep and tf32x3_peak:
        peak, bound, peak_source = tf32x3_peak, "tensor", tf32_source
        desc = ("rank-64 update of the FP32 block sweep on the tensor cores (tcgen05, 3xTF32, 128x128 tiles, "
                "K = 64)")
    elif kname == "gemm_tf32x3_tma_kernel" and tf32x3_peak:
        peak, bound, peak_source = tf32x3_peak, "tensor", tf32_source
        desc = ("128x128 tile 3xTF32 products of the blocked inversion and the selected inversion on the tensor "
                "cores (tcgen05, operands split once and loaded by TMA)")
    else:
        peak, bound = (peak_fp32 if fp32 else peak_fp64), "alu"
        peak_source = ("measured on this GPU: " + ("FP32" if fp32 else "FP64")
                       + " FMA loop over all SMs (libinla_probe.so), of measured")
        desc = (("FP32" if fp32 else "FP64") + (" tile update of the block sweep inversion"
                                                 if kname == "gj_update_kernel" else " tile products"))
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "gj_update_traffic.txt")
    if kname == "gj_update_kernel" and not fp32 and os.path.exists(tfile):
        for line in open(tfile):
            if line.startswith("bytes_per_unit="):
                traffic = float(line.split("=")[1]) * kunits / max(knl, 1)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": f"{kname} ({desc})", "timed_every": PROFILE_EVERY, "peak_source": peak_source,
                "launches_timed": knl, "share_of_step": PROFILE_EVERY * kms / 1e3 / elapsed_p if elapsed_p else None,
                "timed_in": "a second pass of the same steps with event instrumentation (the headline pass has none)"}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        th_host = theta.cpu().numpy().copy()
        model.eval_host(th_host, grad=grad, precision=prec, use_graph=graph)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            model.eval_host(th_host, grad=grad, precision=prec, use_graph=graph)
        e2e_s = (time.perf_counter() - t0) / args.steps
        if dist:
            from paper_2204_04678_gb300.replicas import max_over_ranks
            e2e_s = max_over_ranks(e2e_s)
        nb = th_host.shape[0]
        e2e = {"value": world * per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * nb,
               "d2h_bytes_per_step": nb * (8 + 4 * 8 + 4 + 4)}

    # ---- the workload's other forms (x* and variances, adjoint FP64 / mixed, theta-iterations)
    forms, fouts = None, None
    base_case = cfg in (1, 2) and grad == "fd" and not (args.nt or args.centres != 1)
    if base_case and world == 1 and not args.no_forms:
        forms, fouts = extra_forms(model, centre, stream, 3, world)

    # ---- the oracle on the host cores, and the errors against it at the stencil centre
    cpu, errors = None, None
    if rank == 0 and world == 1 and base_case and not args.no_cpu_baseline:
        try:
            cpu, f_or, g_or = cpu_baseline(cfg, centre)
        except Exception as e:  # reported, not fatal
            cpu, f_or = {"value": None, "error": str(e)[:200]}, None
        if f_or is not None and not args.no_errors:
            errors = {"reference": "oracle/ (FP64 CPU), at the stencil centre; gradients: central differences "
                                   "of oracle f for the FD form, the oracle's adjoint for the adjoint forms"}
            errors["fd_fp64"] = rel_errors(float(out["f"][0]), f_or[0], out["grad"][0].cpu().numpy(), g_or)
            if fouts is not None:
                pool = OraclePool(cfg, 1, os.cpu_count() or 1)
                try:
                    ref = pool.map([centre], want=True)[0]
                finally:
                    pool.close()
                o = fouts["fd_fp64_mode_var"]
                errors["fd_fp64"].update(rel_errors(float(o["f"][0]), ref["f"], x=o["x_mode"][0].cpu().numpy(),
                                                    ref_x=ref["x"], v=o["marg_var"][0].cpu().numpy(),
                                                    ref_v=ref["var"]))
                errors["fd_fp64"].pop("f_rel")
                errors["fd_fp64"]["f_rel"] = rel_errors(float(o["f"][0]), ref["f"])["f_rel"]
                a = fouts["adjoint_fp64"]
                errors["adjoint_fp64"] = rel_errors(float(a["f"][0]), ref["f"], a["grad"][0].cpu().numpy(),
                                                    np.array(ref["grad"]))
                mc = fouts["mixed_centre"]
                errors["adjoint_mixed"] = rel_errors(float(mc["f"][0]), ref["f"], mc["grad"][0].cpu().numpy(),
                                                     np.array(ref["grad"]), mc["x_mode"][0].cpu().numpy(), ref["x"],
                                                     mc["marg_var"][0].cpu().numpy(), ref["var"])
    elif prec == "mixed" and not args.no_errors and world == 1:
        errors = {"vs_fp64_path": mixed_errors(model, theta[:1], grad)}

    line = {}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
                "data": "synthetic",
                "config": config_dict(cfg, world, grad, prec, points, l2=L2_NOTE_FLUSH if flush else L2_NOTE_LARGE),
                "kernel_path": dict({"fp64_inversion": fp64_label} if prec == "fp64" else
                                    {"fp32_inversion": inv_label, "fp32_gemm": "tensor (tcgen05 3xTF32)"
                                     if tensor_gemm else "cuda-core"},
                                    time_chain="split at block n_t/2 into two elimination chains on two streams"
                                    if args.time_parts == 2 and mdl.n_t >= 3 else "one elimination chain"),
                "clocks": clk,
                "gpu_launches": launches,
                "launch_mode": "one captured CUDA graph per step (use_graph)" if graph else "eager launches",
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "f_evals_per_s": 9 * value if grad == "fd" else value,
                "grad_mode": grad,
                "errors_vs_oracle": errors,
                "forms": forms,
                "block_cholesky_tflops": block_cholesky_rate(mdl, points, elapsed / args.steps, peak_dmma),
                "measured_peaks_tflops": {"fp64_fma": peak_fp64, "fp64_dmma": peak_dmma, "fp32_fma": peak_fp32,
                                          "tf32x3_tensor_from_bf16_sustained": tf32x3_peak},
                "kernels": dict({k: {"ms_sampled": v[0], "launches_sampled": v[1],
                                     "tflops": v[2] * flop_per_unit / (v[0] / 1e3) / 1e12 if v[0] else None}
                                 for k, v in kernels.items()},
                                **{k: {"ms_sampled": v[0], "launches_sampled": v[1],
                                       "us_per_launch": 1e3 * v[0] / v[1] if v[1] else None}
                                   for k, v in sweep_aux.items()})}
        if args.nt or args.centres != 1:
            line["config"]["workload"] = f"profiling case: n_t={mdl.n_t}, {args.centres} stencil centres per step"
        print(json.dumps(line))
    model.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
