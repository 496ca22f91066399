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
    ap.add_argument("--graph", action="store_true", help="replay each step as a captured CUDA graph")
    ap.add_argument("--gemm", default=None, choices=["cuda-core", "tensor"],
                    help="FP32 selected-inversion GEMM: 128x128 FP32 FMA tiles or tcgen05 3xTF32")
    ap.add_argument("--sweep", default=None, choices=["cuda-core", "tensor"],
                    help="FP32 block-sweep updates: FP32 FMA tiles (the library's default) or tcgen05 3xTF32")
    ap.add_argument("--nt", type=int, default=None, help="override n_t (profiling case only)")
    ap.add_argument("--centres", type=int, default=1,
                    help="stencil centres per step (FD mode) / copies of the batch (adjoint mode); profiling only")
    ap.add_argument("--theta-iter", action="store_true",
                    help="time theta-iterations (gradient + 16-point line search) in the FD/FP64 form and "
                         "the adjoint/mixed form on the same workload, and run BFGS to the mode with both")
    ap.add_argument("--no-errors", action="store_true", help="skip the mixed-vs-FP64 accuracy check")
    ap.add_argument("--no-bfgs", action="store_true", help="with --theta-iter: skip the runs to the mode")
    ap.add_argument("--bfgs-iters", type=int, default=30, help="with --theta-iter: BFGS iteration limit")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--evals", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--nt-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--with-grad", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle timing

def oracle_sample(cfg, evals, nt_sample, with_grad):
    """Time `evals` oracle evaluations at the first point of the workload (child process).

    For the large workloads the model is built with n_t = nt_sample time steps
    (same grid, observations and batch) and the time is scaled by n_t / nt_sample:
    the block algorithms cost the same per time step.
    """
    from oracle import bta
    from synth import CONFIGS, build, theta_batch, config_model
    c = dict(CONFIGS[cfg])
    scale = 1.0
    if nt_sample and nt_sample < c["n_t"]:
        scale = c["n_t"] / nt_sample
        c["n_t"] = nt_sample
    mdl = build(**c)
    th = theta_batch(cfg, config_model(1) if cfg == 1 else mdl)
    t0 = time.perf_counter()
    for k in range(evals):
        bta.evaluate(mdl, th[k % th.shape[0]], want_grad=with_grad)
    dt = (time.perf_counter() - t0) * scale
    print(json.dumps({"seconds_per_f": dt / evals, "evals": evals, "scale": scale}))


def run_oracle_child(cfg, evals, nt_sample=0, with_grad=False):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--config", str(cfg),
                        "--evals", str(evals), "--nt-sample", str(nt_sample)] + (["--with-grad"] if with_grad else []),
                       capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["seconds_per_f"], cores


NT_SAMPLE = {1: 0, 2: 0, 3: 4, 4: 2, 5: 2}


def cpu_baseline(cfg, grad):
    if grad == "fd":
        sec, cores = run_oracle_child(cfg, 1 if cfg == 2 else 9, NT_SAMPLE[cfg])
        per_grad = 9 * sec   # one f + grad f by central differences = 9 f evaluations
        what = f"oracle f at the stencil centre, {sec:.3f} s per f; 9 f per f+grad f"
    else:
        per_grad, cores = run_oracle_child(cfg, 1, NT_SAMPLE[cfg], with_grad=True)
        what = f"oracle f + adjoint gradient at one point, {per_grad:.3f} s"
    if NT_SAMPLE[cfg]:
        what += f" (built with n_t = {NT_SAMPLE[cfg]}, time scaled linearly to the workload's n_t)"
    return {"value": 1.0 / per_grad, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": what + f"; {cores} host threads (numpy BLAS)"}


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
    if rank != 0:
        return
    cfg = args.config
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; every step below is a fresh evaluation
    times = []
    cores = None
    fd = args.grad == "fd"
    for _ in range(args.steps):
        sec, cores = run_oracle_child(cfg, 1, NT_SAMPLE[cfg], with_grad=not fd)
        times.append(sec)
    t = sum(times) / len(times)
    per = 9 * t if fd else t
    value = 1.0 / per
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * per, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(cfg, world, args.grad, args.precision, l2="CPU oracle: not applicable"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": ("each step: one oracle f evaluation at the stencil centre; "
                                        "f + grad f = 9 such evaluations") if fd else
                                       "each step: one oracle f + adjoint gradient at one point"
                                       + (f" (n_t = {NT_SAMPLE[cfg]}, scaled to the workload's n_t)"
                                          if NT_SAMPLE[cfg] else "")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


L2_BYTES = 129 * 2 ** 20
L2_NOTE_LARGE = "working set (GBs of factor storage per step) exceeds L2; no flush"
L2_NOTE_FLUSH = "working set below 2x L2: a 512 MiB buffer is rewritten before each timed step (outside its events)"


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

def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(args.config, args.evals, args.nt_sample, args.with_grad)
        return
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
    n_p = -(-mdl.n_s // 64) * 64
    tensor_sweep = n_p % 128 == 0 and args.sweep == "tensor"
    if args.gemm or args.sweep:
        model.set_tiles(32, capi.INLA_SWEEP_TF32X3 if tensor_sweep else 64,
                        capi.INLA_GEMM_TF32X3 if args.gemm != "cuda-core" else 128)
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
    for w in range(max(args.warmup, 1)):
        if w == args.warmup - 1:
            model.profile_enable(PROFILE_EVERY)   # creates the event pool outside the timed region
        model.eval(theta, grad=grad, out=out, precision=prec)
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0, "evaluation failed"
    model.profile_enable(PROFILE_EVERY)

    if args.graph:
        model.profile_enable(0)          # event timing and graph replay exclude each other
        model.eval(theta, grad=grad, out=out, precision=prec, use_graph=True)   # capture
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # a working set below twice the L2 would stay cache-resident from step to step: then each
    # step is timed alone, after a buffer larger than L2 has been rewritten
    flush = model.workspace_bytes(theta.shape[0], grad=grad, precision=prec) < 2 * L2_BYTES
    scratch = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda") if flush else None
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    elapsed = 0.0
    if flush:
        for _ in range(args.steps):
            scratch.fill_(1)
            e0.record(stream)
            model.eval(theta, grad=grad, out=out, precision=prec, use_graph=args.graph)
            e1.record(stream)
            launches += model.last_launch_count()
            torch.cuda.synchronize()
            elapsed += e0.elapsed_time(e1) / 1e3
    else:
        e0.record(stream)
        for _ in range(args.steps):
            model.eval(theta, grad=grad, out=out, precision=prec, use_graph=args.graph)
            launches += model.last_launch_count()
        e1.record(stream)
        torch.cuda.synchronize()
        elapsed = e0.elapsed_time(e1) / 1e3
    if dist:
        dist.barrier()
    clk = clocks.stop()
    if dist:
        from paper_2204_04678_gb300.replicas import max_over_ranks
        elapsed = max_over_ranks(elapsed)
    value = world * args.steps * per_step / elapsed

    # dominant instrumented kernel: the sweep's tile update or the selected-inversion GEMM
    fp32 = prec == "mixed"
    tensor_gemm = fp32 and n_p % 128 == 0 and args.gemm != "cuda-core"
    upd_id = capi.KERNEL_GJ_UPDATE32 if fp32 else capi.KERNEL_GJ_UPDATE
    kernels = {"gj_update_kernel": model.profile_read(upd_id), "gemm_nn_kernel": model.profile_read(capi.KERNEL_GEMM)}
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
    if kname == "gj_update_kernel" and fp32 and tensor_sweep and tf32x3_peak:
        peak, bound, peak_source = tf32x3_peak, "tensor", tf32_source
        desc = ("rank-64 update of the FP32 block sweep on the tensor cores (tcgen05, 3xTF32, 128x128 tiles, "
                "K = 64)")
    elif kname == "gemm_nn_kernel" and tensor_gemm and tf32x3_peak:
        peak, bound, peak_source = tf32x3_peak, "tensor", tf32_source
        desc = ("128x128 tile 3xTF32 GEMM of the selected inversion on the tensor cores (tcgen05, operands "
                "split once and loaded by TMA)")
    else:
        peak, bound = (peak_fp32 if fp32 else peak_fp64), "alu"
        peak_source = ("measured on this GPU: " + ("FP32" if fp32 else "FP64")
                       + " FMA loop over all SMs (inla_measure_fp32/fp64_peak), of measured")
        desc = {"gj_update_kernel": ("FP32" if fp32 else "FP64") + " tile update of the block sweep inversion",
                "gemm_nn_kernel": ("FP32" if fp32 else "FP64") + " tile GEMM of the selected inversion"}[kname]
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "gj_update_traffic.txt")
    if kname == "gj_update_kernel" and not fp32 and os.path.exists(tfile):
        for line in open(tfile):
            if line.startswith("bytes_per_unit="):
                traffic = float(line.split("=")[1]) * kunits / max(knl, 1)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "kernel": f"{kname} ({desc})", "timed_every": PROFILE_EVERY, "peak_source": peak_source,
                "launches_timed": knl, "share_of_step": PROFILE_EVERY * kms / 1e3 / elapsed if elapsed else None}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        th_host = theta.cpu().numpy().copy()
        model.eval_host(th_host, grad=grad, precision=prec)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            model.eval_host(th_host, grad=grad, precision=prec)
        e2e_s = (time.perf_counter() - t0) / args.steps
        if dist:
            from paper_2204_04678_gb300.replicas import max_over_ranks
            e2e_s = max_over_ranks(e2e_s)
        nb = th_host.shape[0]
        e2e = {"value": world * per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * nb,
               "d2h_bytes_per_step": nb * (8 + 4 * 8 + 4 + 4)}

    # accuracy of the mixed path against the FP64 path (which matches the oracle
    # to 1e-10 on f): the first point of the batch, with marginal variances
    errors = None
    if prec == "mixed" and not args.no_errors:
        errors = mixed_errors(model, theta[:1], grad)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(cfg, grad)
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "error": str(e)[:200]}

    line = {}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32+f64",
                "data": "synthetic", "config": dict(config_dict(cfg, world, grad, prec, points,
                                                                l2=L2_NOTE_FLUSH if flush else L2_NOTE_LARGE),
                                                    **({"fp32_sweep": "tensor (tcgen05 3xTF32)" if tensor_sweep
                                                        else "cuda-core", "fp32_gemm": "tensor (tcgen05 3xTF32)"
                                                        if tensor_gemm else "cuda-core"} if prec == "mixed" else {})),
                "clocks": clk,
                "gpu_launches": launches,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "f_evals_per_s": 9 * value if grad == "fd" else value,
                "grad_mode": grad,
                "errors_vs_fp64": errors,
                "measured_peaks_tflops": {"fp64_fma": peak_fp64, "fp64_dmma": peak_dmma, "fp32_fma": peak_fp32,
                                          "tf32x3_tensor_from_bf16_sustained": tf32x3_peak},
                "kernels": {k: {"ms_sampled": v[0], "launches_sampled": v[1],
                                "tflops": v[2] * flop_per_unit / (v[0] / 1e3) / 1e12 if v[0] else None}
                            for k, v in kernels.items()}}
        if not (args.nt or args.centres != 1):
            print(json.dumps(line))
    if args.nt or args.centres != 1:
        line["config"]["workload"] = f"profiling case: n_t={mdl.n_t}, {args.centres} stencil centres per step"
        print(json.dumps(line)) if rank == 0 else None
    model.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
