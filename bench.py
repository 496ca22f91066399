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
    2: "st-spde-ar1 n_t=50 grid=32x32 (n_s=1024) n_b=4 m=100000 gaussian; one step = 9-point "
       "central-difference stencil in one FP64 launch",
    1: "st-spde-ar1 n_t=8 grid=8x8 (n_s=64) n_b=2 m=2000 gaussian; one step = 9-point "
       "central-difference stencil in one FP64 launch",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grad", default="fd", choices=["fd", "adjoint"],
                    help="fd: one f+grad from the 9-point stencil per step (the workload's definition); "
                         "adjoint: the 9 stencil points each get f and an adjoint gradient")
    ap.add_argument("--nt", type=int, default=None, help="override n_t (profiling case only)")
    ap.add_argument("--centres", type=int, default=1, help="stencil centres per step (FD mode)")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--evals", type=int, default=1, help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle timing

def oracle_sample(cfg, evals):
    """Time `evals` oracle f evaluations at the stencil centre (runs in a child process)."""
    from oracle import bta
    from synth import config_model, theta_batch
    mdl = config_model(cfg)
    th = theta_batch(cfg, mdl)
    t0 = time.perf_counter()
    for k in range(evals):
        bta.gaussian(mdl, th[k % th.shape[0]])
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds_per_f": dt / evals, "evals": evals}))


def run_oracle_child(cfg, evals):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--config", str(cfg),
                        "--evals", str(evals)], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["seconds_per_f"], cores


def cpu_baseline(cfg):
    sec, cores = run_oracle_child(cfg, 1 if cfg == 2 else 9)
    per_grad = 9 * sec   # one f + grad f by central differences = 9 f evaluations
    return {"value": 1.0 / per_grad, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle f at the stencil centre timed on {cores} host threads (numpy BLAS), "
                      f"{sec:.3f} s per f; 9 f per f+grad f"}


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
    for _ in range(args.steps):
        sec, cores = run_oracle_child(cfg, 1)
        times.append(sec)
    t = sum(times) / len(times)
    value = 1.0 / (9 * t)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * 9 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(cfg, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one oracle f evaluation at the stencil centre; "
                                       "f + grad f = 9 such evaluations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_dict(cfg, world):
    from synth import CONFIGS
    c = CONFIGS[cfg]
    return {"workload": CONFIG_WORKLOAD[cfg], "n_t": c["n_t"], "n_s": c["nx"] ** 2, "n_b": c["n_b"], "m": c["m"],
            "theta_points_per_step": 9, "grad": "central differences (9 points)", "prior_logdet": "kronecker",
            "likelihood": c["lik"], "parallelism": f"theta-replicas x{world}",
            "l2": "working set (>= 3.8 GB factor storage per step) exceeds L2; no flush"}


# ------------------------------------------------------------------ our arm

def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(args.config, args.evals)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
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
    if args.nt:
        from synth import CONFIGS, build
        mdl = build(**dict(CONFIGS[cfg], n_t=args.nt, name="profiling case"))
    else:
        mdl = config_model(cfg)
    centre = theta_batch(cfg, mdl)[0] + 0.01 * rank
    model = pkg.Model(mdl, device=local)
    stream = torch.cuda.current_stream()
    if args.grad == "fd":
        cen = centre[None, :] + 0.01 * np.arange(args.centres)[:, None]
        theta = torch.tensor(cen, dtype=torch.float64, device="cuda")
        per_step = args.centres
    else:
        from synth import fd_stencil
        theta = torch.tensor(fd_stencil(centre), dtype=torch.float64, device="cuda")
        per_step = theta.shape[0]
    grad = args.grad
    out = model.eval(theta, grad=grad)
    for w in range(max(args.warmup, 1)):
        if w == args.warmup - 1:
            model.profile_enable(PROFILE_EVERY)   # creates the event pool outside the timed region
        model.eval(theta, grad=grad, out=out)
    torch.cuda.synchronize()
    assert int(out["status"][0]) == 0, "evaluation failed"
    model.profile_enable(PROFILE_EVERY)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        model.eval(theta, grad=grad, out=out)
        launches += model.last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    if dist:
        t = torch.tensor([elapsed], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t[0])
    value = world * args.steps * per_step / elapsed

    # dominant kernel: rank-64 tile update of the block sweep inversion
    ms, nl, units = model.profile_read(capi.KERNEL_GJ_UPDATE)
    gms, gnl, gunits = model.profile_read(capi.KERNEL_GEMM)
    model.profile_enable(0)
    flop_per_unit = 2.0 * 64 ** 3
    avg_s = ms / 1e3 / max(nl, 1)
    flops_per_launch = units / max(nl, 1) * flop_per_unit
    achieved = flops_per_launch / avg_s / 1e12 if nl else None
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "gj_update_traffic.txt")
    if os.path.exists(tfile):
        for line in open(tfile):
            if line.startswith("bytes_per_unit="):
                traffic = float(line.split("=")[1]) * units / max(nl, 1)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
                "frac": achieved / peak_fp64 if achieved else None, "traffic": traffic,
                "kernel": "gj_update_kernel (FP64 rank-32 tile update of the block sweep inversion)",
                "timed_every": PROFILE_EVERY,
                "peak_source": "measured on this GPU: FP64 FMA loop over all SMs (inla_measure_fp64_peak)",
                "launches_timed": nl, "share_of_step": ms / 1e3 / elapsed if elapsed else None}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        th_host = theta.cpu().numpy().copy()
        model.eval_host(th_host, grad=grad)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            model.eval_host(th_host, grad=grad)
        e2e_s = (time.perf_counter() - t0) / args.steps
        if dist:
            t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t[0])
        nb = th_host.shape[0]
        e2e = {"value": world * per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * nb,
               "d2h_bytes_per_step": nb * (8 + 4 * 8 + 4 + 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(cfg)
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "error": str(e)[:200]}

    line = {}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_dict(cfg, world), "clocks": clk, "gpu_launches": launches,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "f_evals_per_s": 9 * value if grad == "fd" else value,
                "grad_mode": grad,
                "fp64_peaks_tflops": {"fma": peak_fp64, "dmma": peak_dmma},
                "gemm_kernel": {"ms": gms, "launches": gnl,
                                "tflops": gunits * flop_per_unit / (gms / 1e3) / 1e12 if gms else None}}
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
