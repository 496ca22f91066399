"""bench.py's reference arm (the CPU oracle timed on the host cores) keeps the
benchmark's one-line JSON contract; runs on the CPU at the smallest workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("st-spde-ar1 n_t=8 grid=8x8")
    assert abs(line["ms_per_step"] - 1e3 / line["value"]) <= 1e-6 * line["ms_per_step"]
    # both arms describe the workload with the same config dict
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.config_dict(1, 1, "fd", "fp64", l2=bench.L2_NOTE_FLUSH)
    assert line["cpu_baseline"]["nproc"] >= 1 and line["cpu_baseline"]["cpu_model"]
