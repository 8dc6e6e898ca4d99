"""The reference arm of bench.py on the host cores (the FP64 oracle on a
bounded sample of the production workload): one JSON line with the keys the
bench contract names, the same metric and workload keys as the GPU arm, and
a refusal of too few warm-up steps."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    env = dict(os.environ, OMP_NUM_THREADS=str(min(8, os.cpu_count() or 1)))
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout, env=env)


def test_reference_arm_json_line():
    cp = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert cp.returncode == 0, cp.stderr[-2000:]
    line = json.loads(cp.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "GLUPS" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["config"]["workload"] == "lbm-pwfa 512x256x256 dx0.05 regularized driver-in-box"
    assert line["config"]["driver"]["z0"] == 2.0
    assert line["config"]["grid_zyx"] == [512, 256, 256]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_too_few_warmup_steps_refused():
    cp = _run("--impl", "reference", "--steps", "1", "--warmup", "1", timeout=120)
    assert cp.returncode != 0 and "--warmup" in cp.stderr
