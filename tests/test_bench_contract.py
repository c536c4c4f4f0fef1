"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the JSON contract, on the CPU: one line with the metric, value, timing and
baseline keys; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, wall=None):
    import time
    env = dict(os.environ, **env_extra)
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--cpu-budget", "0.3"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    if wall is not None:
        wall.append(time.perf_counter() - t0)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    wall = []
    lines = _run({}, wall)
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in rec, k
    assert rec["value"] > 0 and rec["unit"] == "MLUPS" and rec["higher_is_better"] is True
    assert rec["steps"] == 1 and rec["warmup"] >= 3 and rec["vs_baseline"] is None
    assert "workload" in rec["config"]
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == rec["value"] and cb["sample"]
    assert rec["e2e"] == {"value": rec["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the line reports what it ran: its own step time fits inside the run,
    # and the extrapolation to the workload mix is stated
    assert 0 < rec["ms_per_step"] * (rec["steps"] + rec["warmup"]) / 1e3 <= wall[0]
    assert rec["config"]["ran"] and "extrapolated" in rec["config"]["value_is"]


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
