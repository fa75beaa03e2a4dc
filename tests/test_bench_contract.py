"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the keys the benchmark contract names (CPU only; the GPU
arm needs a GB300)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    import time
    t0 = time.perf_counter()
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "planted2k",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    wall_ms = (time.perf_counter() - t0) * 1e3
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is False and line["unit"] == "ms" and line["value"] > 0
    # ms_per_step is what a timed step took (it fits the process's own wall
    # time); value scales that sample to the whole workload
    assert line["steps"] * line["ms_per_step"] <= wall_ms
    assert abs(line["value"] - line["ms_per_step"] * line["value_scale"]) <= 1e-9 * line["value"]
    assert line["config"]["workload"] and line["config"]["m"] == 2000 and line["config"]["n"] == 1000
    # the same workload dict the GPU arm prints (implementation keys live outside config)
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.workload_config(bench.WORKLOADS["planted2k"], 1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "ms"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "planted2k",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=env)
    assert res.returncode == 0 and not res.stdout.strip()
