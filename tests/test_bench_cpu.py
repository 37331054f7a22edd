"""The benchmark's reference arm (the FP64 oracle on the host cores) and its JSON line, on
the CPU: the same metric, unit and workload as the GPU arm, the reported baseline equal to
the line's value, and no output from ranks other than 0."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    return [l for l in p.stdout.splitlines() if l.strip()]


def test_reference_arm_line():
    lines = run_reference()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "pairs/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"] == bench.arm_config(64, 1, "bf16")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "pairs/s" and cb["cores"] >= 1
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == "pairs/s"
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    assert run_reference({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_sgm_path_roofline_arithmetic():
    # 4 directions: 2 + 3 * 3 = 11 volume passes over 4 launches
    r = bench.sgm_path_roofline(vol_bytes=1e9, path_ms_per_call=4.0, npaths=4, hbm_peak_gbs=5000.0,
                                peak_kind="measured")
    assert r["bound"] == "hbm" and r["kernel"] == "sgm_path"
    assert abs(r["per_launch_bytes"] - 11e9 / 4) < 1
    assert abs(r["avg_launch_ms"] - 1.0) < 1e-12
    assert abs(r["achieved"] - 2750.0) < 1e-6 and abs(r["frac"] - 0.55) < 1e-12
