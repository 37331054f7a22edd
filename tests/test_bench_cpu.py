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


def test_coarse_kernel_bytes():
    # SGM, 4 directions: 2 + 3 + 3 + 2 = 10 volume passes (the last direction writes only the
    # winner-take-all map); DT: every iteration reads and writes the volume once per pass
    V = 4 * 310 * 93 * 48
    assert bench.coarse_kernel_bytes("sgm_path", 1242, 375, 48, 4) == 10 * V + 2 * 310 * 93
    assert bench.coarse_kernel_bytes("dt_rows", 1242, 375, 48, dt_iters=3) == 3 * (2 * V + 4 * 310 * 93)


def test_kernel_rooflines_arithmetic():
    """Per-kernel rooflines: units of a step summed over its pairs, divided by the kernel's
    time per step, against the peak of the kernel's bound."""
    from paper_2305_11566_gb300 import synth
    shape = synth.NET_WIDE
    pk = {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1500.0}
    prof = {"zncc_wta": (4, 2.0), "tc_dec2": (4, 8.0), "edge_up2fix": (8, 1.0)}
    sizes = [(1242, 375), (320, 97)]
    t = bench.kernel_rooflines(prof, 4, shape, sizes, pk, "measured", False, 80.0)
    w1, w2 = bench.pair_work(shape, 1242, 375), bench.pair_work(shape, 320, 97)
    z = t["zncc_wta"]
    assert z["bound"] == "hbm" and z["unit"] == "GB/s"
    assert z["units_per_step"] == w1["zncc_wta"][0] + w2["zncc_wta"][0] == 2 * 1242 * 375 + 2 * 310 * 93 + \
        2 * 320 * 97 + 2 * 80 * 24
    assert abs(z["achieved"] - z["units_per_step"] / 0.5e-3 / 1e9) < 1e-9 and abs(z["frac"] - z["achieved"] / 5000) < 1e-12
    d = t["tc_dec2"]
    assert d["bound"] == "tensor" and d["peak"] == 2000.0 and d["ms_per_step"] == 2.0
    # dec2 of the 4-phase form: 4 taps per output pixel at level 1 (188 x 621 for 1242 x 375)
    assert w1["tc_dec2"][0] == 2 * 188 * 621 * 64 * 4 * 128
    assert t["edge_up2fix"]["bound"] == "alu" and t["edge_up2fix"]["peak"] == 80.0
    # the fused last decoder layer carries the final conv's FLOPs too
    assert w1["tc_dec3_final"][0] == w1["tc_dec3"][0] + w1["final"][0]
    r = bench.dominant_roofline(t)
    assert r["kernel"] == "tc_dec2"


def test_accuracy_report_counts_flips_and_masks_them():
    import numpy as np
    d_o = np.zeros((40, 40), np.int16)
    d_g = d_o.copy()
    d_g[5, 5] = 3                     # one difference, on a near tie of the oracle
    best, sec = np.ones((40, 40)), np.ones((40, 40)) * 0.5
    sec[5, 5] = best[5, 5] - 1e-7
    Yo = np.zeros((160, 160))
    Yg = Yo.copy()
    Yg[20:24, 20:24] = 7.0            # large error inside the flip's reach
    Yg[150, 150] = 0.01               # small error far away
    gt = np.zeros((160, 160), np.float32)
    r = bench.accuracy_report([d_g], [d_o], [best], [sec], [Yg], [Yo], [gt])
    assert r["wta_flips"] == 1 and abs(r["wta_flip_fraction"] - 1 / 1600) < 1e-15
    assert r["wta_flips_off_near_ties"] == 0
    assert r["max_abs_dy_px"] == 7.0 and abs(r["max_abs_dy_px_outside_wta_flips"] - 0.01) < 1e-12
