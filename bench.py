#!/usr/bin/env python3
"""Throughput of the StereoVAE hot path on synthetic 1242x375 stereo pairs.

One step = sv_pipeline over a batch of pairs: coarse ZNCC + WTA on the x4 box-
downsampled pair (D = 48, 9x9 window) and refinement by the 32/64/128 network to a
full-resolution disparity map.  Two forms:
  fp32  the plain method: FP32 CUDA-core convolutions, launched pair by pair;
  bf16  BF16 tcgen05 implicit-GEMM convolutions, all pairs in one persistent launch
        per layer (when the library has it).
The JSON line's value is the headline form (bf16 when available, else fp32);
both forms are listed under "forms".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank processes its own batch (pairs are independent: weak
scaling, no data-path collective); rank 0 prints the line.  --impl reference times
the FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s at 1242×375 D=48 (plain FP32 vs BF16-batched), ΔEPE vs FP64 oracle"
W, H, D, WIN = 1242, 375, 48, 9
DMAX = 190.0
SGM_P1, SGM_P2 = 0.1, 0.5  # penalties of Eq. 4 for the semi-global matching leg (unstated in the paper)
FP32_PEAK_TFLOPS_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "fp32", "bf16", "fp8", "both"])
    ap.add_argument("--pairs", type=int, default=64, help="pairs per step per GPU")
    ap.add_argument("--distinct", type=int, default=0,
                    help="distinct synthetic pairs per GPU, cycled over the batch (0 = one per pair)")
    ap.add_argument("--cpu-sample", type=int, default=8,
                    help="pairs computed by the CPU oracle (timed baseline and accuracy of every form)")
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads (0 = all host cores)")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven-batch leg (64 pairs of widths 320..1242, BF16, tuned, graph-replayed)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the leg of the paper's Table I network (FP32, same pairs)")
    ap.add_argument("--coarse", action="store_true",
                    help="also time the coarse-stage variants (ZNCC / census cost, SGM / DT aggregation, occlusion "
                         "check and median filter) on the same pairs")
    ap.add_argument("--train-pairs", type=int, default=16)
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch plans (fixed launch order, e.g. for profiler captures)")
    ap.add_argument("--tc-ctas", type=int, default=0,
                    help="with --no-tune: CTAs per SM every tensor-core layer is planned for (0 = deepest ring)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from one ncu
# capture, per pair; valid only while the kernel's sources are unchanged since the capture
# (checked by content hash), else the roofline reports traffic as null.
MEASURED_TRAFFIC = {
    "tc_dec3_final": {"bytes_per_pair": (242.922752e6 + 22.4576e6) / 16,
                      "sources": {"paper_2305_11566_gb300/csrc/conv_tc.cu": "78da2f067884",
                                  "paper_2305_11566_gb300/csrc/sv_ctx.cuh": "a591b9b4c3ec",
                                  "paper_2305_11566_gb300/csrc/sv_internal.cuh": "acfab0daefd1"},
                      "capture": "profiles/dec3_final_fused_16x1242x375.md (16 pairs, scaled by pairs)"},
}


def measured_traffic(kernel, pairs):
    import hashlib
    m = MEASURED_TRAFFIC.get(kernel)
    if m is None:
        return None
    for path, h in m["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest()[:12] != h:
                return None
    return m["bytes_per_pair"] * pairs


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            pass
        return rows

    @staticmethod
    def summarise(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def gpu_id_for(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def levels(h, w):
    out = [(h, w)]
    for _ in range(3):
        h, w = (h + 1) // 2, (w + 1) // 2
        out.append((h, w))
    return out


def upfix_pixels(Ho, Wo):
    """Border pixels of a cropped nearest-x2 + 3x3 layer recomputed by the border-fix kernel."""
    return (Wo if Ho & 1 else 0) + ((Ho - (Ho & 1)) if Wo & 1 else 0)


def pair_work(shape, W, H):
    """Algorithmic work of one W x H pair per profiled kernel: {name: (units, bound)}.

    bound "hbm": bytes that must cross HBM (inputs read once, outputs written once);
    "tensor" / "alu": multiply-adds x 2 of the method, counted on the tensor-core
    form's own arithmetic (decoder: 4 output phases of 2x2 taps on the low-resolution
    grid, i.e. 4 taps per output pixel instead of 9)."""
    (H0, W0), (H1, W1), (H2, W2), (H3, W3) = levels(H, W)
    w, h = W // 4, H // 4
    c1, c2, c3 = shape.enc
    d1, d2, d3 = shape.dec
    lat = shape.latent
    dense = {  # the plain form's direct convolutions (9 taps everywhere)
        "enc1": 2 * H1 * W1 * c1 * 9 * 2,
        "enc2": 2 * H2 * W2 * c2 * 9 * c1,
        "enc3": 2 * H3 * W3 * c3 * 9 * c2,
        "latent": 2 * H3 * W3 * lat * c3,
        "dec1": 2 * H2 * W2 * d1 * 9 * lat,
        "dec2": 2 * H1 * W1 * d2 * 9 * d1,
        "dec3": 2 * H0 * W0 * d3 * 9 * d2,
        "final": 2 * H0 * W0 * 9 * d3,
    }
    out = {k: (v, "alu") for k, v in dense.items()}
    out["zncc_wta"] = (2 * W * H + 2 * w * h, "hbm")
    out["edge_enc1"] = (W * H + 2 * w * h + 2 * H1 * W1 * c1, "hbm")
    out["tc_enc2"] = (dense["enc2"], "tensor")
    out["tc_enc3"] = (dense["enc3"], "tensor")
    out["tc_latent"] = (dense["latent"], "tensor")
    out["tc_dec1"] = (2 * H2 * W2 * d1 * 4 * lat, "tensor")
    out["tc_dec2"] = (2 * H1 * W1 * d2 * 4 * d1, "tensor")
    out["tc_dec3"] = (2 * H0 * W0 * d3 * 4 * d2, "tensor")
    out["tc_dec3_final"] = (out["tc_dec3"][0] + dense["final"], "tensor")
    out["edge_up2fix"] = (2 * 6 * (upfix_pixels(H2, W2) * d1 * lat + upfix_pixels(H1, W1) * d2 * d1), "alu")
    out["edge_final"] = (2 * H0 * W0 * d3 + 2 * w * h + 4 * H0 * W0, "hbm")
    out["e1_to_e4m3"] = (3 * H1 * W1 * c1, "hbm")  # FP8 form: BF16 e1 read, E4M3 codes written
    return out


# Layers of the paper's Table I network: (profile name, mode, k, cout, cin, output level);
# mode 0 conv, 1 stride-2 conv, 2 stride-2 deconvolution; level 0 full, 1 half, 2 quarter,
# 3 eighth resolution.
T1_LAYERS = [("t1_fe1", 0, 5, 32, 1, 1), ("t1_fe2", 0, 5, 32, 1, 1), ("t1_en1", 1, 5, 16, 64, 2),
             ("t1_en1r", 0, 5, 8, 16, 2), ("t1_en2", 1, 5, 32, 24, 3), ("t1_en2r", 0, 5, 16, 32, 3),
             ("t1_heads", 0, 1, 2, 48, 3), ("t1_d1", 0, 1, 32, 1, 3), ("t1_d1r", 0, 5, 16, 80, 3),
             ("t1_d2", 2, 5, 16, 96, 2), ("t1_d2r", 0, 5, 8, 40, 2), ("t1_d", 2, 5, 16, 48, 1),
             ("t1_y", 2, 5, 1, 81, 0)]


def t1_work(W, H):
    """FLOPs (multiply-add = 2) of every Table I layer for one W x H pair: a conv k^2 taps per
    output, a stride-2 deconvolution k^2 / 4 (each output phase reads only its own taps)."""
    lv = levels(H, W)
    out = {}
    for name, mode, k, co, ci, lev in T1_LAYERS:
        Ho, Wo = lv[lev]
        taps = k * k / 4.0 if mode == 2 else k * k
        out[name] = 2.0 * Ho * Wo * co * ci * taps
    return out


def work_per_pair(shape):
    """{kernel: FLOPs per 1242x375 pair} and the ZNCC kernel's algorithmic bytes per pair."""
    f = {k: v for k, (v, _) in pair_work(shape, W, H).items()}
    return f, f["zncc_wta"]


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 FMA lanes x 2 flop x clock: 152 SMs x 128 lanes x 2 x f."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_sgemm_tflops():
    """cuBLAS FP32 SGEMM (TF32 off) 8192^3, best of 5, as a measured CUDA-core FP32 figure."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = torch.empty(n, n, device="cuda")
        for _ in range(2):
            torch.matmul(a, b, out=c)
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
        return 2 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# FP8 dense tensor peak from the measured BF16 one: NVIDIA's nominal dense ratio 4.5 / 2.25.
FP8_OVER_BF16 = 2.0


def kernel_rooflines(prof, steps, shape, sizes, pk, pk_kind, sustained, alu_peak, fp8=False):
    """Roofline of every profiled kernel: algorithmic units of one step (summed over the
    step's pairs) / the kernel's measured time per step, against the matching peak (fp8:
    the tensor-core layers against the FP8 peak, the measured BF16 peak x 2)."""
    work = {}
    for (Wp, Hp) in sizes:
        for k, (u, b) in pair_work(shape, Wp, Hp).items():
            work[k] = (work.get(k, (0, b))[0] + u, b)
    table = {}
    for name, (nl, tot_ms) in sorted(prof.items()):
        if name not in work or tot_ms <= 0:
            continue
        units, bound = work[name]
        ms = tot_ms / steps
        if bound == "hbm":
            ach, peak, unit, src = units / (ms / 1e3) / 1e9, pk["hbm_gbs"], "GB/s", f"{pk_kind} hbm_gbs"
        elif bound == "tensor":
            key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
            ach, peak, unit, src = units / (ms / 1e3) / 1e12, pk[key], "TFLOP/s", f"{pk_kind} {key}"
            if fp8 and name.startswith("tc_"):
                peak, src = peak * FP8_OVER_BF16, src + " x 2 (nominal dense FP8 / BF16 ratio 4.5 / 2.25)"
        else:
            ach, peak, unit, src = units / (ms / 1e3) / 1e12, alu_peak, "TFLOP/s", "derived: " + FP32_PEAK_TFLOPS_NOTE
        table[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                       "units_per_step": units, "ms_per_step": ms, "launches_per_step": nl / steps,
                       "peak_source": src}
    return table


# ------------------------------------------------------------------ ranks (host side)
def rank_pair_seeds(rank: int, pairs_per_rank: int, distinct: int):
    """Seeds of one rank's distinct synthetic pairs: every rank gets its own pairs (the
    work is sharded by pairs, no data-path collective), disjoint from every other rank's."""
    return [1000 + rank * pairs_per_rank + i for i in range(min(distinct, pairs_per_rank))]


def rank_reducers(world: int, dist, device: str):
    """barrier() and max_over_ranks(x): the step time of the job is the slowest rank's."""
    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return barrier, max_over_ranks


def whole_job_value(pairs_per_rank: int, world: int, ms_per_step: float) -> float:
    """Pairs per second of the whole job: every rank's pairs over the slowest rank's step."""
    return pairs_per_rank * world / (ms_per_step / 1e3)


# ------------------------------------------------------------------ our implementation
def time_pipeline(ctx, dps, outs, steps, warmup, st, flush, dev, barrier):
    """Warm up, then time `steps` sv_pipeline calls (CUDA events on the launching stream,
    the L2 flushed before each, outside the events), with per-kernel profiling and clock
    samples.  Returns the per-step times and what was recorded."""
    import torch
    with torch.cuda.stream(st):
        for _ in range(warmup):
            ctx.pipeline(dps, out=outs)
    torch.cuda.synchronize()
    ctx.synchronize(st)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    l0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clk = ClockSampler(gpu_id_for(dev))
    barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(st):
        for k in range(steps):
            flush.fill_(k & 0xFF)  # L2 flush between steps, outside the events
            ev[k][0].record(st)
            ctx.pipeline(dps, out=outs)
            ev[k][1].record(st)
            ctx.profile_read(reset=False)  # read this step's per-kernel events (graph replays reuse them)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    rows = clk.stop()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    launches = ctx.launch_count() - l0
    clocks = ClockSampler.summarise(rows)
    if clocks["samples"] < 3:  # short timed region: sample the same step for ~1.5 s
        clk2 = ClockSampler(gpu_id_for(dev))
        clk2.start()
        t = time.perf_counter()
        while time.perf_counter() - t < 1.5:
            with torch.cuda.stream(st):
                ctx.pipeline(dps, out=outs)
            torch.cuda.synchronize()
        c2 = ClockSampler.summarise(clk2.stop())
        c2["note"] = "timed region shorter than the sampling period: sampled while repeating the step"
        clocks = c2
    ctx.synchronize(st)
    return dict(step_ms=step_ms, prof=prof, launches=launches, clocks=clocks, wall_s=wall)


def dominant_roofline(table, measured_traffic_bytes=None):
    """The roofline entry of the kernel with the largest time share."""
    name = max(table, key=lambda k: table[k]["ms_per_step"])
    r = dict(table[name])
    r["kernel"] = name
    r["traffic"] = measured_traffic_bytes
    return r


def accuracy_report(d_gpu, d_orc, best_o, sec_o, Y_gpu, Y_orc, gt):
    """Errors of one form against the FP64 oracle over a sample of pairs: refined disparity
    (max / mean |dY| everywhere and outside the receptive field of WTA differences), EPE
    change against the ground truth, and the fraction of WTA disparities that differ."""
    import numpy as np
    errs, kept, flips, near, npx, epe_g, epe_o = [], [], 0, 0, 0, [], []
    for dg, do, bo, so, Yg, Yo, g in zip(d_gpu, d_orc, best_o, sec_o, Y_gpu, Y_orc, gt):
        Hh, Ww = Yo.shape
        diff = dg != do
        flips += int(diff.sum())
        near += int((diff & ((bo - so) > 1e-4)).sum())
        npx += diff.size
        m = np.zeros_like(diff)
        for y, x in zip(*np.nonzero(diff)):
            m[max(0, y - 16):y + 17, max(0, x - 16):x + 17] = True
        keep = ~np.repeat(np.repeat(m, 4, 0), 4, 1)
        keep = np.pad(keep, ((0, Hh - keep.shape[0]), (0, Ww - keep.shape[1])), mode="edge")
        e = np.abs(Yg.astype(np.float64) - Yo)
        errs.append(e.ravel())
        kept.append(e[keep].ravel())
        epe_g.append(np.abs(Yg - g).mean())
        epe_o.append(np.abs(Yo - g).mean())
    e = np.concatenate(errs)
    k = np.concatenate(kept)
    return {"max_abs_dy_px": float(e.max()), "mean_abs_dy_px": float(e.mean()),
            "max_abs_dy_px_outside_wta_flips": float(k.max()), "mean_abs_dy_px_outside_wta_flips": float(k.mean()),
            "epe_gpu_vs_gt_px": float(np.mean(epe_g)), "epe_oracle_vs_gt_px": float(np.mean(epe_o)),
            "delta_epe_px": float(np.mean(epe_g) - np.mean(epe_o)),
            "wta_flips": flips, "wta_flip_fraction": flips / npx, "wta_flips_off_near_ties": near,
            "pairs": len(Y_orc)}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2305_11566_gb300 import binding, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.cuda.current_device()
    build.build()
    shape = synth.NET_WIDE
    params = synth.he_normal_weights(shape, 7)
    B = args.pairs
    n_distinct = B if args.distinct <= 0 else min(args.distinct, B)
    distinct = [synth.make_pair(W, H, DMAX, sd) for sd in rank_pair_seeds(rank, B, n_distinct)]
    pairs = [distinct[i % len(distinct)] for i in range(B)]
    dps_distinct = [binding.to_device(p, D) for p in distinct]
    dps = [dps_distinct[i % len(distinct)] for i in range(B)]
    pk, pk_kind = peaks()
    alu_peak = fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    sgemm = measure_sgemm_tflops()

    barrier, max_over_ranks = rank_reducers(world, dist, "cuda")

    forms = []
    if args.form in ("auto", "both"):
        forms = ["fp32"]
        for f in ("bf16", "fp8"):
            try:
                c = binding.Context(shape, WIN, f, dev)
                c.close()
                forms.append(f)
            except Exception:
                pass
    else:
        forms = [args.form]

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()  # a side stream: the batched form replays CUDA graphs there
    results = {}
    tuning = None
    for form in forms:
        ctx = binding.Context(shape, WIN, form, dev)
        ctx.set_weights(params)
        if form == "bf16" and args.tc_ctas:
            ctx.set_option("tc_ctas_per_sm", args.tc_ctas)
        outs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(B)]
        try:
            with torch.cuda.stream(st):
                ctx.pipeline(dps[:1], out=outs[:1])
            torch.cuda.synchronize()
        except binding.SvError:
            if form in ("bf16", "fp8"):
                ctx.close()
                continue
            raise
        if form in ("bf16", "fp8") and not args.no_tune:
            tu = ctx.autotune(dps, stream=st)
            if form == "bf16" or tuning is None:
                tuning = tu
        t = time_pipeline(ctx, dps, outs, args.steps, args.warmup, st, flush, dev, barrier)
        total_ms = max_over_ranks(sum(t["step_ms"]))
        t.update(ctx=ctx, outs=outs, ms_per_step=total_ms / args.steps)
        results[form] = t

    # -------------------------------------------------------------- rooflines of every kernel
    head = next(f for f in ("bf16", "fp8", "fp32") if f in results)
    R = results[head]
    sizes = [(W, H)] * B
    tables = {}
    for form, r in results.items():
        sustained = r["ms_per_step"] * args.steps > 1000
        tables[form] = kernel_rooflines(r["prof"], args.steps, shape, sizes, pk, pk_kind, sustained, alu_peak,
                                        fp8=form == "fp8")
    roof = dominant_roofline(tables[head])
    roof["traffic"] = measured_traffic(roof["kernel"], B)
    shares = {k: round(v[1] / sum(x[1] for x in R["prof"].values()), 4) for k, v in sorted(R["prof"].items())}

    # -------------------------------------------------------------- e2e through the host-buffer API
    e2e = None
    if not args.no_e2e:
        ctx = R["ctx"]
        hl = [torch.from_numpy(synth.pitched(p.left)).pin_memory() for p in distinct]
        hr = [torch.from_numpy(synth.pitched(p.right)).pin_memory() for p in distinct]
        L = [hl[i % len(distinct)] for i in range(B)]
        Rr = [hr[i % len(distinct)] for i in range(B)]
        ho = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(B)]
        pitch = L[0].shape[1]
        args_e2e = (L, Rr, [W] * B, [H] * B, [pitch] * B, [D] * B, ho)
        for _ in range(max(1, args.warmup)):
            ctx.pipeline_host(*args_e2e, stream=st)
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            ctx.pipeline_host(*args_e2e, stream=st)
        el = max_over_ranks(time.perf_counter() - t)
        e2e = {"value": B * world * args.steps / el, "unit": "pairs/s",
               "h2d_bytes_per_step": int(sum(x.numel() for x in L) * 2),
               "d2h_bytes_per_step": int(sum(x.numel() * 4 for x in ho)),
               "api": "sv_pipeline_host (pinned host images in, host disparity maps out)"}

    # -------------------------------------------------------------- the uneven batch (64 pairs, widths 320..1242)
    uneven = None
    if not args.no_uneven and "bf16" in results:
        ub = synth.batch_uneven(B, seed=2000 + 1000 * rank)
        udps = [binding.to_device(p, Dp) for p, Dp in ub]
        uctx = binding.Context(shape, WIN, "bf16", dev)
        uctx.set_weights(params)
        uouts = [torch.empty((p.height, p.width), dtype=torch.float32, device="cuda") for p, _ in ub]
        utune = uctx.autotune(udps, stream=st) if not args.no_tune else None
        ut = time_pipeline(uctx, udps, uouts, args.steps, args.warmup, st, flush, dev, barrier)
        ums = max_over_ranks(sum(ut["step_ms"])) / args.steps
        usizes = [(p.width, p.height) for p, _ in ub]
        utable = kernel_rooflines(ut["prof"], args.steps, shape, usizes, pk, pk_kind, ums * args.steps > 1000, alu_peak)
        widths = [p.width for p, _ in ub]
        uneven = {"workload": f"{B} synthetic pairs per GPU, widths drawn from {{320, 640, 960, 1242}} "
                              f"({', '.join(f'{w}: {widths.count(w)}' for w in (320, 640, 960, 1242))}), "
                              "H = round(0.302 W), D = ceil(W / 26), 9x9 window, 32/64/128 net, BF16, "
                              "autotuned, CUDA-graph replay",
                  "pairs_per_s": whole_job_value(B, world, ums), "ms_per_step": ums,
                  "launches_per_step": ut["launches"] / args.steps, "clocks": ut["clocks"],
                  "roofline": dominant_roofline(utable), "rooflines": utable, "tuning": utune}
        uctx.close()

    # -------------------------------------------------------------- CPU oracle baseline + accuracy
    cpu = None
    accuracy = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        n = max(1, min(args.cpu_sample, len(distinct)))
        cores = args.cpu_threads if args.cpu_threads > 0 else (os.cpu_count() or 1)
        oracle.set_threads(cores)
        t = time.perf_counter()
        ref = []
        for i in range(n):
            p = distinct[i]
            ref.append(oracle.pipeline(shape, params, p.left, p.right, WIN, D))
        el = time.perf_counter() - t
        cpu = {"value": n / el, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "sample": f"{n} of the {B} pairs (1242x375, D=48): coarse match + refinement, FP64, "
                         f"{cores} OpenMP threads, {el:.1f} s"}
        for form, r in results.items():
            dg = [d.cpu().numpy() for d in r["ctx"].coarse_match(dps_distinct[:n], stream=st)]
            torch.cuda.synchronize()
            accuracy[form] = accuracy_report(dg, [x[1] for x in ref], [x[2] for x in ref], [x[3] for x in ref],
                                             [r["outs"][i].cpu().numpy() for i in range(n)], [x[0] for x in ref],
                                             [distinct[i].gt for i in range(n)])
        if "fp8" in results:
            # the FP8 form against the oracle's own quantised refinement (same WTA map), one pair
            Yq = oracle.refine_forward_q(shape, params, distinct[0].left, ref[0][1].astype(np.float64))["Y"]
            e = np.abs(results["fp8"]["outs"][0].cpu().numpy().astype(np.float64) - Yq)
            accuracy["fp8"].update({"vs_quantised_oracle_max_abs_dy_px": float(e.max()),
                                    "vs_quantised_oracle_mean_abs_dy_px": float(e.mean()),
                                    "quantised_oracle_delta_epe_px": float(np.abs(Yq - distinct[0].gt).mean()
                                                                           - np.abs(ref[0][0] - distinct[0].gt).mean())})

    # -------------------------------------------------------------- training step (differentiation form)
    train = None
    if not args.no_train and "bf16" in results:
        from paper_2305_11566_gb300 import autograd as sv_autograd
        tshape = synth.NET_SMALL
        tctx = binding.Context(tshape, WIN, "bf16", dev)
        tctx.set_weights(synth.he_normal_weights(tshape, 7))
        nt = args.train_pairs
        tp = [distinct[i % len(distinct)] for i in range(nt)]
        tdp = [dps_distinct[i % len(distinct)] for i in range(nt)]
        H3, W3 = binding.latent_hw(H, W)
        with torch.cuda.stream(st):
            coarse_i = tctx.coarse_match(tdp)
        st.synchronize()
        tco = [c.float() for c in coarse_i]
        teps = [torch.from_numpy(synth.reparam_noise(H3 * W3 * tshape.latent, 3000 + i)).cuda().reshape(H3, W3, -1)
                for i in range(nt)]
        tgt = [torch.from_numpy(p.gt).cuda() for p in tp]
        wt = torch.from_numpy(synth.he_normal_weights(tshape, 7)).cuda().requires_grad_(True)

        def train_step(t):
            Yt, mut, lvt = sv_autograd.refine(tctx, tdp, tco, teps, wt)
            Lt = sv_autograd.loss(tctx, tdp, Yt, tgt, mut, lvt)
            wt.grad = None
            Lt.backward()
            tctx.adam_step(wt.grad, t)
            return Lt

        with torch.cuda.stream(st):
            for t in range(1, 3):
                train_step(t)
            st.synchronize()
            tsteps = 3
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for t in range(3, 3 + tsteps):
                Lt = train_step(t)
            e1.record(st)
            st.synchronize()
            # one more step with per-kernel events: where the step's time goes
            tctx.profile(True)
            tctx.profile_read(reset=True)
            train_step(3 + tsteps)
            st.synchronize()
            tprof = tctx.profile_read(reset=True)
            tctx.profile(False)
        tms = e0.elapsed_time(e1) / tsteps
        train = {"workload": f"training step: {nt} synthetic 1242x375 pairs, 16/32/64 net, BF16 tensor-core forward, "
                             "FP32 master weights and backward (encoder recomputed), smooth-L1 + 1e-3 KL, Adam",
                 "ms_per_step": tms, "steps_per_s": 1e3 / tms, "pairs_per_s": nt * 1e3 / tms,
                 "loss_last": float(Lt.item()),
                 "kernel_ms_profiled_step": {k: round(v[1], 4) for k, v in sorted(tprof.items(), key=lambda kv: -kv[1][1])}}
        tctx.close()

    table1 = None
    if not args.no_table1:
        tctx = binding.Context("table1", WIN, "fp32", dev)
        tctx.set_weights(synth.table1_weights(7))
        touts = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(B)]
        tt = time_pipeline(tctx, dps, touts, args.steps, args.warmup, st, flush, dev, barrier)
        tms = max_over_ranks(sum(tt["step_ms"])) / args.steps
        tw_ = t1_work(W, H)
        ttab = {}
        for kn, (nl, tot) in sorted(tt["prof"].items()):
            kms = tot / args.steps
            e = {"ms_per_step": kms, "launches_per_step": nl / args.steps}
            if kn in tw_:
                ach = tw_[kn] * B / (kms / 1e3) / 1e12
                e.update({"bound": "alu", "flops_per_step": tw_[kn] * B, "achieved": ach, "peak": alu_peak,
                          "unit": "TFLOP/s", "frac": ach / alu_peak, "peak_source": "derived: " + FP32_PEAK_TFLOPS_NOTE})
            ttab[kn] = e
        table1 = {"workload": f"{B} synthetic 1242x375 pairs per GPU: ZNCC + WTA coarse maps (D=48, 9x9) refined by "
                              "the paper's Table I network (FP32 CUDA cores, all pairs per launch)",
                  "pairs_per_s": whole_job_value(B, world, tms), "ms_per_step": tms,
                  "gflop_per_pair": sum(tw_.values()) / 1e9, "launches_per_step": tt["launches"] / args.steps,
                  "kernels": ttab}
        tctx.close()

    coarse = None
    if args.coarse:
        coarse = coarse_variants(binding, shape, dev, dps, B, world, args, st, flush, pk, pk_kind, max_over_ranks)

    value = whole_job_value(B, world, R["ms_per_step"])
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"bf16": "bf16", "fp8": "e4m3", "fp32": "f32"}[head], "data": "synthetic",
        "config": arm_config(B, world, head, n_distinct),
        "roofline": roof,
        "rooflines": tables[head],
        "kernel_time_share": shares,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(R["launches"]),
        "clocks": R["clocks"],
        "fp32_peaks": {"derived_tflops": alu_peak, "derived_from": FP32_PEAK_TFLOPS_NOTE,
                       "measured_sgemm_tflops": sgemm,
                       "measured_how": "cuBLAS SGEMM 8192^3, TF32 off, best of 5, CUDA events"},
        "forms": {f: {"pairs_per_s": B * world / (r["ms_per_step"] / 1e3), "ms_per_step": r["ms_per_step"],
                      "launches_per_step": r["launches"] / args.steps, **accuracy.get(f, {}),
                      **({"rooflines": tables[f]} if f != head else {})}
                  for f, r in results.items()},
        "delta_epe_px": accuracy.get(head, {}).get("delta_epe_px"),
        "wta_flip_fraction": accuracy.get(head, {}).get("wta_flip_fraction"),
        "tuning": tuning,
        "uneven_batch": uneven,
        "table1_net": table1,
        "train_step": train,
    }
    if coarse is not None:
        line["coarse_variants"] = coarse
    if rank == 0:
        print(json.dumps(line))
    for r in results.values():
        r["ctx"].close()
    if world > 1:
        dist.destroy_process_group()


# Coarse-stage variants timed by --coarse: (name, sv_coarse_opts keywords).  The penalties
# and DT scales are not given by the paper: P1, P2 on the ZNCC cost's [0, 2] range and in
# bits for the 5 x 5 census cost, sigma_s in coarse pixels, sigma_r in intensity levels.
COARSE_VARIANTS = [
    ("S4 ZNCC+SGM", dict(cost="zncc", aggregation="sgm", P1=SGM_P1, P2=SGM_P2, npaths=4)),
    ("S4 ZNCC+SGM+SMP+median", dict(cost="zncc", aggregation="sgm", P1=SGM_P1, P2=SGM_P2, npaths=4, smp=True,
                                    median=True)),
    ("S2 census+SGM", dict(cost="census", census_window=5, aggregation="sgm", P1=2.0, P2=12.0, npaths=4)),
    ("S3 ZNCC+DT", dict(cost="zncc", aggregation="dt", dt_sigma_s=8.0, dt_sigma_r=20.0, dt_iters=2)),
    ("S1 census+DT", dict(cost="census", census_window=5, aggregation="dt", dt_sigma_s=8.0, dt_sigma_r=20.0,
                          dt_iters=2)),
]


def coarse_kernel_bytes(name, W, H, D, npaths=4, dt_iters=2):
    """Algorithmic HBM bytes of one call's kernel `name` for one W x H pair with D
    disparities (summed over that kernel's launches in the call): the FP32 cost volume V
    = 4 w h D bytes is the unit; maps are int16, codes uint64, box sums int32."""
    w, h = W // 4, H // 4
    V = 4 * w * h * D
    return {
        "zncc_cost": 2 * W * H + V + 2 * w * h,           # images in, volume and map out
        "box4": 2 * W * H + 8 * w * h,                    # images in, box sums out
        "census_codes": 8 * w * h + 16 * w * h,           # box sums in, codes out
        "census_cost": 16 * w * h + V,                    # codes in, volume out
        # first direction: C in, A out; middle ones: C, A in, A out; the last: C, A in, map out
        "sgm_path": (2 * V if npaths == 1 else 2 * V + 3 * V * (npaths - 2) + 2 * V) + 2 * w * h,
        "dt_rows": dt_iters * (2 * V + 4 * w * h),        # volume in and out, guide in
        "dt_cols": dt_iters * (2 * V + 4 * w * h),
        "vol_wta": V + 2 * w * h,
        "smp": 4 * w * h,                                 # map in, map out
        "median3": 4 * w * h,
    }.get(name, 0)


def coarse_variants(binding, shape, dev, dps, B, world, args, st, flush, pk, pk_kind, max_over_ranks):
    """Time every coarse-stage variant on the step's pairs: pairs/s and the HBM roofline of
    each of its kernels."""
    import torch
    ctx = binding.Context(shape, WIN, "bf16", dev)
    out = {}
    try:
        for name, kw in COARSE_VARIANTS:
            opts = binding.coarse_opts(**kw)
            with torch.cuda.stream(st):
                for _ in range(args.warmup):
                    ctx.coarse_match_ex(dps, opts, stream=st)
            torch.cuda.synchronize()
            ctx.profile(True)
            ctx.profile_read(reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            with torch.cuda.stream(st):
                for k in range(args.steps):
                    flush.fill_(k & 0xFF)
                    ev[k][0].record(st)
                    ctx.coarse_match_ex(dps, opts, stream=st)
                    ev[k][1].record(st)
            torch.cuda.synchronize()
            prof = ctx.profile_read(reset=True)
            ctx.profile(False)
            ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev)) / args.steps
            kernels = {}
            for kn, (nl, tot) in sorted(prof.items()):
                kms = tot / args.steps
                units = sum(coarse_kernel_bytes(kn, dp.width, dp.height, dp.max_disp, kw.get("npaths", 4),
                                                kw.get("dt_iters", 2)) for dp in dps)
                e = {"ms_per_step": kms, "launches_per_step": nl / args.steps}
                if units:
                    ach = units / (kms / 1e3) / 1e9
                    e.update({"bound": "hbm", "bytes_per_step": units, "achieved": ach, "peak": pk["hbm_gbs"],
                              "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "peak_source": f"{pk_kind} hbm_gbs"})
                kernels[kn] = e
            out[name] = {"options": kw, "pairs_per_s": whole_job_value(B, world, ms), "ms_per_step": ms,
                         "kernels": kernels}
    finally:
        ctx.close()
    return out


def arm_config(B, world, head, distinct=None):
    """The workload both arms report (the reference arm times samples of it)."""
    distinct = B if distinct is None else distinct
    return {"workload": f"{B} synthetic 1242x375 stereo pairs per GPU, D=48, 9x9 ZNCC window, "
                        f"32/64/128 encoder, 128 latent, 128/64/32 decoder ({head} form)",
            "distinct_pairs_per_gpu": distinct,
            "global_batch": B * world, "pairs_per_gpu": B, "width": W, "height": H, "max_disp": D,
            "window": WIN, "l2": "flushed between steps (512 MB write outside the timed events)",
            "parallelism": f"replicas x{world} (pairs sharded, no collective)"}


# ------------------------------------------------------------------ reference arm: the CPU oracle
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2305_11566_gb300 import synth
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    shape = synth.NET_WIDE
    params = synth.he_normal_weights(shape, 7)
    p = synth.make_pair(W, H, DMAX, 1000)
    for _ in range(args.warmup):
        oracle.pipeline(shape, params, p.left, p.right, WIN, D)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.pipeline(shape, params, p.left, p.right, WIN, D)
    el = time.perf_counter() - t
    value = args.steps / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args.pairs, args.gpus, "bf16"),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"one pair of the workload per step ({args.steps} timed), coarse match + "
                                   f"refinement, FP64 oracle, {cores} threads"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
