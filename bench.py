"""Benchmark: smoothed-Hessian estimates per second on the mesh workload.

Workload (one "step" = one whole estimate through the hot path: Philox
sampler, 4096 fused render+loss passes, estimator sums): a closed surface of
revolution of 2048 triangles, 256 x 256 RGB, flat Lambert shading, 2 rotation
parameters, sigma = 0.1 rad, aggregate importance sampling of the 2 x 2
Hessian with M = 4096 perturbations.  Inputs are resident on the device when
the timed region starts; L2 (126 MB) is flushed by writing a 256 MiB buffer
before every timed step, outside the timed events.

`value` times the device-pointer entry point (hr_estimate_dev) with CUDA
events on the launching stream; `e2e` times the host-pointer entry point
(hr_estimate_hessian: parameters up, Hessian down) with the host clock.
The roofline line is for the render+loss kernel, timed per launch with the
library's own events; its algorithmic work is an FP32-operation count (see
`revolve_work`).  `cpu_baseline` runs the oracle (plain single-threaded C,
FP64) on a bounded sample of the same estimate.

Multi-GPU: estimates are independent, so N ranks run N replicas (weak
scaling, no collective on the data path); `value` = all ranks' estimates /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian/HVP estimates/s at oracle-matched error; perturbed renders/s; p50/p99 latency"
M_PERTURB = 4096
SEED = 2024

REASONS = ["gpu_idle", "applications_clocks_setting", "sw_power_cap", "hw_slowdown", "sync_boost",
           "sw_thermal_slowdown", "hw_thermal_slowdown", "hw_power_brake_slowdown"]


def workload_config(sc):
    return {"workload": "revolve3d: 2048-triangle surface of revolution, 256x256 RGB, 2 rotation params, "
                        "sigma 0.1 rad, aggregate 2x2 Hessian, M=4096 perturbations",
            "triangles": int(len(sc["triangles"])), "width": sc["width"], "height": sc["height"],
            "n_params": 2, "sigma": sc["sigma"], "n_perturb": M_PERTURB, "strategy": "aggregate",
            "l2": "flushed before every timed step (256 MiB write, outside the timed events)"}


def revolve_work(sc, theta):
    """Algorithmic FP32 operations of one render of the mesh at theta:
    15 per vertex (transform, projection), 40 per triangle (edges, cull,
    bounding box, depth plane, shade), 10 per (pixel, front-facing triangle
    whose pixel bounding box contains the pixel) (3 edge functions, depth,
    compares), 9 per pixel (shading and the 3-channel squared error)."""
    a, b = float(np.float32(theta[0])), float(np.float32(theta[1]))
    ca, sa, cb, sb = math.cos(a), math.sin(a), math.cos(b), math.sin(b)
    R = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]]) @ np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    V = sc["vertices"].astype(np.float64) @ R.T
    W, H = sc["width"], sc["height"]
    Z = float(sc["eye_dist"]) - V[:, 2]
    k = float(sc["scale"])
    sx, sy = k * V[:, 0] / Z + W / 2, -k * V[:, 1] / Z + H / 2
    T = sc["triangles"]
    ax, ay, bx, by, cx, cy = sx[T[:, 0]], sy[T[:, 0]], sx[T[:, 1]], sy[T[:, 1]], sx[T[:, 2]], sy[T[:, 2]]
    area = (bx - ax) * (ay - cy) - (by - ay) * (ax - cx)      # > 0: front-facing in y-down screen space
    front = area > 0
    x0 = np.clip(np.ceil(np.minimum(np.minimum(ax, bx), cx) - 0.5), 0, W)
    x1 = np.clip(np.floor(np.maximum(np.maximum(ax, bx), cx) - 0.5), -1, W - 1)
    y0 = np.clip(np.ceil(np.minimum(np.minimum(ay, by), cy) - 0.5), 0, H)
    y1 = np.clip(np.floor(np.maximum(np.maximum(ay, by), cy) - 0.5), -1, H - 1)
    cand = np.where(front, np.maximum(0, x1 - x0 + 1) * np.maximum(0, y1 - y0 + 1), 0).sum()
    return 15 * len(V) + 40 * len(T) + 10 * float(cand) + 9 * W * H, float(cand)


class ClockSampler:
    def __init__(self, index):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
                mask = int(parts[3], 16)
            except ValueError:
                continue
            for bit, name in enumerate(REASONS):
                if mask & (1 << bit) and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(sc, theta, sample=1024):
    """The oracle, single-threaded, on the first `sample` perturbations of the
    same estimate; scaled to estimates/s of the full M."""
    import oracle as O
    t0 = time.perf_counter()
    r = O.RevolveRenderer(sc)
    tau, _ = O.draw(1, 2, sc["sigma"], sample // 2, SEED, 0, 0)
    w = O.weights(1, 2, sc["sigma"], tau)
    t1 = time.perf_counter()
    losses = np.array([r.loss(O.perturb(theta, tau[m])) for m in range(sample)])
    _ = (w * losses[:, None]).sum(0)
    t2 = time.perf_counter()
    per_render = (t2 - t1) / sample
    est_s = per_render * M_PERTURB + (t1 - t0) * M_PERTURB / sample
    return {"value": 1.0 / est_s, "unit": "estimates/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample} of the {M_PERTURB} perturbations of one estimate (plain C, FP64 values), "
                      f"scaled to one full estimate", "renders_per_s": 1.0 / per_render}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2412_03489_gb300 import workloads as wl
    sc = wl.revolve_scene()
    theta = np.asarray(sc["theta_query"], np.float64)
    sample = 256
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(sc, theta, sample=sample)
        if i >= args.warmup:
            times.append(1.0 / cb["value"])
    est_s = float(np.mean(times))
    val = 1.0 / est_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "estimates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sc),
            "cpu_baseline": {"value": val, "unit": "estimates/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: {sample} of the {M_PERTURB} perturbations, scaled to one estimate"},
            "e2e": {"value": val, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2412_03489_gb300 import hr
    from paper_2412_03489_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    sc = wl.revolve_scene()
    S = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"], np.float64)
    stream = torch.cuda.Stream()            # a real stream handle (the legacy default stream is 0 = NULL)
    torch.cuda.set_stream(stream)
    d_theta = torch.tensor(theta, dtype=torch.float64, device="cuda")
    d_out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    hr.hr_profile_enable(S.handle, True)

    def step(i):
        o = hr.make_opts(sc["sigma"], M_PERTURB, hr.HR_AGGREGATE, SEED, 1000 * rank + i, stream=stream.cuda_stream)
        hr.hr_estimate_dev(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None, o, d_out.data_ptr())

    for i in range(args.warmup):
        flush.fill_(float(i))
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    times, render_ms = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev0.record(stream)
        step(args.warmup + i)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        render_ms.append(float(hr.hr_profile_last(S.handle)[1]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(np.sum(times))
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = world * args.steps / (total_ms / 1e3)

    # end to end through the host-pointer entry point
    hr.hr_profile_enable(S.handle, False)
    Hh = np.zeros((2, 2))
    for i in range(2):
        S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], M_PERTURB, hr.HR_AGGREGATE, SEED, 500000 + i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(3, args.steps // 3)
    for i in range(ne):
        o = hr.make_opts(sc["sigma"], M_PERTURB, hr.HR_AGGREGATE, SEED, 600000 + i)
        hr.hr_estimate_hessian(S.handle, theta, o, Hh)
    e2e_s = (time.perf_counter() - t0) / ne

    if rank == 0:
        peaks, src = measured_peaks()
        ops, cand = revolve_work(sc, theta)
        render_avg_s = float(np.mean(render_ms)) / 1e3
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        peak_ops = n_sm * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        achieved = ops * M_PERTURB / render_avg_s
        line = {"metric": METRIC, "value": value, "unit": "estimates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(sc),
                "renders_per_s": value * M_PERTURB,
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                "roofline": {"bound": "alu", "kernel": "revolve_kernel (render + loss)",
                             "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                             "frac": achieved / peak_ops, "traffic": None,
                             "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                            f"({src} max SM clock); one FMA = one operation",
                             "ops_per_render": ops, "pixel_triangle_candidates_per_render": cand,
                             "render_ms_per_launch": render_avg_s * 1e3},
                "e2e": {"value": 1.0 / e2e_s, "unit": "estimates/s", "h2d_bytes_per_step": 8 + 40,
                        "d2h_bytes_per_step": 32},
                "gpu_launches": 3 * args.steps,
                "clocks": clk}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(sc, theta)
        print(json.dumps(line))
    S.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
