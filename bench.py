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
`revolve_work`).  `cpu_baseline` runs the oracle (plain C renders, FP64
sums) on the same estimate with its renders split over all host threads, and
on a bounded sample with one thread (`single_thread`).

`secondary` (rank 0, after the headline's timed region; --no-secondary
skips it) reports the other configurations compactly: the path-traced HVP
(8,192 perturbations) with its roofline from counted rays, one batched
Newton-CG step (64 instances, CUDA graph), serving on a seeded stream of
1,200 requests against the same requests one at a time, and the disc
configuration's element-wise Hessians through the persistent queue (one
resident launch, batched host submission) against the same requests one at
a time; the path tracer's sampled renders are checked against the oracle in
the cpu_baseline leg.

Multi-GPU: estimates are independent, so N ranks run N replicas (weak
scaling, no collective on the data path); `value` = all ranks' estimates /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
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
# From the ncu capture of the current mesh kernel (its compact-layout launch,
# which does the renders of this workload); set to None when the kernel
# changes until it is captured again: DRAM bytes (read + write) of one
# render+loss launch, and the fraction of instruction issue slots busy
# (smsp__issue_active) — the kernel is bound by compare / select issue on the
# ALU pipe rather than by FP32 arithmetic.
TRAFFIC_BYTES = 543232
ISSUE_ACTIVE_NCU = 0.727
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


def ptbox_work(W, H, spp, hit_rays, shadow_rays, vertices):
    """Algorithmic FP32 operations of one path-traced render from its ray
    counts (measured by the counting build): 154 per closest-hit ray from
    inside the box (3 forward walls, 6 block faces and the light at 10
    operations each: subtract, multiply, two FMAs, six compares; 3 spheres at
    18 each), 124 per shadow ray (the 6 block faces and the light; no wall
    when the light lies inside them), 40 per shaded vertex (hit point,
    normal, light sample, direction, distance, cosines, throughput), 33 per
    continuation (disc sample, lift, orthonormal basis, direction), 12 per
    camera ray and 12 per pixel (average, squared error).  The Philox words
    (integer) are not counted."""
    cam = W * H * spp
    return (154.0 * hit_rays + 124.0 * shadow_rays + 40.0 * vertices + 33.0 * (hit_rays - cam) + 12.0 * cam
            + 12.0 * W * H)


def secondary_workloads(torch, hr, wl, stream, flush, peaks, n_sm):
    """The other configurations, compactly, outside the headline's timed
    region: the path-traced HVP (8,192 perturbations, 3 timed steps, roofline
    from counted rays), one batched Newton-CG step (64 instances, graph, 3
    timed steps), and serving on a 1,200-request seeded stream against the
    same requests one at a time."""
    out = {}
    # path tracer
    sc = wl.ptbox_scene()
    S = hr.Scene(sc)
    d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
    d_v = torch.tensor(sc["v"], dtype=torch.float64, device="cuda")
    d_out = torch.zeros(6, dtype=torch.float64, device="cuda")
    tuning = tune_scene(hr, S, sc["theta_query"], 2048)
    hr.hr_profile_enable(S.handle, True)
    M = 8192
    stage = []

    def pt_step(i):
        o = hr.make_opts(sc["sigma"], M, hr.HR_AGGREGATE, SEED, i, stream=stream.cuda_stream)
        hr.hr_estimate_dev(S.handle, hr.HR_HVP, d_theta.data_ptr(), d_v.data_ptr(), o, d_out.data_ptr())
    times = []
    for i in range(4):
        flush.fill_(float(i))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        pt_step(i)
        ev1.record(stream)
        ev1.synchronize()
        if i:
            times.append(ev0.elapsed_time(ev1))
            stage.append(hr.hr_profile_last(S.handle).astype(np.float64))
    hr.hr_profile_enable(S.handle, False)
    # work per render from the counting build (512 renders, other requests)
    hr.hr_scene_count_work(S.handle, True)
    S.estimate(hr.HR_HVP, np.asarray(sc["theta_query"]), sc["sigma"], 512, hr.HR_AGGREGATE, SEED, 7000, v=sc["v"])
    hr.hr_scene_count_work(S.handle, False)
    st = hr.hr_scene_get_stats(S.handle)
    n = max(1, st.pt_counted_renders)
    rays = (st.pt_hit_rays / n, st.pt_shadow_rays / n, st.pt_vertices / n)
    ops = ptbox_work(sc["width"], sc["height"], sc["spp"], *rays)
    render_ms = float(np.mean([x[1] for x in stage]))
    peak_ops = n_sm * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    achieved = ops * M / (render_ms / 1e3)
    t = float(np.mean(times))
    out["ptbox_hvp"] = {
        "workload": "path-traced box 128x128 RGB, 4 spp, depth 3, 6 params, sigma 0.05, aggregate HVP, "
                    "8192 perturbations", "steps": len(times),
        "estimates_per_s": 1e3 / t, "renders_per_s": M * 1e3 / t, "ms_per_estimate": t,
        "stage_ms": dict(zip(("sample", "render_loss", "sums"), np.mean(stage, axis=0).tolist())),
        "roofline": {"bound": "alu", "kernel": "ptbox_kernel (path tracing + loss)", "achieved": achieved / 1e12,
                     "peak": peak_ops / 1e12, "unit": "TFLOP/s", "frac": achieved / peak_ops,
                     "ops_per_render": ops, "rays_per_render": {"closest_hit": rays[0], "shadow": rays[1],
                                                               "shaded_vertices": rays[2]}},
        "tuning": tuning}
    S.close()
    # Newton-CG
    sc = wl.tris2d_scene()
    S = hr.Scene(sc)
    B = 64
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 32, 32, 10
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base = 1e-3, 0.05, SEED, 0
    opts.use_graph, opts.stream = 1, stream.cuda_stream
    st_ = hr.hr_optstate_create(S.handle, B, np.ascontiguousarray(sc["theta_init"], np.float64), opts)
    times = _timed_steps(torch, stream, flush, lambda i: hr.hr_newton_cg_step(S.handle, st_, None), 3, 3)
    hr.hr_optstate_destroy(st_)
    S.close()
    t = float(np.mean(times))
    out["newton_cg"] = {
        "workload": "16 coloured triangles 256x256, 64 params, 64 instances, 32 gradient + 10 x 32 HVP renders "
                    "per instance-step, CUDA graph", "steps": len(times),
        "launch_steps_per_s": 1e3 / t, "instance_steps_per_s": B * 1e3 / t, "ms_per_step": t,
        "renders_per_s": B * (32 + 10 * 32) * 1e3 / t}
    # serving
    sv = serving_bench(torch, hr, wl, n_requests=1200, sweep=False)
    out["serving"] = {"workload": sv["config"]["workload"] + " (1,200 requests)", "requests": sv["requests"],
                      "plain_one_at_a_time_estimates_per_s": sv["plain_one_at_a_time"]["estimates_per_s"],
                      "served_saturated_estimates_per_s": sv["served_saturated"]["estimates_per_s"],
                      "speedup_vs_plain": sv["served_saturated"]["speedup_vs_plain"],
                      "results_identical_to_plain": sv["served_saturated"]["results_identical_to_plain"]}
    out["disc_queue"] = disc_queue_bench(torch, hr, wl, stream, flush)
    return out


def disc_queue_bench(torch, hr, wl, stream, flush, n_requests=20000, batch=512, window=4096):
    """The disc configuration's element-wise Hessians (64x64, n = 2, 3 x 1024
    perturbations each) through the persistent queue, end to end from host
    arrays to host results: requests go in with hr_queue_submit_many in
    batches, at most `window` in flight, and come back with hr_queue_wait_many.
    Beside it the same requests one at a time: through hr_estimate_dev timed
    on the device (sampler, render, sums: three launches per estimate) and
    through the host entry point hr_estimate_hessian.  A single request's
    submit-to-result latency through the queue is sampled alone."""
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    M = 1024
    g = np.random.default_rng(SEED)
    thetas = np.asarray(sc["theta_query"], np.float64) + g.normal(0.0, 0.01, (n_requests, 2))
    seeds = np.arange(n_requests) + SEED
    arr = hr.opts_array(sc["sigma"], M, hr.HR_ELEMENTWISE, seeds, np.arange(n_requests))
    osz = ctypes.sizeof(hr.hr_opts)
    # plain, one request at a time: device-timed (hr_estimate_dev) and host entry point
    d_theta = torch.tensor(thetas[0], dtype=torch.float64, device="cuda")
    d_out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    n_dev = 2000

    def dev_batch(i):
        for k in range(n_dev):
            o = hr.make_opts(sc["sigma"], M, hr.HR_ELEMENTWISE, int(seeds[k]), k, stream=stream.cuda_stream)
            hr.hr_estimate_dev(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None, o, d_out.data_ptr())
    dev_ms = float(np.mean(_timed_steps(torch, stream, flush, dev_batch, 1, 2))) / n_dev
    host_out = np.zeros((2, 2))
    t0 = time.perf_counter()
    for k in range(n_dev):
        hr.hr_estimate_hessian(S.handle, thetas[k], arr[k], host_out)
    host_s = (time.perf_counter() - t0) / n_dev
    # through the queue
    q = hr.hr_queue_create(S, max_requests=window, idle_budget_us=2000, arena_bytes=1 << 30)
    out = np.zeros((n_requests, 4))

    def run_all():
        sub, waited, inflight = 0, 0, []
        while waited < n_requests:
            if sub < n_requests and sub - waited < window:
                cnt = min(batch, n_requests - sub, window - (sub - waited))
                view = (hr.hr_opts * cnt).from_buffer(arr, sub * osz)
                t = hr.hr_queue_submit_many(q, hr.HR_HESSIAN, thetas[sub:sub + cnt], None, view)
                if len(t):
                    inflight.append((sub, t))
                    sub += len(t)
                if len(t) == cnt:
                    continue
            st, t = inflight.pop(0)
            hr.hr_queue_wait_many(q, t, out[st:st + len(t)])
            waited += len(t)
    run_all()                                   # warm-up pass
    t0 = time.perf_counter()
    run_all()
    q_s = time.perf_counter() - t0
    lat = []
    one = np.zeros((1, 4))
    for k in range(300):
        view = (hr.hr_opts * 1).from_buffer(arr, k * osz)
        a = time.perf_counter()
        t = hr.hr_queue_submit_many(q, hr.HR_HESSIAN, thetas[k:k + 1], None, view)
        hr.hr_queue_wait_many(q, t, one)
        lat.append(time.perf_counter() - a)
    status, launches = hr.hr_queue_status(q)
    hr.hr_queue_destroy(q)
    same = True
    for k in list(range(0, n_requests, n_requests // 64)) + [n_requests - 1]:
        hr.hr_estimate_hessian(S.handle, thetas[k], arr[k], host_out)
        same &= bool(np.array_equal(host_out.ravel(), out[k]))
    S.close()
    rate = n_requests / q_s
    return {"workload": "disc2d 64x64 gray, r 0.2, 2 params, sigma 0.05, element-wise Hessian, 3 x 1024 "
                        "perturbations", "requests": n_requests, "batch": batch, "window": window,
            "queue_estimates_per_s": rate, "queue_renders_per_s": rate * 3 * M,
            "plain_device_estimates_per_s": 1e3 / dev_ms, "plain_host_estimates_per_s": 1.0 / host_s,
            "speedup_vs_plain_device": rate * dev_ms / 1e3,
            "alone_latency_us": {"p50": 1e6 * float(np.percentile(lat, 50)),
                                 "p99": 1e6 * float(np.percentile(lat, 99))},
            "launches": int(launches), "results_identical_to_plain": same}


def ptbox_oracle_match(hr, wl):
    """Sampled renders of the path-traced HVP request against the oracle's
    path tracer on the same perturbations (cpu_baseline leg): 8 renders spread
    over the 8,192, max relative loss difference."""
    import oracle as O
    sc = wl.ptbox_scene()
    S = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"])
    M = 8192
    _, dbg = S.estimate(hr.HR_HVP, theta, sc["sigma"], M, hr.HR_AGGREGATE, SEED, 0, v=sc["v"], debug=True)
    S.close()
    r = O.PtboxRenderer(sc)
    picks = [0, 1, 2047, 2048, 4095, 6000, 8190, 8191]
    ref = np.array([r.loss(O.perturb(theta, dbg["tau"][m]), dict(seed=SEED, request=0, sub=0, k=m // 2))
                    for m in picks])
    rel = np.abs(dbg["losses"][picks].astype(np.float64) - ref) / np.abs(ref)
    return {"renders_compared": len(picks), "max_rel_loss_err": float(rel.max()), "tolerance": 1e-4}


class ClockSampler:
    def __init__(self, index):
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="hr_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "10"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout_s=5.0):
        """Block until nvidia-smi has written its first sample (it takes a
        while to start), so that the timed region that follows is sampled."""
        if self.proc is None:
            return
        t0 = time.time()
        while time.time() - t0 < timeout_s and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

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
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
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


def cpu_baseline(sc, theta, sample=1024, threads=1, keep_estimate=False):
    """The oracle (plain C renders, FP64 sums) on the first `sample`
    perturbations of the same estimate, the renders split over `threads`
    host threads (contiguous slices; the C calls run without the GIL);
    scaled to estimates/s of the full M."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    r = O.RevolveRenderer(sc)
    tau, _ = O.draw(1, 2, sc["sigma"], sample // 2, SEED, 0, 0)
    w = O.weights(1, 2, sc["sigma"], tau)
    t1 = time.perf_counter()

    def part(lo, hi):
        return [r.loss(O.perturb(theta, tau[m])) for m in range(lo, hi)]
    if threads <= 1:
        losses = np.array(part(0, sample))
    else:
        cut = np.linspace(0, sample, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            losses = np.concatenate(list(ex.map(lambda i: np.array(part(cut[i], cut[i + 1])), range(threads))))
    wl_ = w * losses[:, None]
    flat = np.array([math.fsum(wl_[:, e]) for e in range(w.shape[1])]) / sample
    t2 = time.perf_counter()
    per_render = (t2 - t1) / sample
    est_s = per_render * M_PERTURB + (t1 - t0) * M_PERTURB / sample
    out = {"value": 1.0 / est_s, "unit": "estimates/s", "cores": max(1, threads), "kind": "oracle",
           "sample": f"{sample} of the {M_PERTURB} perturbations of one estimate (plain C renders, FP64 sums) "
                     f"on {max(1, threads)} host thread(s), scaled to one full estimate",
           "renders_per_s": 1.0 / per_render}
    if keep_estimate and sample == M_PERTURB:
        # the oracle's own estimate of request 0 (upper triangle) and the sums' scale
        out["_estimate"] = flat
        out["_scale"] = np.array([math.fsum(np.abs(wl_[:, e])) for e in range(w.shape[1])]) / sample
    return out


def oracle_match(hr, S, sc, theta, cb):
    """Error of the GPU estimate of request 0 against the oracle's estimate of
    the same request on the same perturbations: max over the Hessian's unique
    entries of |gpu - oracle| / max(|oracle|, A_e), A_e = 1/(2P) sum |w f|."""
    H = S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], M_PERTURB, hr.HR_AGGREGATE, SEED, 0)
    gpu = H[np.triu_indices(2)]
    ref, scale = cb.pop("_estimate"), cb.pop("_scale")
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), scale)
    return {"max_rel_err": float(rel.max()), "tolerance": 1e-4, "entries": int(rel.size),
            "request": 0, "gpu": gpu.tolist(), "oracle": ref.tolist()}


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2412_03489_gb300 import workloads as wl
    sc = wl.revolve_scene()
    theta = np.asarray(sc["theta_query"], np.float64)
    threads = host_threads()
    # every step is one whole estimate: all M perturbations rendered by the
    # oracle on every host thread, FP64 sums (nothing extrapolated)
    sample = M_PERTURB
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(sc, theta, sample=sample, threads=threads)
        if i >= args.warmup:
            times.append(1.0 / cb["value"])
    est_s = float(np.mean(times))
    val = 1.0 / est_s
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "estimates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sc),
            "cpu_baseline": {"value": val, "unit": "estimates/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: one whole estimate, all {M_PERTURB} perturbations rendered "
                                       f"on {threads} host threads, FP64 sums"},
            "e2e": {"value": val, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def whole_job_rate(local_ms, steps, world, device):
    """Estimates per second of the whole job: every rank runs `steps` independent
    estimates (replicas, no data-path collective); the job takes as long as
    its slowest rank, so the time is the max over ranks.  Returns (rate, max ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
        dist.barrier()
    return world * steps / (local_ms / 1e3), local_ms


def tune_scene(hr, S, theta, n_probe):
    """The library's autotuner on this scene (launch shapes that leave every
    result bit-identical); returns the choice and the probe timings."""
    i = hr.hr_autotune(S.handle, theta, n_probe)
    return {"render_variant": i.render_variant, "sample_threads": i.sample_threads,
            "render_ms": [round(i.render_ms[k], 4) for k in range(i.n_render_variants)],
            "sample_ms": [round(i.sample_ms[k], 4) for k in range(i.n_sample_variants)],
            "probe_perturbations_requested": n_probe}


def _timed_steps(torch, stream, flush, fn, warmup, steps):
    """CUDA-event time of `fn(i)` per step (L2 flushed before each, untimed)."""
    for i in range(warmup):
        flush.fill_(float(i))
        fn(i)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for i in range(steps):
        flush.fill_(float(i))
        ev0.record(stream)
        fn(warmup + i)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    return np.asarray(times)


def run_secondary(args):
    """The other configurations: disc Hessians, path-traced HVPs, batched
    Newton-CG steps, and the serving mix against one-request-at-a-time."""
    import torch
    from paper_2412_03489_gb300 import hr
    from paper_2412_03489_gb300 import workloads as wl
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(0)
    clocks.wait_first()
    line = {"workload": args.workload, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic"}
    if args.workload in ("disc", "ptbox"):
        sc = wl.disc_scene() if args.workload == "disc" else wl.ptbox_scene()
        S = hr.Scene(sc)
        n = sc["n_params"]
        d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
        d_v = torch.tensor(sc.get("v", np.ones(n)), dtype=torch.float64, device="cuda")
        d_out = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        line["tuning"] = tune_scene(hr, S, sc["theta_query"], 2048)
        variants = ([("hessian_elementwise_3x1024", hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 1024, 3 * 1024),
                     ("hessian_aggregate_1024", hr.HR_HESSIAN, hr.HR_AGGREGATE, 1024, 1024)]
                    if args.workload == "disc" else [("hvp_aggregate_8192", hr.HR_HVP, hr.HR_AGGREGATE, 8192, 8192)])
        for name, q, strat, M, renders in variants:
            stage = []

            def fn(i):
                o = hr.make_opts(sc["sigma"], M, strat, SEED, i, stream=stream.cuda_stream)
                hr.hr_estimate_dev(S.handle, q, d_theta.data_ptr(), d_v.data_ptr() if q == hr.HR_HVP else None,
                                   o, d_out.data_ptr())
            # the rate is timed without the library's stage events (they add
            # about 10 us per estimate, a fifth of a small estimate); a second
            # pass with them gives the stage breakdown
            times = []
            for profiled in (False, True):
                hr.hr_profile_enable(S.handle, profiled)
                for i in range(args.warmup + args.steps):
                    flush.fill_(float(i))
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    fn(i)
                    ev1.record(stream)
                    ev1.synchronize()
                    if i >= args.warmup:
                        if profiled:
                            stage.append(hr.hr_profile_last(S.handle).astype(np.float64))
                        else:
                            times.append(ev0.elapsed_time(ev1))
            t = float(np.mean(times))
            line[name] = {"estimates_per_s": 1e3 / t, "renders_per_s": renders * 1e3 / t, "ms_per_estimate": t,
                          "latency_ms": {"p50": float(np.percentile(times, 50)),
                                         "p99": float(np.percentile(times, 99))},
                          "stage_ms": dict(zip(("sample", "render_loss", "sums"),
                                               np.mean(stage, axis=0).tolist()))}
        if args.workload == "disc" and not args.no_queue:
            line["queue"] = disc_queue_bench(torch, hr, wl, stream, flush)
        line["config"] = ({"workload": "disc2d 64x64 gray, r 0.2, 2 params, sigma 0.05"} if args.workload == "disc"
                          else {"workload": "path-traced box 128x128 RGB, 4 spp, depth 3, 6 params, sigma 0.05, "
                                            "aggregate HVP, 8192 perturbations"})
        S.close()
    elif args.workload == "newton":
        sc = wl.tris2d_scene()
        S = hr.Scene(sc)
        B, n = 64, sc["n_params"]
        opts = hr.hr_cg_opts()
        opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 32, 32, 10
        opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base = 1e-3, 0.05, SEED, 0
        opts.use_graph, opts.stream = 1, stream.cuda_stream
        th0 = np.ascontiguousarray(sc["theta_init"], np.float64)
        st = hr.hr_optstate_create(S.handle, B, th0, opts)
        times = _timed_steps(torch, stream, flush, lambda i: hr.hr_newton_cg_step(S.handle, st, None),
                             args.warmup, args.steps)
        info = (hr.hr_step_info * B)()
        hr.hr_newton_cg_step(S.handle, st, info)
        t = float(np.mean(times))
        renders = B * (32 + 10 * 32)
        line.update({"metric": "Newton-CG steps/s (64 instances per launch, CUDA graph)",
                     "instance_steps_per_s": B * 1e3 / t, "launch_steps_per_s": 1e3 / t, "ms_per_step": t,
                     "renders_per_s": renders * 1e3 / t,
                     "mean_cg_iters": float(np.mean([info[b].iters for b in range(B)])),
                     "config": {"workload": "16 coloured triangles 256x256, 64 params, 64 instances, "
                                            "32 gradient + 10 x 32 HVP renders per instance-step, graph-captured"}})
        hr.hr_optstate_destroy(st)
        S.close()
    elif args.workload == "boxes":
        line.update(boxes_variance_bench(hr, wl))
    elif args.workload == "optimise":
        line.update(optimise_bench(torch, hr, wl, stream, args))
    else:
        line.update(serving_bench(torch, hr, wl))
    line["clocks"] = clocks.stop()
    print(json.dumps(line))
    return 0


def optimise_bench(torch, hr, wl, stream, args):
    """The published optimiser (annealed sigma, line search, recompute) on the
    bench mesh scene: 64 instances started around the target, their
    evaluation rate, and the median relative parameter error against device
    time, beside fixed-sigma truncated Newton-CG at the same renders per step."""
    sc = wl.revolve_scene()
    S = hr.Scene(sc)
    B, E, M = 64, 80, 256
    tgt = np.asarray(sc["theta_target"])
    th0 = np.ascontiguousarray(tgt + np.random.default_rng(0xC5).normal(0.0, 0.1, size=(B, 2)), np.float64)
    e0 = np.linalg.norm(th0 - tgt, axis=1)

    def ncg_opts():
        o = hr.hr_ncg_opts()
        for k, v in dict(sigma_start=0.1, sigma_end=0.01, anneal_iters=30, n_grad=M, n_hvp=M, ls_iters=2,
                         ls_tol=1e-3, recompute=1, residual_mode=0, trust_radius=0.02, lambda_rel=0.0, seed=SEED,
                         request_base=0, use_graph=1, stream=stream.cuda_stream).items():
            setattr(o, k, v)
        return o

    def rel_err(th):
        return float(np.median(np.linalg.norm(th - tgt, axis=1) / e0))

    # rate: E - 1 evaluations in one call, device time on the state's stream
    times = []
    for rep in range(args.warmup + max(1, args.steps)):
        st = hr.hr_ncg_create(S.handle, B, th0, ncg_opts())
        hr.hr_ncg_run(S.handle, st, 1)                       # graph capture, untimed
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        hr.hr_ncg_run(S.handle, st, E - 1)
        ev1.record(stream)
        ev1.synchronize()
        if rep >= args.warmup:
            times.append(ev0.elapsed_time(ev1) / (E - 1))
        hr.hr_ncg_destroy(st)
    ms_eval = float(np.median(times))
    # error curve (same seeds, so the same trajectory), read every 4 evaluations
    st = hr.hr_ncg_create(S.handle, B, th0, ncg_opts())
    th = np.zeros_like(th0)
    curve = [[0.0, 1.0]]
    for e in range(0, E, 4):
        hr.hr_ncg_run(S.handle, st, 4)
        hr.hr_ncg_theta(st, th)
        curve.append([round((e + 4) * ms_eval, 3), round(rel_err(th), 4)])
    hr.hr_ncg_destroy(st)
    # truncated Newton-CG at fixed sigma: M gradient + 1 x M HVP renders per step
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = 0.02, M, M, 1
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base = 1e-3, 0.02, SEED, 0
    opts.use_graph, opts.stream = 1, stream.cuda_stream
    nst = hr.hr_optstate_create(S.handle, B, th0, opts)
    hr.hr_newton_cg_step(S.handle, nst, None)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(E):
        hr.hr_newton_cg_step(S.handle, nst, None)
    ev1.record(stream)
    ev1.synchronize()
    ms_step = ev0.elapsed_time(ev1) / E
    hr.hr_optstate_destroy(nst)
    nst = hr.hr_optstate_create(S.handle, B, th0, opts)
    ncurve = [[0.0, 1.0]]
    for k in range(0, E, 4):
        for _ in range(4):
            hr.hr_newton_cg_step(S.handle, nst, None)
        hr.hr_optstate_theta(nst, th)
        ncurve.append([round((k + 4) * ms_step, 3), round(rel_err(th), 4)])
    hr.hr_optstate_destroy(nst)
    S.close()
    return {"metric": "optimiser evaluations/s and median relative parameter error vs device time",
            "evals_per_s": 1e3 / ms_eval, "instance_evals_per_s": B * 1e3 / ms_eval, "ms_per_eval": ms_eval,
            "renders_per_s": B * 2 * M * 1e3 / ms_eval,
            "curve_published": curve, "curve_newton_fixed_sigma": ncurve, "newton_ms_per_step": ms_step,
            "config": {"workload": "mesh 2048 triangles 256x256 RGB, 2 params, 64 instances started at target "
                                   "+ N(0, 0.1^2); published: sigma 0.1 -> 0.01 over 30 iterations, 256 gradient + "
                                   "256 HVP renders per evaluation, line search 2 steps (tol 1e-3), recompute 1, "
                                   "trust 0.02; Newton-CG: sigma 0.02, 256 + 1 x 256 renders per step, trust 0.02",
                       "l2": "not flushed between evaluations (back-to-back optimiser iterations)"}}


def boxes_variance_bench(hr, wl):
    """Box2 / Box10 plateau tasks: Hessian variance per render of element-wise
    IS, aggregate IS and plain Gaussian sampling at equal renders (the paper's
    variance analysis), from 64 independent estimates each, and their rate."""
    out = {"metric": "Hessian variance per render and estimates/s, Box2 / Box10 (squares)"}
    for K in (1, 5):
        sc = wl.boxes_scene(n_boxes=K)
        S = hr.Scene(sc)
        n = 2 * K
        E = n * (n + 1) // 2
        th = np.asarray(sc["theta_target"]) + 0.05
        renders = 3 * 1024 if K == 1 else E * 64
        res = {}
        for name, strat in (("elementwise", hr.HR_ELEMENTWISE), ("aggregate", hr.HR_AGGREGATE),
                            ("plain", hr.HR_PLAIN)):
            M = renders // E if strat == hr.HR_ELEMENTWISE else renders
            M -= M % 2
            ests = []
            t0 = time.perf_counter()
            for rq in range(64):
                H = S.estimate(hr.HR_HESSIAN, th, sc["sigma"], M, strat, 7, rq)
                ests.append(H[np.triu_indices(n)])
            dt = time.perf_counter() - t0
            var = np.var(np.asarray(ests), axis=0, ddof=1)
            res[name] = {"renders_per_estimate": M * (E if strat == hr.HR_ELEMENTWISE else 1),
                         "mean_variance_per_render": float(np.mean(var) * renders),
                         "estimates_per_s": 64 / dt}
        out[f"box{2 * K}"] = res
        S.close()
    return out


def serving_bench(torch, hr, wl, n_requests=1200, sweep=True):
    """Poisson arrivals through the server versus the plain one-request-at-a-
    time entry points on the same request list (estimates of every kind and
    Newton-CG steps on resident optimizer states); with `sweep`, the arrival
    rate swept from a quarter of the saturated rate to past it."""
    import threading
    scenes = wl.serving_scenes()
    S = {k: hr.Scene(v) for k, v in scenes.items()}
    reqs = wl.serving_requests(scenes, n_requests=n_requests)
    specs = wl.serving_newton_states(scenes)

    def new_states():
        out = []
        for sp in specs:
            o = hr.hr_cg_opts()
            o.sigma, o.n_grad, o.n_hvp, o.cg_iters = sp["sigma"], sp["n_grad"], sp["n_hvp"], sp["cg_iters"]
            o.lambda_rel, o.trust_radius, o.seed, o.request_base, o.use_graph = 1e-3, sp["trust_radius"], 3, 0, 1
            out.append(hr.hr_optstate_create(S[sp["scene"]].handle, sp["B"],
                                             np.ascontiguousarray(sp["theta0"], np.float64), o))
        return out

    def out_for(r):
        if r["quantity"] == hr.HR_NEWTON_STEP:
            return (hr.hr_step_info * specs[r["state"]]["B"])()
        n = S[r["scene"]].n
        return np.zeros((n, n) if r["quantity"] == hr.HR_HESSIAN else n)

    def as_array(o):
        if isinstance(o, np.ndarray):
            return o
        return np.array([(x.grad_norm, x.step_norm, x.iters) for x in o])

    def make(r, states):
        if r["quantity"] == hr.HR_NEWTON_STEP:
            return hr.make_request(S[r["scene"]], hr.HR_NEWTON_STEP, optstate=states[r["state"]])
        o = hr.make_opts(r["sigma"], r["M"], r["strategy"], r["seed"], r["request"])
        return hr.make_request(S[r["scene"]], r["quantity"], r["theta"], r["v"], o)

    def plain_one(r, states):
        if r["quantity"] == hr.HR_NEWTON_STEP:
            o = out_for(r)
            hr.hr_newton_cg_step(S[r["scene"]].handle, states[r["state"]], o)
            return as_array(o)
        return S[r["scene"]].estimate(r["quantity"], r["theta"], r["sigma"], r["M"], r["strategy"], r["seed"],
                                      r["request"], v=r["v"])

    # plain: one request at a time through hr_estimate_* / hr_newton_cg_step
    st_plain = new_states()
    for r in reqs[:8]:
        plain_one(r, st_plain)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [plain_one(r, st_plain) for r in reqs]
    plain_s = time.perf_counter() - t0

    srv = hr.hr_server_create(4 << 30, max_active=32, chunk=2048)
    st_srv = new_states()
    for r in reqs[:8]:                                   # warm the lanes (same requests as the plain warm-up)
        req, keep = make(r, st_srv)
        hr.hr_server_wait(srv, hr.hr_server_submit(srv, req), out_for(r), hr.hr_request_info())
    # saturation: everything submitted at once
    t0 = time.perf_counter()
    tk = []
    for r in reqs:
        req, keep = make(r, st_srv)
        tk.append((hr.hr_server_submit(srv, req), keep, r))
    sat = []
    for t, keep, r in tk:
        o = out_for(r)
        hr.hr_server_wait(srv, t, o, hr.hr_request_info())
        sat.append(as_array(o))
    sat_s = time.perf_counter() - t0
    same = all(np.array_equal(a, b) for a, b in zip(plain, sat))
    sat_rate = len(reqs) / sat_s

    def poisson(frac, seed):
        rate = frac * sat_rate
        arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=len(reqs)))
        tickets = [None] * len(reqs)
        ready = threading.Semaphore(0)

        def submitter():
            start = time.perf_counter()
            for i, r in enumerate(reqs):
                d = arrivals[i] - (time.perf_counter() - start)
                if d > 0:
                    time.sleep(d)
                req, keep = make(r, st_srv)
                tickets[i] = (hr.hr_server_submit(srv, req), keep)
                ready.release()
        th = threading.Thread(target=submitter)
        t1 = time.perf_counter()
        th.start()
        lat = []
        for i, r in enumerate(reqs):
            ready.acquire()
            info = hr.hr_request_info()
            hr.hr_server_wait(srv, tickets[i][0], out_for(r), info)
            lat.append(info.done_ms - info.submit_ms)
        th.join()
        dt = time.perf_counter() - t1
        return {"offered_fraction_of_saturated": frac, "arrival_rate_hz": rate,
                "estimates_per_s": len(reqs) / dt,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}}

    sweep = [poisson(f, 0xC5 + k) for k, f in enumerate((0.25, 0.5, 0.7, 0.9, 1.1))] if sweep else []
    hr.hr_server_destroy(srv)
    for st in st_plain + st_srv:
        hr.hr_optstate_destroy(st)
    for v in S.values():
        v.close()
    n_newton = sum(r["quantity"] == hr.HR_NEWTON_STEP for r in reqs)
    return {"metric": "estimates/s and p50/p99 latency, serving mix vs one request at a time",
            "requests": len(reqs), "newton_step_requests": int(n_newton),
            "plain_one_at_a_time": {"estimates_per_s": len(reqs) / plain_s},
            "served_saturated": {"estimates_per_s": sat_rate,
                                 "speedup_vs_plain": plain_s / sat_s, "results_identical_to_plain": same},
            "served_poisson_sweep": sweep,
            "config": {"workload": "Poisson arrivals over 8 resident scenes (disc 64/512, mesh 128/256/512, "
                                   "path-traced box 64, triangles 128 (n 64) / 256 (n 16)), 256..16384 samples, "
                                   "grad / Hessian / HVP, element-wise and aggregate, and Newton-CG steps on 2 "
                                   "resident optimizer states (8 and 4 instances)"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-queue", action="store_true",
                    help="--workload disc: skip the persistent-queue measurement")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the compact path-tracer, Newton-CG and serving measurements of the headline line")
    ap.add_argument("--workload", default="revolve", choices=["revolve", "disc", "ptbox", "newton", "serving", "boxes", "optimise"],
                    help="revolve (default) is the headline workload; the others report the remaining "
                         "configurations in their own JSON lines")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "revolve":
        return run_secondary(args)

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
    tuning = tune_scene(hr, S, theta, 1024)
    compact_slots = int(hr.hr_scene_get_stats(S.handle).mesh_compact_slots)
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
    clocks.wait_first()
    times, render_ms, stage_ms = [], [], []
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
        st = hr.hr_profile_last(S.handle)
        stage_ms.append(st.astype(np.float64))
        render_ms.append(float(st[1]))
    torch.cuda.synchronize()
    clk = clocks.stop()
    value, total_ms = whole_job_rate(float(np.sum(times)), args.steps, world, "cuda")

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
    # whole job, like `value`: all ranks' estimates over the slowest rank's time
    e2e_rate, _ = whole_job_rate((time.perf_counter() - t0) * 1e3, ne, world, "cuda")

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
                "roofline": {"bound": "alu",
                             "kernel": ("revolve_kernel (render + loss; compact layout, two CTAs per SM, "
                                        "then the full layout for renders handed over)") if compact_slots
                             else "revolve_kernel (render + loss)",
                             "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                             "frac": achieved / peak_ops, "traffic": TRAFFIC_BYTES,
                             "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                            f"({src} max SM clock); one FMA = one operation",
                             "ops_per_render": ops, "pixel_triangle_candidates_per_render": cand,
                             "render_ms_per_launch": render_avg_s * 1e3,
                             "issue_slots_busy_ncu": ISSUE_ACTIVE_NCU},
                "e2e": {"value": e2e_rate, "unit": "estimates/s", "h2d_bytes_per_step": 8 + 40,
                        "d2h_bytes_per_step": 32},
                "stage_ms": dict(zip(("sample", "render_loss", "sums"), np.mean(stage_ms, axis=0).tolist())),
                # sampler (also writes theta in FP32), render + loss (with a compact
                # layout: loss words marked free, compact launch, full-layout redo
                # launch), sums
                "gpu_launches": (5 if compact_slots else 3) * args.steps,
                "tuning": tuning,
                "clocks": clk}
        # statistical error of one estimate against a converged reference: the
        # same estimator at 2^20 perturbations (other seed), outside the timed region
        Hc = S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], 1 << 20, hr.HR_AGGREGATE, SEED + 1, 0)
        He = S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], M_PERTURB, hr.HR_AGGREGATE, SEED, 0)
        line["converged_reference"] = {
            "perturbations": 1 << 20, "reference": Hc.tolist(), "estimate": He.tolist(),
            "max_abs_err_over_max_entry": float(np.max(np.abs(He - Hc)) / np.max(np.abs(Hc)))}
        if not args.no_secondary:
            line["secondary"] = secondary_workloads(torch, hr, wl, stream, flush, peaks, n_sm)
        if not args.no_cpu_baseline:
            threads = host_threads()
            line["cpu_baseline"] = cpu_baseline(sc, theta, sample=M_PERTURB, threads=threads, keep_estimate=True)
            line["oracle_match"] = oracle_match(hr, S, sc, theta, line["cpu_baseline"])
            line["cpu_baseline"]["single_thread"] = cpu_baseline(sc, theta, sample=256, threads=1)
            if "secondary" in line:
                line["secondary"]["ptbox_hvp"]["oracle_match"] = ptbox_oracle_match(hr, wl)
        print(json.dumps(line))
    S.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
