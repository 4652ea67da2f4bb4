#!/usr/bin/env python
"""Benchmark: RK4 geodesic steps/s and rays/s on GB300 (FP32-mixed headline, FP64 plain
leg), with the roofline fraction, the end-to-end rate through the host C-ABI call,
and the FP64 CPU oracle timed on the host cores.

Default workload ("mn1000"): Manko-Novikov spacetime M = 0.5, S = 0.24, q = 2, camera
at r0 = 30M, inclination 80 deg, FOV 75 deg, 1000x1000 rays, step_precision 1.5e-4,
at most 20,000 RK4 steps per ray, escape at 1.5 r0.  One benchmark step traces the
whole image.  Under torchrun each rank traces its own camera of an inclination sweep
(theta0 = 80 deg - rank deg): independent problems, no collective on the data path.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2310_15183_gb300 import workloads as W  # noqa: E402

METRIC = "RK4 geodesic steps/s & rays/s on GB300: FP64 plain vs FP32-mixed vs surrogate"
UNIT = "RK4 steps/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
FP64_NOMINAL = 1.25e12  # GB300 dense FP64 (non-tensor) FLOP/s
L2_FLUSH_BYTES = 256 << 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(wl: W.Workload, target_s: float = 12.0, seed: int = 3) -> dict:
    """Time the FP64 oracle, as it stands, on a bounded pixel sample of the workload."""
    import numpy as np

    import oracle
    cam = wl.camera
    threads = os.cpu_count() or 1
    n = max(threads, 16)
    while True:  # grow the sample until it takes a few seconds, then size it to target_s
        pix = W.sample_pixels(cam.n_rays, n, seed)
        t0 = time.perf_counter()
        out = oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                 cam.res_x, cam.res_y, wl.n_steps, wl.step_precision,
                                 pixels=pix, threads=threads)
        dt = time.perf_counter() - t0
        if dt > 2.0 or n >= cam.n_rays:
            break
        n = min(cam.n_rays, int(n * max(2.0, 2.5 / max(dt, 1e-3))))
    if dt < target_s and n < cam.n_rays:
        n = min(cam.n_rays, int(n * target_s / dt))
        pix = W.sample_pixels(cam.n_rays, n, seed)
        t0 = time.perf_counter()
        out = oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                 cam.res_x, cam.res_y, wl.n_steps, wl.step_precision,
                                 pixels=pix, threads=threads)
        dt = time.perf_counter() - t0
    steps = float(np.sum(out["nsteps"].astype(np.float64)))
    return {"steps_per_s": steps / dt, "rays_per_s": n / dt, "seconds": dt, "rays": int(n),
            "steps": steps, "cores": threads,
            "sample": f"{n} seeded pixels of the {cam.res_x}x{cam.res_y} {wl.name} camera, "
                      f"{wl.n_steps} max steps each, {threads} threads"}


def run_reference(args, rank: int, world: int):
    """Reference arm: the CPU oracle on this host's cores (rank 0 only)."""
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_rate(wl, target_s=2.0)
    rates = [oracle_rate(wl, target_s=max(2.0, 60.0 / max(1, args.steps)), seed=100 + k)
             for k in range(args.steps)]
    steps = sum(r["steps"] for r in rates)
    secs = sum(r["seconds"] for r in rates)
    value = steps / secs
    cam = wl.camera
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "M": cam.M, "S": cam.S, "Q": cam.Q, "r0": cam.r0,
                   "theta0_deg": round(cam.theta0 / W.DEG, 6), "fov_deg": cam.fov_deg,
                   "res": [cam.res_x, cam.res_y], "n_steps": wl.n_steps,
                   "step_precision": wl.step_precision, "mode": "oracle-fp64-cpu"},
        "rays_per_s": sum(r["rays"] for r in rates) / secs,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": rates[0]["cores"],
                         "kind": "oracle", "sample": rates[0]["sample"] + " per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mn1000", choices=sorted(W.WORKLOADS))
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-rows", type=int, default=64,
                    help="image rows traced by the FP64 plain leg (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2310_15183_gb300 import build, geotrace

    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = W.WORKLOADS[args.workload]
    cam = wl.camera
    th0 = cam.theta0 - rank * W.DEG if world > 1 else cam.theta0
    mode = geotrace.MODE_FP32_MIXED if args.mode == "mixed" else geotrace.MODE_FP64
    tr = geotrace.Tracer(local)
    stream = tr.stream
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
    n = cam.n_rays
    out = tr.alloc_outputs(n)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        tr.trace(wl.n_steps, wl.step_precision, mode, out)
    barrier()

    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between timed steps (outside the events)
            evs[k][0].record(stream)
            tr.trace(wl.n_steps, wl.step_precision, mode, out)
            evs[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(step_ms) / 1e3
    nsteps = out["nsteps"].cpu().numpy().view(np.uint32).astype(np.float64)
    status = out["status"].cpu().numpy()
    steps_per_pass = float(nsteps.sum())
    if dist is not None:
        tt = torch.tensor([t_dev, steps_per_pass], dtype=torch.float64, device="cuda")
        tmax = tt.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[1:], op=dist.ReduceOp.SUM)
        t_job, steps_job = float(tmax[0]), float(tt[1])
    else:
        t_job, steps_job = t_dev, steps_per_pass
    value = args.steps * steps_job / t_job
    rays_per_s = args.steps * n * world / t_job

    # ---------------- roofline of the dominant kernel (the trace kernel)
    counts = build.op_counts()
    kind = "mn" if cam.Q != 0 else "kerr"
    flops_per_step = counts[f"{kind}_step_flops_mixed" if mode else f"{kind}_step_flops"]
    kernel_s = t_dev / args.steps
    achieved = flops_per_step * steps_per_pass / kernel_s
    if mode == geotrace.MODE_FP32_MIXED:
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6
        peak_note = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"
        measured_peak = geotrace.measure_fma_peak(local, fp64=False)
    else:
        peak = FP64_NOMINAL
        peak_note = "FP64 dense 1.25 TFLOP/s (nominal)"
        measured_peak = geotrace.measure_fma_peak(local, fp64=True, iters=200)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": peak_note, "measured_fma_peak": measured_peak / 1e12,
                "frac_of_measured_fma_peak": achieved / measured_peak,
                "flops_per_rk4_step": flops_per_step,
                "flop_convention": "add/mul 1, fma 2, div/rsqrt/exp 1, sincos 2 (opcount.cpp)"}

    # ---------------- FP64 plain leg on a band of image rows
    modes = {}
    if args.fp64_rows > 0 and mode == geotrace.MODE_FP32_MIXED:
        rows = min(args.fp64_rows, cam.res_y)
        first = (cam.res_y // 2 - rows // 2) * cam.res_x
        cnt = rows * cam.res_x
        o64 = tr.alloc_outputs(cnt)
        tr.trace_range(first, cnt, wl.n_steps, wl.step_precision, geotrace.MODE_FP64, o64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            tr.trace_range(first, cnt, wl.n_steps, wl.step_precision, geotrace.MODE_FP64, o64)
            e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        s64 = float(o64["nsteps"].cpu().numpy().view(np.uint32).astype(np.float64).sum())
        f64 = counts[f"{kind}_step_flops"]
        modes["fp64_plain"] = {
            "steps_per_s": s64 / t64, "rays_per_s": cnt / t64, "seconds": t64,
            "sample": f"{rows} central rows ({cnt} rays) of the same camera",
            "achieved_tflops": f64 * s64 / t64 / 1e12, "frac_of_fp64_nominal": f64 * s64 / t64 / FP64_NOMINAL}
        modes["fp32_mixed"] = {"steps_per_s": value / world, "rays_per_s": rays_per_s / world}
        modes["speedup_mixed_over_fp64"] = (value / world) / (s64 / t64)

    # ---------------- end to end through the host-pointer C-ABI call
    e2e = None
    if not args.no_e2e:
        host = {k: torch.empty(n, dtype=torch.float64, pin_memory=True) for k in ("t", "r", "th", "ph")}
        host["status"] = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        host["nsteps"] = torch.empty(n, dtype=torch.int32, pin_memory=True)
        tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
        tr.trace_host(wl.n_steps, wl.step_precision, mode, host)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            # re-uploading the camera makes each step carry its inputs host -> device
            tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
            tr.trace_host(wl.n_steps, wl.step_precision, mode, host)
        barrier()
        te = time.perf_counter() - t0
        if dist is not None:
            tt = torch.tensor([te], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            te = float(tt[0])
        desc_bytes = 8 * 6 + 8 + 8  # M, S, Q, r0, theta0, fov + res_x, res_y + offset
        e2e = {"value": args.steps * steps_job / te, "unit": UNIT,
               "h2d_bytes_per_step": desc_bytes, "d2h_bytes_per_step": n * (4 * 8 + 4 + 1),
               "rays_per_s": args.steps * n * world / te}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(wl)
        cpu = {"value": r["steps_per_s"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "rays_per_s": r["rays_per_s"], "seconds": r["seconds"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_job / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 zone" if mode else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "M": cam.M, "S": cam.S, "Q": cam.Q, "r0": cam.r0,
                       "theta0_deg": round(cam.theta0 / W.DEG, 6), "fov_deg": cam.fov_deg,
                       "res": [cam.res_x, cam.res_y], "n_steps": wl.n_steps,
                       "step_precision": wl.step_precision,
                       "mode": "fp32_mixed" if mode else "fp64_plain",
                       "parallelism": f"rays sharded by camera, {world} rank(s)",
                       "l2": "flushed between timed steps (256 MiB write, outside the events); "
                             "the kernel reads no input arrays"},
            "rays_per_s": rays_per_s,
            "status_counts": {str(s): int(c) for s, c in zip(*np.unique(status, return_counts=True))},
            "wall_s_timed_region": wall,
            "roofline": roofline, "modes": modes, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clocks, "gpu_launches": args.steps,
        }
        print(json.dumps(line), flush=True)
    tr.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
