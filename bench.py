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
import dataclasses
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

from paper_2310_15183_gb300 import sharding  # noqa: E402
from paper_2310_15183_gb300 import workloads as W  # noqa: E402

METRIC = "RK4 geodesic steps/s & rays/s on GB300: FP64 plain vs FP32-mixed vs surrogate"
UNIT = "RK4 steps/s"
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


# ------------------------------------------------------------------ ncu traffic record
# sources that define the ray-tracing kernels (a traffic record stays valid while they do)
TRACE_SOURCES = ("trace.cu", "spacetime.cuh", "internal.cuh", "camera.cuh", "compensated.cuh",
                 "df.cuh", "zone_df.cuh")


def source_sha1() -> str:
    """Hash of the CUDA sources of the ray-tracing kernels."""
    import hashlib
    h = hashlib.sha1()
    for name in TRACE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2310_15183_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def measured_traffic(kernel: str, rays: int):
    """DRAM bytes per launch of `kernel` scaled from the committed ncu capture record
    (profiles/traffic.json), or None when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha1") != source_sha1():
        return None
    return rec["dram_bytes_per_ray"] * rays


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
            "steps": steps, "cores": threads, "pixels": pix, "out": out,
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


# ------------------------------------------------------------------ extra legs
def _timed(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        r = fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / 1e3


def _steps(out):
    import numpy as np
    return float(out["nsteps"].cpu().numpy().view(np.uint32).astype(np.float64).sum())


def leg_batch(tr, geotrace, args, torch):
    """64 Kerr cameras of uneven size (sides / batch_scale), 500,000-step cap, FP32-mixed:
    autotuned launch shape, one persistent launch replayed from a CUDA graph (FP64 zone
    inline) and the round-based launch for comparison."""
    import dataclasses
    cams = [dataclasses.replace(c, res_x=max(1, c.res_x // args.batch_scale),
                                res_y=max(1, c.res_y // args.batch_scale))
            for c in W.batch_cameras()]
    n = sum(c.n_rays for c in cams)
    rep = cams[0]
    tr.set_spacetime(rep.M, rep.S, rep.Q)
    tr.set_camera(rep.r0, rep.theta0, rep.fov_deg, 256, 256)
    tr.set_options()
    b, k, rpt, v = tr.autotune(geotrace.MODE_FP32_MIXED, trial_rays=1 << 16, trial_steps=300,
                               cache_path=os.path.join(ROOT, "paper_2310_15183_gb300", "_build",
                                                       "autotune.txt"))
    res = {"cameras": len(cams), "rays": n, "n_steps": 500000,
           "sides": [min(c.res_x for c in cams), max(c.res_x for c in cams)],
           "scale": f"camera sides divided by {args.batch_scale}",
           "autotuned": {"block_size": b, "blocks_per_sm": k, "rays_per_thread": rpt,
                         "trial_steps_per_s": v}}
    out = tr.alloc_outputs(n)
    for label, flags in (("graph", geotrace.FLAG_GRAPH), ("rounds", 0)):
        tr.set_options(block_size=b, blocks_per_sm=k, flags=flags, rays_per_thread=rpt)
        tr.trace_batch(cams, 500000, 1.5e-4, geotrace.MODE_FP32_MIXED, out=out)  # warm-up/capture
        _, t = _timed(torch, tr.stream,
                      lambda: tr.trace_batch(cams, 500000, 1.5e-4, geotrace.MODE_FP32_MIXED, out=out))
        st = _steps(out)
        res[label] = {"seconds": t, "steps_per_s": st / t, "rays_per_s": n / t}
    tr.set_options()
    return res


def leg_surrogate(tr, geotrace, args, torch):
    """Surrogate: label sg_samples rays with the integrator (FP32-mixed, 500,000-step cap)
    over the batch ranges at r0 = 30M, train, then image a sg_res^2 Kerr camera (a = 0.9M,
    80 deg) with the gates alone and with integrator probes + fallback; integrator-only
    time from a pixel subsample; accuracy against the FP64 integrator on a 64x64 pixel
    subsample (the network's pixels among them)."""
    import numpy as np
    M, r0, sp, cap = 0.5, 15.0, 1.5e-4, 500000
    host = W.surrogate_samples(args.sg_samples, seed=15183, M=M, r0=r0)
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in host]
    lab, t_label = _timed(torch, tr.stream,
                          lambda: tr.trace_rays(*dev, M, r0, cap, sp, geotrace.MODE_FP32_MIXED))
    labels = [lab["status"], lab["th"], lab["ph"]]
    sg = geotrace.Surrogate(0, r0=r0, seed=7)
    t0 = time.perf_counter()
    losses = sg.train(tr, dev, labels, epochs=args.sg_epochs, batch=args.sg_batch, lr=2e-3,
                      dir_weight=args.sg_dir_weight)
    t_train = time.perf_counter() - t0
    cam = W.Camera(M=M, S=0.9 * M * M, Q=0.0, r0=r0, theta0=80 * W.DEG, fov_deg=75.0,
                   res_x=args.sg_res, res_y=args.sg_res)
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tr.set_options()
    res = {"train_rays": args.sg_samples, "label_seconds": t_label,
           "label_steps_per_s": _steps(lab) / t_label, "train_seconds": t_train,
           "epochs": args.sg_epochs, "batch": args.sg_batch, "dir_weight": args.sg_dir_weight,
           "loss_first_last": [float(losses[0]), float(losses[-1])],
           "image": [cam.res_x, cam.res_y]}
    step = max(1, cam.res_x // 64)
    # judged pixels off the probe lattices (no multiple of 8 or 32 in either coordinate)
    off = step // 2 + 3
    jj, ii = np.meshgrid(np.arange(off, cam.res_y, step), np.arange(off, cam.res_x, step),
                         indexing="ij")
    judge_pix = (jj * cam.res_x + ii).ravel().astype(np.int64)
    judge = tr.trace_pixels(torch.tensor(judge_pix, device="cuda"), cap, sp, geotrace.MODE_FP64)
    torch.cuda.synchronize()
    jd = {k: (v.cpu().numpy().view(np.uint32) if k == "nsteps" else v.cpu().numpy())
          for k, v in judge.items()}
    sub_step = max(1, cam.res_x // 256)
    jj, ii = np.meshgrid(np.arange(sub_step // 2, cam.res_y, sub_step),
                         np.arange(sub_step // 2, cam.res_x, sub_step), indexing="ij")
    sub_pix = torch.tensor((jj * cam.res_x + ii).ravel().astype(np.int64), device="cuda")
    sub, t_sub = _timed(torch, tr.stream,
                        lambda: tr.trace_pixels(sub_pix, cap, sp, geotrace.MODE_FP32_MIXED))
    integ_full_s = t_sub * cam.n_rays / sub_pix.numel()
    mix = tr.trace_pixels(torch.tensor(judge_pix, device="cuda"), cap, sp, geotrace.MODE_FP32_MIXED)
    torch.cuda.synchronize()
    md = {k: v.cpu().numpy() for k, v in mix.items()}

    def angle(a_th, a_ph, b_th, b_ph):
        h = (np.sin((b_th - a_th) / 2) ** 2 +
             np.sin(a_th) * np.sin(b_th) * np.sin((b_ph - a_ph) / 2) ** 2)
        return 2 * np.arcsin(np.sqrt(np.clip(h, 0, 1)))

    def accuracy(got, ref=None):
        ref = jd if ref is None else ref
        same = (got["status"] == 0) == (ref["status"] == 0)
        both = (got["status"] == 0) & (ref["status"] == 0)
        ang = angle(got["th"][both], got["ph"][both], ref["th"][both], ref["ph"][both])
        return {"classification_agreement": float(same.mean()) if same.size else 1.0,
                "angle_err_max": float(ang.max()) if ang.size else 0.0,
                "angle_err_p99": float(np.percentile(ang, 99)) if ang.size else 0.0,
                "angle_err_median": float(np.median(ang)) if ang.size else 0.0}

    res["fp32_mixed_vs_fp64"] = accuracy(md)
    settings = (("tau2_band0.02", dict(tau=2.0, band=0.02)),
                ("tau2_band0.02_dirtol0.005", dict(tau=2.0, band=0.02, dir_tol=0.005)),
                ("probes8_tol1e-3_axis0.02", dict(tau=2.0, band=0.02, axis=0.02, probe_stride=8,
                                                  probe_tol=1e-3)),
                ("probes32_tol1e-3_axis0.02", dict(tau=2.0, band=0.02, axis=0.02,
                                                   probe_stride=32, probe_tol=1e-3)))
    for name, gate in settings:
        out = tr.alloc_outputs(cam.n_rays)
        gate = dict(gate)
        tau, band = gate.pop("tau"), gate.pop("band")
        run = lambda: sg.infer(tr, tau, band, cap, sp, geotrace.MODE_FP32_MIXED, out=out,
                               with_probes=True, **gate)
        (out, nfb, npr), t_inf = _timed(torch, tr.stream, run)
        got = {k: out[k][torch.tensor(judge_pix, device="cuda")].cpu().numpy()
               for k in ("status", "th", "ph", "nsteps")}
        net = got["nsteps"].view(np.uint32) == 0  # judge the network's pixels
        res[name] = {
            "seconds": t_inf, "fallback_pixels": nfb, "probe_pixels": npr,
            "integrated_frac": (nfb + npr) / cam.n_rays,
            "speedup_vs_integrator_only": integ_full_s / t_inf,
            "judged_network_pixels": int(net.sum()),
            **accuracy({k: v[net] for k, v in got.items()},
                       {k: v[net] for k, v in jd.items()})}
    res["integrator_only_seconds_extrapolated"] = integ_full_s
    res["integrator_subsample"] = f"{sub_pix.numel()} pixels (every {sub_step}th in x and y)"
    res["judge"] = f"FP64 integrator on {judge_pix.size} pixels (every {step}th in x and y)"
    sg.close()
    return res


def leg_surrogate_mn(tr, geotrace, args, torch):
    """A surrogate with the Manko-Novikov deviation as a live input: label 2^21 rays with
    q ~ U[-2, 2], a/M ~ U[0.1, 0.99], inclination ~ U[5, 90] deg at r0 = 30M (FP32-mixed,
    500,000-step cap), train, and image the listing's spacetime (q = 2, S = 0.24) at 80 deg,
    1024^2, with integrator probes every 8 pixels (tolerance 1e-3), the axis gate and
    fallback; against integrator-only on the same image (time) and the FP64 integrator on
    4096 of the network's pixels (error)."""
    import numpy as np
    M, r0, sp, cap = 0.5, 15.0, 1.5e-4, 500000
    host = W.surrogate_samples(1 << 21, seed=2310, M=M, r0=r0, q_max=2.0)
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in host]
    lab, t_label = _timed(torch, tr.stream,
                          lambda: tr.trace_rays(*dev, M, r0, cap, sp, geotrace.MODE_FP32_MIXED))
    sg = geotrace.Surrogate(0, r0=r0, seed=9)
    t0 = time.perf_counter()
    losses = sg.train(tr, dev, [lab["status"], lab["th"], lab["ph"]], epochs=80, batch=8192,
                      lr=2e-3, dir_weight=100.0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    cam = W.Camera(M=M, S=0.24, Q=2.0, r0=r0, theta0=80 * W.DEG, fov_deg=75.0, res_x=1024,
                   res_y=1024)
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tr.set_options()
    full, t_full = _timed(torch, tr.stream, lambda: tr.trace(cap, sp, geotrace.MODE_FP32_MIXED))
    out = tr.alloc_outputs(cam.n_rays)
    run = lambda: sg.infer(tr, 2.0, 0.0, cap, sp, geotrace.MODE_FP32_MIXED, out=out,
                           probe_stride=8, probe_tol=1e-3, axis=0.02, with_probes=True)
    (out, nfb, npr), t_inf = _timed(torch, tr.stream, run)
    ns = out["nsteps"].cpu().numpy().view(np.uint32)
    net = np.flatnonzero(ns == 0)
    judge = net[W.sample_pixels(net.size, min(4096, net.size), seed=43)]
    ref = tr.trace_pixels(torch.tensor(judge, device="cuda"), cap, sp, geotrace.MODE_FP64)
    torch.cuda.synchronize()
    ref = {k: (v.cpu().numpy().view(np.uint32) if k == "nsteps" else v.cpu().numpy())
           for k, v in ref.items()}
    acc = accuracy(host_sample(out, judge), ref)
    acc.pop("max_rel_err")
    sg.close()
    # where the integrator's share of the image goes: the integrator-only image's status of
    # the pixels that gated inference integrated, and of all pixels
    fst = full["status"].cpu().numpy()
    ost = out["status"].cpu().numpy()
    counts = lambda a: {str(x): int(y) for x, y in zip(*np.unique(a, return_counts=True))}
    return {"integrated_pixels_status_in_full_image": counts(fst[ns > 0]),
            "full_image_status_counts": counts(fst),
            "network_pixels_status_agreement_with_full_image": float(
                np.mean(ost[net] == fst[net])) if net.size else None,
            "train_rays": 1 << 21, "label_seconds": t_label, "train_seconds": t_train,
            "loss_first_last": [float(losses[0]), float(losses[-1])],
            "label_status_counts": {str(a): int(b) for a, b in zip(
                *np.unique(lab["status"].cpu().numpy(), return_counts=True))},
            "image": "listing's Manko-Novikov (q = 2, S = 0.24), 80 deg, 1024x1024",
            "seconds": t_inf, "integrator_only_seconds": t_full,
            "speedup_vs_integrator_only": t_full / t_inf, "probe_pixels": npr,
            "fallback_pixels": nfb, "network_pixel_fraction": net.size / cam.n_rays,
            "accuracy_vs_fp64": acc}


def leg_gemm(geotrace, args, torch):
    """tcgen05 BF16 GEMM at the surrogate's hidden-layer shape (M = 2^20 rows, N = K = 256,
    bias + SiLU epilogue, bf16 output) and at its weight-gradient shape (M = N = 256,
    K = 2^16, split-K), timed with CUDA events; fraction of the measured bf16 peak."""
    import ctypes
    lib = geotrace.load_library()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    peak = peaks.get("bf16_tflops", 1900.0)
    res = {"peak_tflops": peak, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"}
    g = torch.Generator(device="cuda").manual_seed(1)
    hbm = peaks.get("hbm_gbs", 6800.0)
    res["peak_hbm_gbs"] = hbm
    for name, (M, N, K, splits, bn) in {"forward_hidden": (1 << 20, 256, 256, 1, 128),
                                        "forward_hidden_bn256": (1 << 20, 256, 256, 1, 256),
                                        # the split-precision forward: K' = 3 x 256
                                        "forward_hidden_split_k768": (1 << 20, 256, 768, 1, 256),
                                        "weight_grad": (256, 256, 1 << 16, 128, 128)}.items():
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.zeros(M, N, device="cuda", dtype=torch.float32)
        bias = torch.zeros(N, device="cuda", dtype=torch.float32)
        act = 1 if splits == 1 else 0

        def run():
            if splits > 1:
                C.zero_()
            rc = lib.gt_gemm_bf16(0, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  M, N, K, ctypes.c_void_p(A.data_ptr()), K, 1,
                                  ctypes.c_void_p(B.data_ptr()), K, 1,
                                  ctypes.c_void_p(bias.data_ptr()) if act else None, act,
                                  ctypes.c_void_p(C.data_ptr()), N, int(splits > 1), splits, bn)
            assert rc == 0
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        tf = 2.0 * M * N * K / t / 1e12
        # algorithmic bytes: both operands read once, the FP32 result written once
        # (read as well when split-K accumulates into it)
        nbytes = 2 * (M * K + N * K) + 4 * M * N * (2 if splits > 1 else 1)
        res[name] = {"M": M, "N": N, "K": K, "splits": splits, "bn": bn, "seconds": t,
                     "tflops": tf, "frac_of_peak": tf / peak, "bytes": nbytes,
                     "gbs": nbytes / t / 1e9, "frac_of_hbm": nbytes / t / 1e9 / hbm}
    return res


def leg_sweep(tr, geotrace, args, torch):
    """Inclination sweep at a = 0.9M, 4096^2, step_precision 2e-5, 200,000 steps: frames
    k = 0, 21, 42, 63 of 64 (theta0 = 5 + 85 k/63 deg) on a 256x256 pixel subsample
    (pixels 16m+8), FP64 plain vs FP32-mixed; the FP64 CPU oracle judges a 16x16 subset of
    it (pixels 256m+136) of each frame."""
    import numpy as np

    import oracle
    res, frames = {}, (0, 21, 42, 63)
    jj, ii = np.meshgrid(np.arange(8, 4096, 16), np.arange(8, 4096, 16), indexing="ij")
    pix = (jj * 4096 + ii).ravel().astype(np.int64)
    dpix = torch.tensor(pix, device="cuda")
    oj, oi = np.meshgrid(np.arange(136, 4096, 256), np.arange(136, 4096, 256), indexing="ij")
    opix = (oj * 4096 + oi).ravel().astype(np.int64)
    sel = np.searchsorted(pix, opix)
    assert np.array_equal(pix[sel], opix)
    for k in frames:
        th0 = (5 + 85 * k / 63) * W.DEG
        tr.set_spacetime(0.5, 0.9 * 0.25, 0.0)
        tr.set_camera(15.0, th0, 75.0, 4096, 4096)
        tr.set_options()
        f = {}
        for name, mode in (("fp64", geotrace.MODE_FP64), ("fp32_mixed", geotrace.MODE_FP32_MIXED)):
            out, t = _timed(torch, tr.stream,
                            lambda: tr.trace_pixels(dpix, 200000, 2e-5, mode))
            o = {kk: (v.cpu().numpy().view(np.uint32) if kk == "nsteps" else v.cpu().numpy())
                 for kk, v in out.items()}
            f[name] = {"seconds": t, "steps_per_s": float(o["nsteps"].astype(float).sum()) / t,
                       "out": o}
        ref = oracle.trace_image(0.5, 0.225, 0.0, 15.0, th0, 75.0, 4096, 4096, 200000, 2e-5,
                                 pixels=opix)
        for name in ("fp64", "fp32_mixed"):
            o = f[name].pop("out")
            err = max(float(np.max(np.abs(o[kk][sel] - ref[kk]) / np.maximum(1, np.abs(ref[kk]))))
                      for kk in ("t", "r", "th", "ph"))
            f[name]["max_rel_err_vs_oracle"] = err
            f[name]["status_equal"] = bool(np.array_equal(o["status"][sel], ref["status"]))
        res[f"frame{k}"] = f
    res["subsample"] = "256x256 pixels (16m+8) of 4096x4096; oracle on 16x16 (256m+136)"
    return res


def leg_paper(tr, geotrace, args, torch):
    """The paper's own method on GB300: the listing's numerics (forward-difference metric
    derivatives, float32 I/O, 0.1667 weights, v^phi = alpha; FP64 arithmetic) on the
    listing's camera (r0 = 16M, theta0 = pi/2, FOV 75 deg, 1000x1000) at its 500,000-step
    cap, Kerr (S = 0.24, Q = 0) and the listing's Manko-Novikov (q = 2), on a seeded pixel
    sample, seconds per megapixel extrapolated; beside this build's exact FP64 and
    FP32-mixed paths on the same pixels.  The paper quotes ~300 s (Kerr) and 1,200-3,000 s
    (Manko-Novikov) per megapixel on its GPU."""
    import numpy as np
    res = {}
    for name, (S, Q, n_pix) in {"kerr": (0.24, 0.0, 65536), "mn": (0.24, 2.0, 16384)}.items():
        cam = W.Camera(M=0.5, S=S, Q=Q, r0=8.0, theta0=math.pi / 2, fov_deg=75.0,
                       res_x=1000, res_y=1000)
        pix = torch.tensor(W.sample_pixels(cam.n_rays, n_pix, seed=51), device="cuda")
        tr.set_spacetime(cam.M, cam.S, cam.Q)
        tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
        r = {"sample_pixels": n_pix}
        for label, flags, mode in (("paper_numerics_fp64", geotrace.FLAGS_PAPER, geotrace.MODE_FP64),
                                   ("exact_fp64", 0, geotrace.MODE_FP64),
                                   ("exact_fp32_mixed", 0, geotrace.MODE_FP32_MIXED)):
            tr.set_options(flags=flags)
            out, t = _timed(torch, tr.stream, lambda: tr.trace_pixels(pix, 500000, 1.5e-4, mode))
            st = _steps(out)
            r[label] = {"seconds": t, "seconds_per_mpx": t * 1e6 / n_pix, "steps_per_s": st / t}
        res[name] = r
    tr.set_options()
    res["paper_seconds_per_mpx"] = {"kerr": 300, "mn": [1200, 3000],
                                    "hardware": "unnamed 2016 consumer GPU (paper, Sec. 4)"}
    return res


def leg_mn_sweep(tr, geotrace, args, torch):
    """Inclination sweep of the listing's Manko-Novikov spacetime (q = 2, S = 0.24, r0 =
    30M, FOV 75 deg) at the 500,000-step cap, frames theta0 = 5, 35, 62, 90 deg, whole
    1000x1000 images, FP32-mixed; status counts, the zone's share of the steps and the
    share of its field evaluations done in FP64.
    (Small pixel samples are timed by the few trapped rays that run the whole cap one after
    another, not by throughput, so whole images are traced.)"""
    import numpy as np
    res = {}
    for th_deg in (5.0, 35.0, 62.0, 90.0):
        tr.set_spacetime(0.5, 0.24, 2.0)
        tr.set_camera(15.0, th_deg * W.DEG, 75.0, 1000, 1000)
        tr.set_options()
        out, t = _timed(torch, tr.stream,
                        lambda: tr.trace(500000, 1.5e-4, geotrace.MODE_FP32_MIXED))
        zone, zone_f64 = tr.zone_stats()
        steps = _steps(out)
        st = out["status"].cpu().numpy()
        res[f"theta0_{th_deg:g}"] = {
            "seconds": t, "steps_per_s": steps / t, "seconds_per_mpx": t,
            "status_counts": {str(a): int(b) for a, b in zip(*np.unique(st, return_counts=True))},
            "zone_step_fraction": zone / steps,
            "zone_f64_eval_fraction": zone_f64 / (4 * zone) if zone else 0.0}
    return res


def leg_zone(tr, geotrace, args, torch):
    """The listing's Manko-Novikov image (1000x1000, 500,000-step cap, FP32-mixed) with the
    zone's field in double-float (the default) and in FP64 (GT_FLAG_ZONE_FP64): the time of
    each whole image, the zone statistics, and the agreement of the two images (status of
    every pixel; end angle of the pixels both call escaped), with both against the FP64
    integrator on 256 seeded pixels that are not trapped (the trapped rays' end states at
    the cap are chaotic); and the Kerr a = 0.9M image at the cap without a zone (the
    default) and with a double-float zone at r < 4M."""
    import numpy as np
    cam = W.MN_1000
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    res, outs = {}, {}
    for name, flags in (("double_float", 0), ("fp64", geotrace.FLAG_ZONE_FP64)):
        tr.set_options(flags=flags)
        out, t = _timed(torch, tr.stream,
                        lambda: tr.trace(500000, 1.5e-4, geotrace.MODE_FP32_MIXED))
        zone, f64 = tr.zone_stats()
        steps = _steps(out)
        outs[name] = host_sample(out, slice(None))
        st = outs[name]["status"]
        res[name] = {"seconds": t, "steps_per_s": steps / t,
                     "status_counts": {str(a): int(b) for a, b in
                                       zip(*np.unique(st, return_counts=True))},
                     "zone_step_fraction": zone / steps,
                     "zone_f64_eval_fraction": f64 / (4 * zone) if zone else 0.0}
    tr.set_options()
    res["double_float_vs_fp64_zone"] = accuracy(outs["double_float"], outs["fp64"])
    res["speedup"] = res["fp64"]["seconds"] / res["double_float"]["seconds"]
    st = outs["fp64"]["status"]
    cand = np.flatnonzero(st != 2)
    pix = cand[W.sample_pixels(cand.size, 256, seed=77)]
    ref = tr.trace_pixels(torch.tensor(pix, device="cuda"), 500000, 1.5e-4,
                          geotrace.MODE_FP64)
    ref = host_sample(ref, slice(None))
    for name in ("double_float", "fp64"):
        acc = accuracy({k: v[pix] for k, v in outs[name].items()}, ref)
        res[name]["vs_fp64_integrator_256_untrapped_pixels"] = acc
    # Kerr a = 0.9M, 80 deg, 1000x1000 at the cap: no zone (the default) against a
    # double-float zone over the horizon approach and the photon region (r < 4M)
    kerr = W.Camera(M=0.5, S=0.9 * 0.25, Q=0.0, r0=15.0, theta0=80 * W.DEG, fov_deg=75.0,
                    res_x=1000, res_y=1000)
    tr.set_spacetime(kerr.M, kerr.S, kerr.Q)
    tr.set_camera(kerr.r0, kerr.theta0, kerr.fov_deg, kerr.res_x, kerr.res_y)
    kres, kouts = {}, {}
    for name, r_sw in (("no_zone", 0.0), ("double_float_zone_4M", 4 * kerr.M)):
        tr.set_options(r_switch=r_sw)
        out, t = _timed(torch, tr.stream,
                        lambda: tr.trace(500000, 1.5e-4, geotrace.MODE_FP32_MIXED))
        zone, f64 = tr.zone_stats()
        steps = _steps(out)
        kouts[name] = host_sample(out, slice(None))
        kres[name] = {"seconds": t, "steps_per_s": steps / t, "zone_step_fraction": zone / steps,
                      "zone_f64_eval_fraction": f64 / (4 * zone) if zone else 0.0}
    tr.set_options()
    kres["zone_vs_no_zone"] = accuracy(kouts["double_float_zone_4M"], kouts["no_zone"])
    kres["cost"] = kres["double_float_zone_4M"]["seconds"] / kres["no_zone"]["seconds"]
    res["kerr1000_T"] = kres
    return res


# ------------------------------------------------------------------ accuracy and extra modes
def great_circle(th1, ph1, th2, ph2):
    import numpy as np
    a = np.sin((th2 - th1) / 2) ** 2 + np.sin(th1) * np.sin(th2) * np.sin((ph2 - ph1) / 2) ** 2
    return 2 * np.arcsin(np.sqrt(np.clip(a, 0, 1)))


def accuracy(got: dict, ref: dict) -> dict:
    """Error of a GPU result against the FP64 oracle (or the FP64 GPU path) on the same
    rays: classification agreement, end-angle error of rays both call escaped, and the
    largest relative error of t, r, theta, phi on rays of equal status."""
    import numpy as np
    same = got["status"] == ref["status"]
    esc = same & (ref["status"] == 0)
    ang = great_circle(got["th"][esc], got["ph"][esc], ref["th"][esc], ref["ph"][esc])
    rel = 0.0
    for k in ("t", "r", "th", "ph"):
        if k in got and k in ref and same.any():
            e = np.abs(got[k][same] - ref[k][same]) / np.maximum(1.0, np.abs(ref[k][same]))
            rel = max(rel, float(np.nanmax(e)))
    return {"rays": int(ref["status"].size), "classification_agreement": float(same.mean()),
            "angle_err_max": float(ang.max()) if ang.size else 0.0,
            "angle_err_median": float(np.median(ang)) if ang.size else 0.0,
            "max_rel_err": rel}


def host_sample(out: dict, idx) -> dict:
    import numpy as np
    res = {}
    for k, v in out.items():
        a = v.cpu().numpy()
        if k == "nsteps":
            a = a.view(np.uint32)
        res[k] = a[idx]
    return res


def oracle_sample(cam, n_steps, sp, pixels) -> dict:
    """The FP64 CPU oracle on listed pixels (a CPU-baseline sample; also the reference the
    GPU results of that sample are judged against)."""
    import oracle
    return oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg, cam.res_x,
                              cam.res_y, n_steps, sp, pixels=pixels)


def mode_terminating(tr, geotrace, torch) -> dict:
    """The paper's terminating workloads at the listing's 500,000-step cap, FP32-mixed, as
    whole 1000x1000 images: Kerr a = 0.9M and the listing's Manko-Novikov spacetime (whose
    trapped rays run in the zone); each with its error against the FP64 oracle on a
    pixel sample (that sample's CPU baseline) and the share of steps taken in the zone."""
    import numpy as np
    res = {}
    cap, sp = 500000, 1.5e-4
    kerr = W.Camera(M=0.5, S=0.9 * 0.25, Q=0.0, r0=15.0, theta0=80 * W.DEG, fov_deg=75.0,
                    res_x=1000, res_y=1000)
    cases = (("kerr1000_T", kerr, None, 32), ("mn1000_T", W.MN_1000, None, 16))
    for name, cam, n_sample, n_judge in cases:
        tr.set_spacetime(cam.M, cam.S, cam.Q)
        tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
        tr.set_options()
        if n_sample is None:
            pix = None
            run = lambda: tr.trace(cap, sp, geotrace.MODE_FP32_MIXED)
            n = cam.n_rays
        else:
            pix = W.sample_pixels(cam.n_rays, n_sample, seed=31)
            dpix = torch.tensor(pix, device="cuda")
            run = lambda: tr.trace_pixels(dpix, cap, sp, geotrace.MODE_FP32_MIXED)
            n = n_sample
        out, t = _timed(torch, tr.stream, run)
        zone, zone_f64 = tr.zone_stats()
        steps = _steps(out)
        st = out["status"].cpu().numpy()
        judge = W.sample_pixels(n, n_judge, seed=32)
        got = host_sample(out, judge)
        t0 = time.perf_counter()
        ref = oracle_sample(cam, cap, sp, judge if pix is None else pix[judge])
        t_cpu = time.perf_counter() - t0
        res[name] = {
            "rays": n, "seconds": t, "steps_per_s": steps / t, "rays_per_s": n / t,
            "seconds_per_mpx": t * 1e6 / n, "mean_steps_per_ray": steps / n,
            "status_counts": {str(a): int(b) for a, b in zip(*np.unique(st, return_counts=True))},
            "zone_step_fraction": zone / steps if steps else 0.0,
            "zone_f64_eval_fraction": zone_f64 / (4 * zone) if zone else 0.0,
            "sample": "whole image" if pix is None else f"{n} seeded pixels of 1000x1000",
            "accuracy_vs_oracle": accuracy(got, ref),
            "cpu_baseline": {"value": float(ref["nsteps"].astype(np.float64).sum()) / t_cpu,
                             "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": f"{n_judge} seeded pixels of the GPU sample",
                             "seconds": t_cpu},
            "paper_seconds_per_mpx": 300 if name.startswith("kerr") else [1200, 3000]}
        if name.startswith("kerr"):
            # the same image with a double-float zone over the horizon approach and the
            # photon region (r < 4M; Kerr runs without one by default)
            tr.set_options(r_switch=4 * cam.M)
            out_z, t_z = _timed(torch, tr.stream, run)
            zone_z, _ = tr.zone_stats()
            tr.set_options()
            steps_z = _steps(out_z)
            host_z = host_sample(out_z, slice(None))
            host_0 = host_sample(out, slice(None))
            res[name]["with_double_float_zone_4M"] = {
                "seconds": t_z, "cost": t_z / t, "zone_step_fraction": zone_z / steps_z,
                "vs_no_zone_whole_image": accuracy(host_z, host_0),
                "accuracy_vs_oracle": accuracy(host_sample(out_z, judge), ref)}
    return res


def mode_surrogate(tr, geotrace, torch, args) -> dict:
    """Surrogate + fallback at a reduced training budget: label sg_default_rays rays with the
    integrator (FP32-mixed, 500,000-step cap) over the training ranges at r0 = 30M, train,
    then image a Kerr a = 0.9M, 80 deg camera of sg_default_res^2 pixels with integrator
    probes every 8 pixels (tolerance 1e-3), the photon-ring and axis gates (0.02) and
    fallback; against integrator-only on the same
    image (time) and the FP64 integrator on a pixel sample of the network's pixels (error)."""
    import numpy as np
    M, r0, sp, cap = 0.5, 15.0, 1.5e-4, 500000
    host = W.surrogate_samples(args.sg_default_rays, seed=15183, M=M, r0=r0)
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in host]
    lab, t_label = _timed(torch, tr.stream,
                          lambda: tr.trace_rays(*dev, M, r0, cap, sp, geotrace.MODE_FP32_MIXED))
    sg = geotrace.Surrogate(0, r0=r0, seed=7)
    t0 = time.perf_counter()
    losses = sg.train(tr, dev, [lab["status"], lab["th"], lab["ph"]],
                      epochs=args.sg_default_epochs, batch=8192, lr=2e-3, dir_weight=100.0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res_ = args.sg_default_res
    cam = W.Camera(M=M, S=0.9 * M * M, Q=0.0, r0=r0, theta0=80 * W.DEG, fov_deg=75.0,
                   res_x=res_, res_y=res_)
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tr.set_options()
    full = tr.trace(cap, sp, geotrace.MODE_FP32_MIXED)  # warm
    full, t_full = _timed(torch, tr.stream, lambda: tr.trace(cap, sp, geotrace.MODE_FP32_MIXED))
    out = tr.alloc_outputs(cam.n_rays)
    infer = lambda: sg.infer(tr, 2.0, 0.02, cap, sp, geotrace.MODE_FP32_MIXED, out=out,
                             probe_stride=8, probe_tol=1e-3, axis=0.02, with_probes=True)
    infer()
    (out, nfb, npr), t_inf = _timed(torch, tr.stream, infer)
    ns = out["nsteps"].cpu().numpy().view(np.uint32)
    net = np.flatnonzero(ns == 0)
    judge = net[W.sample_pixels(net.size, min(4096, net.size), seed=41)]
    ref = tr.trace_pixels(torch.tensor(judge, device="cuda"), cap, sp, geotrace.MODE_FP64)
    torch.cuda.synchronize()
    ref = {k: (v.cpu().numpy().view(np.uint32) if k == "nsteps" else v.cpu().numpy())
           for k, v in ref.items()}
    got = host_sample(out, judge)
    acc = accuracy(got, ref)
    acc.pop("max_rel_err")  # network pixels carry no t, r
    # the network alone (no probes, no fallback gates) on the same judged pixels
    raw = tr.alloc_outputs(cam.n_rays)
    sg.infer(tr, 0.0, 0.0, cap, sp, geotrace.MODE_FP32_MIXED, out=raw)
    acc_raw = accuracy(host_sample(raw, judge), ref)
    acc_raw.pop("max_rel_err")
    sg.close()
    return {"train_rays": args.sg_default_rays, "epochs": args.sg_default_epochs,
            "label_seconds": t_label, "train_seconds": t_train,
            "loss_first_last": [float(losses[0]), float(losses[-1])],
            "image": [cam.res_x, cam.res_y], "seconds": t_inf,
            "rays_per_s": cam.n_rays / t_inf,
            "integrator_only_seconds": t_full, "speedup_vs_integrator_only": t_full / t_inf,
            "probe_pixels": npr, "fallback_pixels": nfb,
            "network_pixel_fraction": net.size / cam.n_rays,
            "gates": {"tau": 2.0, "band": 0.02, "axis": 0.02, "probe_stride": 8,
                      "probe_tol": 1e-3},
            "accuracy_vs_fp64": acc, "network_alone_vs_fp64": acc_raw,
            "judge": f"FP64 integrator on {judge.size} seeded network pixels"}


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mn1000", choices=sorted(W.WORKLOADS))
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-rows", type=int, default=-1,
                    help="image rows traced by the FP64 plain leg (-1 = the whole image, 0 = skip)")
    ap.add_argument("--no-terminating", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--sg-default-rays", type=int, default=1 << 21)
    ap.add_argument("--sg-default-epochs", type=int, default=80)
    ap.add_argument("--sg-default-res", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="",
                    help="extra legs: batch,surrogate,surrogate_mn,sweep,gemm,paper,mn_sweep,zone "
                         "(comma list)")
    ap.add_argument("--sg-samples", type=int, default=1 << 22)
    ap.add_argument("--sg-epochs", type=int, default=120)
    ap.add_argument("--sg-batch", type=int, default=8192)
    ap.add_argument("--sg-dir-weight", type=float, default=100.0)
    ap.add_argument("--sg-res", type=int, default=4096)
    ap.add_argument("--batch-scale", type=int, default=8,
                    help="batch leg: camera sides divided by this factor")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default launch shape instead of the autotuner's")
    ap.add_argument("--rays-per-thread", type=int, default=0,
                    help="with --no-autotune: FP32 rays per thread (1 or 2)")
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
    th0 = sharding.sweep_camera(cam, rank, world).theta0
    mode = geotrace.MODE_FP32_MIXED if args.mode == "mixed" else geotrace.MODE_FP64
    tr = geotrace.Tracer(local)
    stream = tr.stream
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
    n = cam.n_rays
    out = tr.alloc_outputs(n)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # launch shape from the autotuner (block size x resident blocks x rays per thread),
    # timed on a central pixel range of this camera before the warm-up
    launch = {"block_size": 128, "blocks_per_sm": 4, "rays_per_thread": 1, "autotuned": False}
    if not args.no_autotune:
        tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
        b, k, rpt, v = tr.autotune(mode, trial_rays=1 << 18, trial_steps=300,
                                   step_precision=wl.step_precision)
        launch = {"block_size": b, "blocks_per_sm": k, "rays_per_thread": rpt, "autotuned": True,
                  "trial_steps_per_s": v}
    if args.no_autotune and args.rays_per_thread:
        launch["rays_per_thread"] = args.rays_per_thread
        if args.rays_per_thread == 2:
            launch["blocks_per_sm"] = 3
    opts = {k: launch[k] for k in ("block_size", "blocks_per_sm", "rays_per_thread")}
    tr.set_options(**opts)

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
        t_job, steps_job = sharding.reduce_timing(dist, t_dev, steps_per_pass, device="cuda")
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
        sms = tr.sm_count()
        peak = sms * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6
        peak_note = f"FP32 FMA: {sms} SMs x 128 lanes x 2 flop x 2070 MHz (derived)"
        measured_peak = geotrace.measure_fma_peak(local, fp64=False)
    else:
        peak = FP64_NOMINAL
        peak_note = "FP64 dense 1.25 TFLOP/s (nominal)"
        measured_peak = geotrace.measure_fma_peak(local, fp64=True, iters=200)
    kname = f"trace_kernel<{2 if mode else 0},{1 if cam.Q != 0 else 0},0>"
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": measured_traffic(kname, n), "kernel": kname,
                "peak_source": peak_note, "measured_fma_peak": measured_peak / 1e12,
                "frac_of_measured_fma_peak": achieved / measured_peak,
                "flops_per_rk4_step": flops_per_step,
                "flop_convention": "add/mul 1, fma 2, div/rsqrt/exp 1, sincos 2 (opcount.cpp)"}

    # ---------------- the CPU oracle on a bounded sample (rank 0, N = 1): the CPU baseline,
    # and the FP64 reference every GPU result of this workload is judged against
    cpu, acc_pix, acc_ref = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(wl)
        cpu = {"value": r["steps_per_s"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "rays_per_s": r["rays_per_s"], "seconds": r["seconds"]}
        acc_pix, acc_ref = r["pixels"], r["out"]
    modes = {}
    if acc_ref is not None:
        modes["fp32_mixed"] = {"accuracy_vs_oracle": accuracy(host_sample(out, acc_pix), acc_ref)}

    # ---------------- FP64 plain leg (the whole image unless --fp64-rows limits it)
    if args.fp64_rows != 0 and mode == geotrace.MODE_FP32_MIXED:
        rows = cam.res_y if args.fp64_rows < 0 else min(args.fp64_rows, cam.res_y)
        first = (cam.res_y // 2 - rows // 2) * cam.res_x
        cnt = rows * cam.res_x
        o64 = tr.alloc_outputs(cnt)
        tr.set_options()  # the FP64 kernel at its default shape
        tr.trace_range(first + (rows // 2) * cam.res_x, cam.res_x, wl.n_steps, wl.step_precision,
                       geotrace.MODE_FP64, o64)  # warm-up: one row
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
            "sample": "the whole image" if rows == cam.res_y else
                      f"{rows} central rows ({cnt} rays) of the same camera",
            "achieved_tflops": f64 * s64 / t64 / 1e12, "frac_of_fp64_nominal": f64 * s64 / t64 / FP64_NOMINAL,
            "flops_per_rk4_step": f64}
        if acc_ref is not None and rows == cam.res_y:
            modes["fp64_plain"]["accuracy_vs_oracle"] = accuracy(host_sample(o64, acc_pix), acc_ref)
        modes.setdefault("fp32_mixed", {}).update(
            {"steps_per_s": value / world, "rays_per_s": rays_per_s / world})
        modes["speedup_mixed_over_fp64"] = (value / world) / (s64 / t64)

    # ---------------- the paper's terminating workloads and the surrogate (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_terminating:
        t0 = time.perf_counter()
        modes["terminating"] = mode_terminating(tr, geotrace, torch)
        modes["terminating"]["wall_s"] = time.perf_counter() - t0
    if rank == 0 and world == 1 and not args.no_surrogate:
        t0 = time.perf_counter()
        modes["surrogate"] = mode_surrogate(tr, geotrace, torch, args)
        modes["surrogate"]["wall_s"] = time.perf_counter() - t0
    tr.set_spacetime(cam.M, cam.S, cam.Q)
    tr.set_camera(cam.r0, th0, cam.fov_deg, cam.res_x, cam.res_y)
    tr.set_options(**opts)

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


    legs = {}
    for leg in [x for x in args.legs.split(",") if x]:
        t0 = time.perf_counter()
        if leg == "batch":
            legs["batch"] = leg_batch(tr, geotrace, args, torch)
        elif leg == "surrogate":
            legs["surrogate"] = leg_surrogate(tr, geotrace, args, torch)
        elif leg == "sweep":
            legs["sweep"] = leg_sweep(tr, geotrace, args, torch)
        elif leg == "gemm":
            legs["gemm"] = leg_gemm(geotrace, args, torch)
        elif leg == "paper":
            legs["paper"] = leg_paper(tr, geotrace, args, torch)
        elif leg == "mn_sweep":
            legs["mn_sweep"] = leg_mn_sweep(tr, geotrace, args, torch)
        elif leg == "zone":
            legs["zone"] = leg_zone(tr, geotrace, args, torch)
        elif leg == "surrogate_mn":
            legs["surrogate_mn"] = leg_surrogate_mn(tr, geotrace, args, torch)
        else:
            raise SystemExit(f"unknown leg {leg}")
        legs[leg]["leg_wall_s"] = time.perf_counter() - t0
        log(f"leg {leg}: {legs[leg]}")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_job / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64/df zone" if mode else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "M": cam.M, "S": cam.S, "Q": cam.Q, "r0": cam.r0,
                       "theta0_deg": round(cam.theta0 / W.DEG, 6), "fov_deg": cam.fov_deg,
                       "res": [cam.res_x, cam.res_y], "n_steps": wl.n_steps,
                       "step_precision": wl.step_precision,
                       "mode": "fp32_mixed" if mode else "fp64_plain",
                       "parallelism": f"rays sharded by camera, {world} rank(s)",
                       "launch": launch,
                       "l2": "flushed between timed steps (256 MiB write, outside the events); "
                             "the kernel reads no input arrays"},
            "rays_per_s": rays_per_s,
            "status_counts": {str(s): int(c) for s, c in zip(*np.unique(status, return_counts=True))},
            "wall_s_timed_region": wall,
            "accuracy_vs_oracle": modes.get("fp32_mixed", {}).get("accuracy_vs_oracle"),
            "roofline": roofline, "modes": modes, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clocks, "gpu_launches": args.steps,
        }
        if legs:
            line["legs"] = legs
        print(json.dumps(line), flush=True)
    tr.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
