"""Thin Python binding of libgeotrace.so (include/geotrace.h) -- argument marshalling only.

PyTorch supplies device memory and the CUDA stream; every step of the ray tracing
runs in the library's CUDA kernels.  The binding never falls back to any other
implementation: if the compiled library is missing or the device is not sm_103 it
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeotrace.so")

GT_OK = 0
ERRORS = {-1: "invalid argument", -2: "not configured", -3: "CUDA error", -4: "out of memory",
          -5: "device watchdog timeout", -6: "unsupported device or feature"}
ESCAPED, HORIZON, MAXSTEPS, NONFINITE, TIMEOUT, DISK = 0, 1, 2, 3, 4, 5
MODE_FP64, MODE_FP32_MIXED = 0, 1
FLAG_COMPAT_WEIGHTS, FLAG_COMPAT_CAMERA, FLAG_ONE_SHOT, FLAG_GRAPH, FLAG_PRECISE_MN = 1, 2, 4, 8, 16
FLAG_FD_DERIVS, FLAG_F32_IO, FLAG_EULER, FLAG_ZONE_FP64 = 32, 64, 128, 256
# the listing's numerics: forward differences, float32 I/O, 0.1667 weights, v^phi = alpha
FLAGS_PAPER = FLAG_FD_DERIVS | FLAG_F32_IO | FLAG_COMPAT_WEIGHTS | FLAG_COMPAT_CAMERA

# every symbol include/geotrace.h declares
EXPORTS = ("gt_create", "gt_destroy", "gt_set_stream", "gt_set_spacetime", "gt_set_camera",
           "gt_set_options", "gt_trace", "gt_trace_range", "gt_trace_pixels", "gt_trace_host", "gt_trace_batch", "gt_sync",
           "gt_device_sm_count", "gt_measure_fma_peak", "gt_gemm_bf16", "gt_trace_batch_noalloc",
           "gt_trace_rays", "gt_autotune", "gt_surrogate_num_params", "gt_surrogate_create",
           "gt_surrogate_destroy", "gt_surrogate_get_params", "gt_surrogate_set_params",
           "gt_surrogate_eval", "gt_surrogate_grad", "gt_surrogate_train", "gt_surrogate_infer",
           "gt_trace_disk", "gt_trace_states", "gt_surrogate_get_grads", "gt_get_stats",
           "gt_strerror")


class GeotraceError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERRORS.get(code, 'error')} (code {code})")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("flags", ctypes.c_int), ("reproject_every", ctypes.c_int),
                ("r_switch", ctypes.c_double), ("timeout_seconds", ctypes.c_double),
                ("rays_per_thread", ctypes.c_int)]


class SurrogateNorm(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_double), ("fov_deg", ctypes.c_double),
                ("spin_max", ctypes.c_double), ("q_max", ctypes.c_double),
                ("theta0_min", ctypes.c_double), ("theta0_max", ctypes.c_double)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("dir_weight", ctypes.c_double)]


class GateCfg(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("band", ctypes.c_double), ("axis", ctypes.c_double),
                ("dir_tol", ctypes.c_float), ("probe_stride", ctypes.c_int),
                ("probe_tol", ctypes.c_float)]


class CameraDesc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double), ("S", ctypes.c_double), ("Q", ctypes.c_double),
                ("r0", ctypes.c_double), ("theta0", ctypes.c_double),
                ("fov_deg", ctypes.c_double), ("res_x", ctypes.c_int32),
                ("res_y", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgeotrace.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libgeotrace.so is not built; run paper_2310_15183_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.gt_create.argtypes = [ctypes.POINTER(vp), i, vp]
    lib.gt_destroy.argtypes = [vp]
    lib.gt_set_stream.argtypes = [vp, vp]
    lib.gt_set_spacetime.argtypes = [vp, d, d, d]
    lib.gt_set_camera.argtypes = [vp, d, d, d, i, i]
    lib.gt_set_options.argtypes = [vp, ctypes.POINTER(Options)]
    out6 = [vp] * 6
    lib.gt_trace.argtypes = [vp, i64, d, i] + out6
    lib.gt_trace_range.argtypes = [vp, i64, i64, i64, d, i] + out6
    lib.gt_trace_pixels.argtypes = [vp, vp, i64, i64, d, i] + out6
    lib.gt_trace_host.argtypes = [vp, i64, d, i] + out6
    lib.gt_trace_disk.argtypes = [vp, d, d, d, i64, d, i] + out6 + [vp]
    lib.gt_trace_states.argtypes = [vp, i64] + [vp] * 8 + [d, i64, d, i, vp, vp]
    lib.gt_trace_batch.argtypes = [vp, ctypes.POINTER(CameraDesc), i, i64, d, i] + out6
    lib.gt_sync.argtypes = [vp]
    lib.gt_device_sm_count.argtypes = [vp, ctypes.POINTER(i)]
    lib.gt_get_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.gt_measure_fma_peak.argtypes = [i, i, i, ctypes.POINTER(d)]
    lib.gt_gemm_bf16.argtypes = [i, vp, i, i, i, vp, i64, i64, vp, i64, i64, vp, i, vp, i64,
                                 i, i, i]
    lib.gt_trace_batch_noalloc.argtypes = [i, vp, ctypes.POINTER(CameraDesc), i, i64, d, i] + out6
    lib.gt_autotune.argtypes = [vp, i, i64, i64, d, ctypes.c_char_p, ctypes.POINTER(i),
                                ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d)]
    lib.gt_trace_rays.argtypes = [vp, i64] + [vp] * 5 + [d, d, i64, d, i] + out6
    lib.gt_surrogate_num_params.argtypes = [ctypes.POINTER(i64)]
    lib.gt_surrogate_create.argtypes = [i, ctypes.POINTER(SurrogateNorm), ctypes.c_uint64,
                                        ctypes.POINTER(vp)]
    lib.gt_surrogate_destroy.argtypes = [vp]
    lib.gt_surrogate_get_params.argtypes = [vp, vp, i64]
    lib.gt_surrogate_set_params.argtypes = [vp, vp, i64]
    lib.gt_surrogate_eval.argtypes = [vp, vp, i64] + [vp] * 5 + [vp]
    lib.gt_surrogate_grad.argtypes = [vp, vp, i64] + [vp] * 8 + [ctypes.c_float, vp, vp]
    lib.gt_surrogate_train.argtypes = [vp, vp, ctypes.POINTER(TrainCfg), i64] + [vp] * 8 + [vp]
    lib.gt_surrogate_infer.argtypes = [vp, vp, ctypes.POINTER(GateCfg), i64, d, i] + out6 + [
        ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.gt_surrogate_get_grads.argtypes = [vp, vp, i64]
    lib.gt_strerror.argtypes = [i]
    lib.gt_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "gt_strerror":
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != GT_OK:
        raise GeotraceError(rc, what)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def measure_fma_peak(device: int = 0, fp64: bool = True, iters: int = 2000) -> float:
    """FLOP/s of independent FMA chains on `device` (gt_measure_fma_peak)."""
    v = ctypes.c_double()
    _check(load_library().gt_measure_fma_peak(device, 1 if fp64 else 0, iters, ctypes.byref(v)),
           "gt_measure_fma_peak")
    return v.value


class Tracer:
    """One library context (gt_ctx) on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self.lib.gt_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)),
               "gt_create")
        self.ctx = h
        self.res = (0, 0)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zone_stats(self):
        """(RK4 steps the last trace took in the zone, field evaluations of them done in
        FP64) (gt_get_stats)."""
        v, f = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.gt_get_stats(self.ctx, ctypes.byref(v), ctypes.byref(f)),
               "gt_get_stats")
        return v.value, f.value

    def zone_steps(self) -> int:
        """RK4 steps the last trace took in the zone (gt_get_stats)."""
        return self.zone_stats()[0]

    def sm_count(self) -> int:
        n = ctypes.c_int()
        _check(self.lib.gt_device_sm_count(self.ctx, ctypes.byref(n)), "gt_device_sm_count")
        return n.value

    def set_spacetime(self, M: float, S: float, Q: float):
        _check(self.lib.gt_set_spacetime(self.ctx, M, S, Q), "gt_set_spacetime")

    def set_camera(self, r0: float, theta0: float, fov_deg: float, res_x: int, res_y: int):
        _check(self.lib.gt_set_camera(self.ctx, r0, theta0, fov_deg, res_x, res_y),
               "gt_set_camera")
        self.res = (res_x, res_y)

    def set_options(self, block_size=0, blocks_per_sm=0, flags=0, reproject_every=0,
                    r_switch=0.0, timeout_seconds=0.0, rays_per_thread=0):
        o = Options(block_size, blocks_per_sm, flags, reproject_every, r_switch, timeout_seconds,
                    rays_per_thread)
        _check(self.lib.gt_set_options(self.ctx, ctypes.byref(o)), "gt_set_options")

    def alloc_outputs(self, n: int) -> dict:
        torch = self._torch
        dev = torch.device("cuda", self.device)
        out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("t", "r", "th", "ph")}
        out["status"] = torch.empty(n, dtype=torch.uint8, device=dev)
        out["nsteps"] = torch.empty(n, dtype=torch.int32, device=dev)  # read as uint32
        return out

    def trace(self, n_steps: int, step_precision: float, mode: int = MODE_FP64,
              out: Optional[dict] = None) -> dict:
        """gt_trace into device tensors (allocated here when `out` is None)."""
        n = self.res[0] * self.res[1]
        if out is None:
            out = self.alloc_outputs(n)
        rc = self.lib.gt_trace(self.ctx, int(n_steps), float(step_precision), int(mode),
                               *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph", "status",
                                                             "nsteps")])
        _check(rc, "gt_trace")
        return out

    def trace_range(self, first: int, count: int, n_steps: int, step_precision: float,
                    mode: int = MODE_FP64, out: Optional[dict] = None) -> dict:
        """gt_trace_range: pixels [first, first + count) into device tensors."""
        if out is None:
            out = self.alloc_outputs(count)
        rc = self.lib.gt_trace_range(self.ctx, int(first), int(count), int(n_steps),
                                     float(step_precision), int(mode),
                                     *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph",
                                                                   "status", "nsteps")])
        _check(rc, "gt_trace_range")
        return out

    def trace_pixels(self, pixels, n_steps: int, step_precision: float, mode: int = MODE_FP64,
                     out: Optional[dict] = None) -> dict:
        """gt_trace_pixels: the listed flat pixels (int64 device tensor), compact outputs."""
        n = pixels.numel()
        if out is None:
            out = self.alloc_outputs(n)
        rc = self.lib.gt_trace_pixels(self.ctx, _ptr(pixels), n, int(n_steps),
                                      float(step_precision), int(mode),
                                      *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph",
                                                                    "status", "nsteps")])
        _check(rc, "gt_trace_pixels")
        return out

    def trace_disk(self, r_in: float, r_out: float, half_thickness: float, n_steps: int,
                   step_precision: float, mode: int = MODE_FP64,
                   out: Optional[dict] = None) -> dict:
        """gt_trace_disk: the camera with the ring as an exit; adds "z" (redshift factor)."""
        n = self.res[0] * self.res[1]
        if out is None:
            out = self.alloc_outputs(n)
            out["z"] = self._torch.empty(n, dtype=self._torch.float64,
                                         device=out["t"].device)
        rc = self.lib.gt_trace_disk(self.ctx, float(r_in), float(r_out), float(half_thickness),
                                    int(n_steps), float(step_precision), int(mode),
                                    *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph", "status",
                                                                  "nsteps", "z")])
        _check(rc, "gt_trace_disk")
        return out

    def trace_states(self, states: dict, r_escape: float, n_steps: int, step_precision: float,
                     mode: int = MODE_FP64, out: Optional[dict] = None) -> dict:
        """gt_trace_states: integrate the float64 device tensors states["t", "r", "th",
        "ph", "pt", "pr", "pth", "pph"] in place; returns status and nsteps of this call."""
        torch = self._torch
        n = states["t"].numel()
        if out is None:
            dev = states["t"].device
            out = {"status": torch.empty(n, dtype=torch.uint8, device=dev),
                   "nsteps": torch.empty(n, dtype=torch.int32, device=dev)}
        rc = self.lib.gt_trace_states(self.ctx, n, *[_ptr(states[k]) for k in
                                                     ("t", "r", "th", "ph", "pt", "pr", "pth",
                                                      "pph")],
                                      float(r_escape), int(n_steps), float(step_precision),
                                      int(mode), _ptr(out["status"]), _ptr(out["nsteps"]))
        _check(rc, "gt_trace_states")
        return out

    def trace_host(self, n_steps: int, step_precision: float, mode: int = MODE_FP64,
                   out: Optional[dict] = None) -> dict:
        """gt_trace_host into host (numpy or pinned torch) arrays."""
        n = self.res[0] * self.res[1]
        if out is None:
            out = {k: np.empty(n) for k in ("t", "r", "th", "ph")}
            out["status"] = np.empty(n, dtype=np.uint8)
            out["nsteps"] = np.empty(n, dtype=np.uint32)
        rc = self.lib.gt_trace_host(self.ctx, int(n_steps), float(step_precision), int(mode),
                                    *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph",
                                                                  "status", "nsteps")])
        _check(rc, "gt_trace_host")
        return out

    def trace_batch(self, cams: Sequence, n_steps: int, step_precision: float,
                    mode: int = MODE_FP64, out: Optional[dict] = None) -> dict:
        """gt_trace_batch over camera objects with M, S, Q, r0, theta0, fov_deg, res_x, res_y."""
        arr = (CameraDesc * len(cams))()
        total = 0
        for k, c in enumerate(cams):
            arr[k] = CameraDesc(c.M, c.S, c.Q, c.r0, c.theta0, c.fov_deg, c.res_x, c.res_y)
            total += c.res_x * c.res_y
        if out is None:
            out = self.alloc_outputs(total)
        rc = self.lib.gt_trace_batch(self.ctx, arr, len(cams), int(n_steps),
                                     float(step_precision), int(mode),
                                     *[_ptr(out.get(k)) for k in ("t", "r", "th", "ph",
                                                                   "status", "nsteps")])
        _check(rc, "gt_trace_batch")
        return out

    def autotune(self, mode: int, trial_rays: int = 1 << 17, trial_steps: int = 400,
                 step_precision: float = 1.5e-4, cache_path: Optional[str] = None):
        """gt_autotune: returns (block_size, blocks_per_sm, rays_per_thread, trial steps/s)
        and keeps them in the context's options."""
        b, k, rpt, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(self.lib.gt_autotune(self.ctx, int(mode), int(trial_rays), int(trial_steps),
                                    float(step_precision),
                                    cache_path.encode() if cache_path else None,
                                    ctypes.byref(b), ctypes.byref(k), ctypes.byref(rpt),
                                    ctypes.byref(v)),
               "gt_autotune")
        return b.value, k.value, rpt.value, v.value

    def trace_rays(self, alpha, beta, spin, q, theta0, M: float, r0: float, n_steps: int,
                   step_precision: float, mode: int = MODE_FP32_MIXED,
                   out: Optional[dict] = None) -> dict:
        """gt_trace_rays: one spacetime and camera per ray (float64 device tensors)."""
        n = alpha.numel()
        if out is None:
            out = self.alloc_outputs(n)
        rc = self.lib.gt_trace_rays(self.ctx, n, *[_ptr(x) for x in (alpha, beta, spin, q, theta0)],
                                    float(M), float(r0), int(n_steps), float(step_precision),
                                    int(mode), *[_ptr(out.get(k)) for k in
                                                 ("t", "r", "th", "ph", "status", "nsteps")])
        _check(rc, "gt_trace_rays")
        return out

    def sync(self):
        _check(self.lib.gt_sync(self.ctx), "gt_sync")


class Surrogate:
    """The surrogate network (gt_surrogate_*): training and gated inference."""

    def __init__(self, device: int = 0, r0: float = 15.0, fov_deg: float = 75.0,
                 spin_max: float = 0.99, q_max: float = 2.0, theta0_min: float = 0.0872664626,
                 theta0_max: float = 1.5707963268, seed: int = 1):
        self.lib = load_library()
        self.device = device
        self.norm = SurrogateNorm(r0, fov_deg, spin_max, q_max, theta0_min, theta0_max)
        h = ctypes.c_void_p()
        _check(self.lib.gt_surrogate_create(device, ctypes.byref(self.norm), seed, ctypes.byref(h)),
               "gt_surrogate_create")
        self.h = h
        n = ctypes.c_int64()
        _check(self.lib.gt_surrogate_num_params(ctypes.byref(n)), "gt_surrogate_num_params")
        self.n_params = n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.gt_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self.lib.gt_surrogate_get_params(self.h, out.ctypes.data, self.n_params),
               "gt_surrogate_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self.lib.gt_surrogate_set_params(self.h, p.ctypes.data, p.size),
               "gt_surrogate_set_params")

    def eval(self, tracer: "Tracer", inputs) -> "object":
        import torch
        n = inputs[0].numel()
        out = torch.empty(n, 4, dtype=torch.float32, device=inputs[0].device)
        _check(self.lib.gt_surrogate_eval(tracer.ctx, self.h, n, *[_ptr(x) for x in inputs],
                                          _ptr(out)), "gt_surrogate_eval")
        return out

    def grad(self, tracer: "Tracer", inputs, labels, dir_weight: float):
        n = inputs[0].numel()
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self.lib.gt_surrogate_grad(tracer.ctx, self.h, n, *[_ptr(x) for x in inputs],
                                          *[_ptr(x) for x in labels], float(dir_weight),
                                          g.ctypes.data, ctypes.byref(loss)), "gt_surrogate_grad")
        return g, loss.value

    def train(self, tracer: "Tracer", inputs, labels, epochs: int, batch: int, lr: float,
              weight_decay: float = 0.0, dir_weight: float = 10.0) -> np.ndarray:
        n = inputs[0].numel()
        cfg = TrainCfg(epochs, batch, lr, weight_decay, dir_weight)
        losses = np.zeros(epochs, dtype=np.float32)
        _check(self.lib.gt_surrogate_train(tracer.ctx, self.h, ctypes.byref(cfg), n,
                                           *[_ptr(x) for x in inputs], *[_ptr(x) for x in labels],
                                           losses.ctypes.data), "gt_surrogate_train")
        return losses

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self.lib.gt_surrogate_get_grads(self.h, out.ctypes.data, self.n_params),
               "gt_surrogate_get_grads")
        return out

    def infer(self, tracer: "Tracer", tau: float, band: float, n_steps: int,
              step_precision: float, mode: int = MODE_FP32_MIXED, out: Optional[dict] = None,
              dir_tol: float = 0.0, probe_stride: int = 0, probe_tol: float = 0.0,
              axis: float = 0.0, with_probes: bool = False):
        """gt_surrogate_infer; returns (outputs, integrated pixels besides the probes) or,
        with with_probes, (outputs, fallback pixels, probe pixels)."""
        n = tracer.res[0] * tracer.res[1]
        if out is None:
            out = tracer.alloc_outputs(n)
        nfb, npr = ctypes.c_int64(), ctypes.c_int64()
        gate = GateCfg(float(tau), float(band), float(axis), float(dir_tol), int(probe_stride),
                       float(probe_tol))
        _check(self.lib.gt_surrogate_infer(tracer.ctx, self.h, ctypes.byref(gate),
                                           int(n_steps), float(step_precision), int(mode),
                                           *[_ptr(out[k]) for k in ("t", "r", "th", "ph",
                                                                    "status", "nsteps")],
                                           ctypes.byref(nfb), ctypes.byref(npr)),
               "gt_surrogate_infer")
        if with_probes:
            return out, nfb.value, npr.value
        return out, nfb.value
