"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle legs.

This module holds parameters and seeded random draws only -- none of the method's
arithmetic -- so both the CUDA path and the CPU oracle may take their inputs from it.

Spacetime and camera values follow the paper where it prints them: M = 0.5,
S = 0.24, q = 2.0, FOV 75 deg, 1000x1000 pixels, step_precision 1.5e-4 (appendix
listing), 500,000 steps per image (listing's kernel call), escape at 1.5 r0.
Where the paper is silent the values below are stated choices.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEG = math.pi / 180.0


@dataclasses.dataclass(frozen=True)
class Camera:
    """One (M, S, Q) spacetime plus a pinhole camera (Sec. 3.3.1)."""
    M: float
    S: float
    Q: float
    r0: float
    theta0: float  # radians
    fov_deg: float
    res_x: int
    res_y: int

    @property
    def n_rays(self) -> int:
        return self.res_x * self.res_y


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    camera: Camera
    n_steps: int
    step_precision: float


# Schwarzschild, camera at r0 = 20M, 64x64.
SCHW_64 = Camera(M=0.5, S=0.0, Q=0.0, r0=10.0, theta0=math.pi / 2, fov_deg=75.0,
                 res_x=64, res_y=64)
# Rotating Manko-Novikov hole of the listing (M=0.5, S=0.24, q=2), r0 = 30M,
# inclination 80 deg, the paper's 1000x1000 resolution.
MN_1000 = Camera(M=0.5, S=0.24, Q=2.0, r0=15.0, theta0=80 * DEG, fov_deg=75.0,
                 res_x=1000, res_y=1000)

WORKLOADS = {
    # literal step caps: every ray stops as MAXSTEPS
    "schw64": Workload("schw64", SCHW_64, 2000, 1.5e-4),
    "mn1000": Workload("mn1000", MN_1000, 20000, 1.5e-4),
    # terminating variants: step cap high enough for rays to escape or fall in
    "schw64_T": Workload("schw64_T", SCHW_64, 400000, 1.5e-4),
    "mn1000_T": Workload("mn1000_T", MN_1000, 500000, 1.5e-4),
}


# smaller cases of the same kernels, for profiler captures
WORKLOADS["mn256"] = Workload("mn256", dataclasses.replace(MN_1000, res_x=256, res_y=256),
                              20000, 1.5e-4)
WORKLOADS["mn512"] = Workload("mn512", dataclasses.replace(MN_1000, res_x=512, res_y=512),
                              20000, 1.5e-4)
WORKLOADS["mn256_short"] = Workload("mn256_short",
                                    dataclasses.replace(MN_1000, res_x=256, res_y=256),
                                    2000, 1.5e-4)
# the camera inside the Manko-Novikov zone (r0 = 3.8M < 4M): every FP32-mixed ray is handed
# to the zone kernel after its first step, so its launches carry the work
WORKLOADS["mn256_zone"] = Workload("mn256_zone",
                                   dataclasses.replace(MN_1000, r0=1.9, res_x=256, res_y=256),
                                   4000, 1.5e-4)


def sub_camera(cam: Camera, res_x: int, res_y: int) -> Camera:
    """Same spacetime and viewpoint at another resolution."""
    return dataclasses.replace(cam, res_x=res_x, res_y=res_y)


def sample_pixels(n_rays: int, n_sample: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of flat pixel indices (without replacement)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_sample = min(n_sample, n_rays)
    return np.sort(rng.choice(n_rays, size=n_sample, replace=False)).astype(np.int64)


def batch_cameras(n_cams: int = 64, seed: int = 2310, M: float = 0.5,
                  side_min: int = 128, side_max: int = 1024) -> list:
    """Uneven batch of Kerr cameras: side n = round(exp(U[ln side_min, ln side_max]))
    (square), spin a ~ U[0, 0.99M] (S = a M), q = 0, inclination ~ U[5, 90] deg,
    r0 ~ U[15M, 50M], FOV 75 deg; PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cams = []
    for _ in range(n_cams):
        side = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        a = rng.uniform(0.0, 0.99 * M)
        th0 = rng.uniform(5.0, 90.0) * DEG
        r0 = rng.uniform(15.0 * M, 50.0 * M)
        cams.append(Camera(M=M, S=a * M, Q=0.0, r0=r0, theta0=th0, fov_deg=75.0,
                           res_x=side, res_y=side))
    return cams


def surrogate_samples(n: int, seed: int = 15183, M: float = 0.5, fov_deg: float = 75.0,
                      r0: float = 15.0, q_max: float = 0.0):
    """Training inputs of the surrogate: pixel direction (alpha, beta) uniform over the
    FOV square of a camera at r0, dimensionless spin a/M ~ U[0, 0.99] (S = (a/M) M^2),
    q = 0, inclination ~ U[5, 90] deg.  With q_max > 0 the Manko-Novikov deviation is a
    live input, q ~ U[-q_max, q_max], and the spin is drawn from U[0.1, 0.99] (q != 0
    needs S != 0; the paper's "non-rotating" Manko-Novikov holes use S = 0.1 M^2).
    Returns float64 arrays (alpha, beta, a/M, q, theta0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    V = math.tan(0.5 * fov_deg * DEG) / r0
    H = math.atan(math.tan(V))
    alpha = rng.uniform(-H, H, n)
    beta = rng.uniform(-V, V, n)
    a = rng.uniform(0.1 if q_max > 0 else 0.0, 0.99, n)
    q = rng.uniform(-q_max, q_max, n) if q_max > 0 else np.zeros(n)
    th0 = rng.uniform(5.0, 90.0, n) * DEG
    return alpha, beta, a, q, th0
