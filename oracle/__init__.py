"""FP64 CPU oracle of the null-geodesic ray tracer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  The product path
(``paper_2310_15183_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``geodesic_oracle.c`` (plain C, no fast-math, no FMA
contraction).  This module only builds it with gcc and marshals arguments
through ctypes.  Each wrapped C function cites the paper passage it follows
in the C source.

Status codes: 0 ESCAPED, 1 HORIZON, 2 MAXSTEPS, 3 NONFINITE, 5 DISK (the ray entered the
ring volume).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geodesic_oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

ESCAPED, HORIZON, MAXSTEPS, NONFINITE, DISK = 0, 1, 2, 3, 5
FLAG_COMPAT_WEIGHTS = 1
FLAG_COMPAT_CAMERA = 2
FLAG_FD_DERIVS = 4  # forward-difference metric derivatives (listing's derPrecision 1e-8)
FLAG_F32_IO = 8     # float32 spacetime parameters, initial state and outputs (listing)
FLAG_EULER = 16     # explicit Euler (Sec. 3.1.1)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(_SRC)):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(LIB_PATH)
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        pd = ctypes.POINTER(ctypes.c_double)
        pi = ctypes.POINTER(ctypes.c_int)
        pi64 = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        for name in ("or_metric_lower", "or_metric_upper", "or_mn_fields",
                     "or_mn_metric_upper", "or_mn_metric_lower"):
            getattr(lib, name).argtypes = [d, d, d, d, d, pd]
            getattr(lib, name).restype = i
        lib.or_dmetric_upper.argtypes = [d, d, d, d, d, i, pd]
        lib.or_dmetric_upper.restype = i
        lib.or_vector_field.argtypes = [d, d, d, pd, pd, pd, pd]
        lib.or_vector_field.restype = i
        lib.or_hamiltonian.argtypes = [d, d, d, pd, pd, pd]
        lib.or_hamiltonian.restype = i
        lib.or_camera_ray.argtypes = [d, d, d, d, d, d, i, i, i, i, i, pd, pd]
        lib.or_camera_ray.restype = i
        lib.or_camera_dir.argtypes = [d, d, d, d, d, d, d, i, pd, pd]
        lib.or_camera_dir.restype = i
        lib.or_trace_ray.argtypes = [d, d, d, pd, pd, d, i64, d, i, pi, pi64, pd]
        lib.or_trace_ray.restype = i
        lib.or_trace_ray_path.argtypes = [d, d, d, pd, pd, d, i64, d, i, pd, i64, pi64]
        lib.or_trace_ray_path.restype = i
        lib.or_trace_image.argtypes = [d, d, d, d, d, d, i, i, i64, d, i, vp, i64, i,
                                       vp, vp, vp, vp, vp, vp, vp, vp]
        lib.or_trace_image.restype = i
        lib.or_trace_image_disk.argtypes = [d, d, d, d, d, d, i, i, i64, d, i, d, d, d, vp, i64,
                                            i, vp, vp, vp, vp, vp, vp, vp]
        lib.or_trace_image_disk.restype = i
        lib.or_circular_orbit.argtypes = [d, d, d, d, d, i, pd]
        lib.or_circular_orbit.restype = i
        lib.or_redshift.argtypes = [d, d, d, d, d, pd, pd, i, pd]
        lib.or_redshift.restype = i
        _lib = lib
        return lib


def _arr(n):
    return (ctypes.c_double * n)()


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid argument (rc={rc})")


def metric_lower(M, S, Q, r, th) -> np.ndarray:
    """g_{mu nu}(r, theta), 4x4, index order (t, r, theta, phi)."""
    g = _arr(16)
    _check(_load().or_metric_lower(M, S, Q, r, th, g), "metric_lower")
    return np.array(g[:]).reshape(4, 4)


def metric_upper(M, S, Q, r, th) -> np.ndarray:
    """g^{mu nu}(r, theta) as used by the integrator."""
    g = _arr(16)
    _check(_load().or_metric_upper(M, S, Q, r, th, g), "metric_upper")
    return np.array(g[:]).reshape(4, 4)


def dmetric_upper(M, S, Q, r, th, method=0) -> np.ndarray:
    """d[mu, nu, sigma] = d_mu g^{nu sigma}; method 0 = integrator's, 1 = complex step."""
    g = _arr(64)
    _check(_load().or_dmetric_upper(M, S, Q, r, th, method, g), "dmetric_upper")
    return np.array(g[:]).reshape(4, 4, 4)


def mn_fields(M, S, Q, r, th) -> dict:
    """Manko-Novikov scalar functions (Q may be 0 here: q -> 0 limit)."""
    o = _arr(8)
    _check(_load().or_mn_fields(M, S, Q, r, th, o), "mn_fields")
    keys = ("f", "omega", "e2gamma", "rho2", "Delta", "alpha", "k", "beta")
    return dict(zip(keys, o[:]))


def mn_metric_upper(M, S, Q, r, th) -> np.ndarray:
    g = _arr(16)
    _check(_load().or_mn_metric_upper(M, S, Q, r, th, g), "mn_metric_upper")
    return np.array(g[:]).reshape(4, 4)


def mn_metric_lower(M, S, Q, r, th) -> np.ndarray:
    g = _arr(16)
    _check(_load().or_mn_metric_lower(M, S, Q, r, th, g), "mn_metric_lower")
    return np.array(g[:]).reshape(4, 4)


def vector_field(M, S, Q, q, p):
    qa, pa, dq, dp = _arr(4), _arr(4), _arr(4), _arr(4)
    qa[:] = list(map(float, q))
    pa[:] = list(map(float, p))
    _check(_load().or_vector_field(M, S, Q, qa, pa, dq, dp), "vector_field")
    return np.array(dq[:]), np.array(dp[:])


def hamiltonian(M, S, Q, q, p) -> float:
    qa, pa, h = _arr(4), _arr(4), ctypes.c_double()
    qa[:] = list(map(float, q))
    pa[:] = list(map(float, p))
    _check(_load().or_hamiltonian(M, S, Q, qa, pa, ctypes.byref(h)), "hamiltonian")
    return h.value


def camera_ray(M, S, Q, r0, th0, fov_deg, resX, resY, i, j, flags=0):
    """Initial (q, p) of pixel (i, j): i along phi (resX), j along theta (resY)."""
    q, p = _arr(4), _arr(4)
    _check(_load().or_camera_ray(M, S, Q, r0, th0, fov_deg, resX, resY, i, j, flags, q, p),
           "camera_ray")
    return np.array(q[:]), np.array(p[:])


def camera_dir(M, S, Q, r0, th0, alpha, beta, flags=0):
    """Initial (q, p) of the ray leaving a camera at (r0, th0) in direction (alpha, beta)."""
    q, p = _arr(4), _arr(4)
    _check(_load().or_camera_dir(M, S, Q, r0, th0, float(alpha), float(beta), flags, q, p),
           "camera_dir")
    return np.array(q[:]), np.array(p[:])


def trace_ray(M, S, Q, q, p, r_start, n_steps, sp, flags=0):
    """Integrate one ray; returns (q_end, p_end, status, nsteps, min_sin)."""
    qa, pa = _arr(4), _arr(4)
    qa[:] = list(map(float, q))
    pa[:] = list(map(float, p))
    st, ns, ms = ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
    _check(_load().or_trace_ray(M, S, Q, qa, pa, r_start, int(n_steps), sp, flags,
                                ctypes.byref(st), ctypes.byref(ns), ctypes.byref(ms)),
           "trace_ray")
    return np.array(qa[:]), np.array(pa[:]), st.value, ns.value, ms.value


def trace_path(M, S, Q, q, p, r_start, n_steps, sp, flags=0, max_states=None) -> np.ndarray:
    """All accepted states (n, 8) = (q, p) starting with the initial one."""
    if max_states is None:
        max_states = int(n_steps) + 1
    qa, pa = _arr(4), _arr(4)
    qa[:] = list(map(float, q))
    pa[:] = list(map(float, p))
    buf = np.zeros((max_states, 8))
    n = ctypes.c_int64()
    _check(_load().or_trace_ray_path(M, S, Q, qa, pa, r_start, int(n_steps), sp, flags,
                                     buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     max_states, ctypes.byref(n)), "trace_path")
    return buf[: n.value].copy()


def circular_orbit(M, S, Q, r, th, flags=0) -> np.ndarray:
    """Momentum (p_t, p_r, p_theta, p_phi) of the ring's circular-orbit emitter at (r, th)."""
    p = _arr(4)
    _check(_load().or_circular_orbit(M, S, Q, r, th, flags, p), "circular_orbit")
    return np.array(p[:])


def redshift(M, S, Q, r0, th0, q, p, flags=0) -> float:
    """Redshift factor of a ray (q, p) at the ring against a static observer at (r0, th0)."""
    qa, pa, z = _arr(4), _arr(4), ctypes.c_double()
    qa[:] = list(map(float, q))
    pa[:] = list(map(float, p))
    _check(_load().or_redshift(M, S, Q, r0, th0, qa, pa, flags, ctypes.byref(z)), "redshift")
    return z.value


def trace_image_disk(M, S, Q, r0, th0, fov_deg, resX, resY, n_steps, sp, r_in, r_out,
                     half_thickness, flags=0, pixels=None, threads=None) -> dict:
    """trace_image with the ring as an exit; adds the redshift factor "z" per ray."""
    if threads is None:
        threads = os.cpu_count() or 1
    if pixels is not None:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        n = pixels.size
    else:
        n = int(resX) * int(resY)
    out = {k: np.zeros(n) for k in ("t", "r", "th", "ph", "z")}
    out["status"] = np.zeros(n, dtype=np.uint8)
    out["nsteps"] = np.zeros(n, dtype=np.uint32)
    rc = _load().or_trace_image_disk(
        M, S, Q, r0, th0, fov_deg, int(resX), int(resY), int(n_steps), sp, int(flags),
        r_in, r_out, half_thickness, None if pixels is None else pixels.ctypes.data, int(n),
        int(threads), *[out[k].ctypes.data for k in ("t", "r", "th", "ph", "status", "nsteps",
                                                      "z")])
    _check(rc, "trace_image_disk")
    return out


def trace_image(M, S, Q, r0, th0, fov_deg, resX, resY, n_steps, sp, flags=0,
                pixels=None, threads=None, want_p=False, want_min_sin=False) -> dict:
    """Trace a camera (or the listed flat pixel indices j*resX + i) on host threads."""
    if threads is None:
        threads = os.cpu_count() or 1
    if pixels is not None:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        n = pixels.size
    else:
        n = int(resX) * int(resY)
    out = {k: np.zeros(n) for k in ("t", "r", "th", "ph")}
    out["status"] = np.zeros(n, dtype=np.uint8)
    out["nsteps"] = np.zeros(n, dtype=np.uint32)
    if want_p:
        out["p"] = np.zeros((n, 4))
    if want_min_sin:
        out["min_sin"] = np.zeros(n)

    def ptr(a):
        return None if a is None else a.ctypes.data

    rc = _load().or_trace_image(
        M, S, Q, r0, th0, fov_deg, int(resX), int(resY), int(n_steps), sp, int(flags),
        ptr(pixels), int(n), int(threads),
        ptr(out["t"]), ptr(out["r"]), ptr(out["th"]), ptr(out["ph"]),
        ptr(out["status"]), ptr(out["nsteps"]), ptr(out.get("p")), ptr(out.get("min_sin")))
    _check(rc, "trace_image")
    return out
