"""Comparison helpers for the GPU-vs-oracle parity tests (not a test module)."""
import numpy as np

KEYS = ("t", "r", "th", "ph")
TOL_FP64 = 1e-9  # relative, per component: |gpu - oracle| <= 1e-9 max(1, |oracle|)


def to_numpy(out):
    res = {}
    for k, v in out.items():
        a = v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v)
        if k == "nsteps":
            a = a.view(np.uint32)
        res[k] = a
    return res


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(1.0, np.abs(ref))


def assert_fp64_parity(got, ref, exclude=None, tol=TOL_FP64, what=""):
    """Element-wise parity on t, r, theta, phi; identical status and step counts.
    `exclude` masks rays in a stated chaotic band (they are reported, not compared)."""
    n = ref["r"].size
    keep = np.ones(n, bool) if exclude is None else ~exclude
    assert keep.sum() > 0
    bad = {}
    for k in KEYS:
        e = rel_err(got[k][keep], ref[k][keep])
        if np.max(e) > tol:
            i = np.flatnonzero(keep)[np.argmax(e)]
            bad[k] = (float(np.max(e)), int(i), float(got[k][i]), float(ref[k][i]))
    st_ok = np.array_equal(got["status"][keep], ref["status"][keep])
    ns_ok = np.array_equal(got["nsteps"][keep], ref["nsteps"][keep])
    assert not bad and st_ok and ns_ok, (what, bad, st_ok, ns_ok,
                                         np.flatnonzero(got["status"][keep] != ref["status"][keep])[:10])
    return int(n - keep.sum())


def great_circle(th1, ph1, th2, ph2):
    """Angle between the directions (theta1, phi1) and (theta2, phi2) (haversine)."""
    a = np.sin((th2 - th1) / 2) ** 2 + np.sin(th1) * np.sin(th2) * np.sin((ph2 - ph1) / 2) ** 2
    return 2 * np.arcsin(np.sqrt(np.clip(a, 0, 1)))


def mixed_report(got, ref, exclude=None):
    """Classification agreement and end-angle error of a reduced-precision result."""
    n = ref["r"].size
    keep = np.ones(n, bool) if exclude is None else ~exclude
    agree = np.mean(got["status"][keep] == ref["status"][keep])
    same = keep & (got["status"] == ref["status"])
    ang = great_circle(got["th"][same], got["ph"][same], ref["th"][same], ref["ph"][same])
    esc = same & (ref["status"] == 0)
    ang_esc = great_circle(got["th"][esc], got["ph"][esc], ref["th"][esc], ref["ph"][esc])
    return {"agree": float(agree), "max_angle": float(ang.max()) if ang.size else 0.0,
            "max_angle_escaped": float(ang_esc.max()) if ang_esc.size else 0.0,
            "n": int(keep.sum())}


def schwarzschild_band(oracle, cam, M, width=1e-3):
    """Rays whose impact parameter lies within `width` M of 3 sqrt(3) M (photon ring)."""
    bc = 3 * np.sqrt(3) * M
    mask = np.zeros(cam.res_x * cam.res_y, bool)
    for j in range(cam.res_y):
        for i in range(cam.res_x):
            _, p = oracle.camera_ray(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                     cam.res_x, cam.res_y, i, j)
            b = np.sqrt(p[2] ** 2 + p[3] ** 2 / np.sin(cam.theta0) ** 2) / abs(p[0])
            mask[j * cam.res_x + i] = abs(b - bc) < width * M
    return mask


def neighbour_band(status, res_x, res_y):
    """Pixels whose status differs from one of their 8 neighbours (chaotic boundary)."""
    s = status.reshape(res_y, res_x)
    m = np.zeros_like(s, bool)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            if di == 0 and dj == 0:
                continue
            sh = np.full_like(s, 255)
            ys = slice(max(0, dj), res_y + min(0, dj))
            yd = slice(max(0, -dj), res_y + min(0, -dj))
            xs = slice(max(0, di), res_x + min(0, di))
            xd = slice(max(0, -di), res_x + min(0, -di))
            sh[yd, xd] = s[ys, xs]
            m |= (sh != 255) & (sh != s)
    return m.ravel()


def sensitive_rays(oracle, cam, n_steps, sp, ref, eps=1e-13, thresh=1e-10, threads=16):
    """Rays of a camera whose oracle end state moves by more than `thresh` (relative, per
    component) when the initial p_r is scaled by (1 + eps): chaotic rays, where the rounding
    differences of two correct FP64 integrations (different but exact derivative routes)
    grow past the parity tolerance.  `ref` is the unperturbed oracle result of the image."""
    from concurrent.futures import ThreadPoolExecutor

    def one(k):
        j, i = divmod(k, cam.res_x)
        q, p = oracle.camera_ray(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                 cam.res_x, cam.res_y, i, j)
        p = p.copy()
        p[1] *= 1.0 + eps
        qe, _, st, _, _ = oracle.trace_ray(cam.M, cam.S, cam.Q, q, p, cam.r0, n_steps, sp)
        base = np.array([ref[x][k] for x in KEYS])
        return st != ref["status"][k] or bool(np.any(
            np.abs(qe - base) > thresh * np.maximum(1.0, np.abs(base))))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return np.array(list(ex.map(one, range(cam.res_x * cam.res_y))))
