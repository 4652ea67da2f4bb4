"""GPU parity of the ring and redshift (Sec. 3.3.3), the paper's own numerics
(forward-difference derivatives, float32 I/O, listing weights and camera), explicit
Euler (Sec. 3.1.1), integration from arbitrary states -- timelike orbits (Sec. 3.2.1)
and checkpoint/resume -- and the out-of-memory path, all through the C ABI against the
FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2310_15183_gb300 import workloads as W

from .parity import assert_fp64_parity, mixed_report, neighbour_band, to_numpy

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15183_gb300 import build, geotrace
    build.build()
    return geotrace


@pytest.fixture()
def tracer(g):
    t = g.Tracer(0)
    yield t
    t.close()


def _setup(tracer, cam, **opts):
    tracer.set_spacetime(cam.M, cam.S, cam.Q)
    tracer.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tracer.set_options(**opts)


# the ring renders of Sec. 5: Kerr a = 0.98M and Manko-Novikov a = 0.1M, q = -2
RING_CAMS = [
    (W.Camera(M=0.5, S=0.98 * 0.25, Q=0.0, r0=15.0, theta0=80 * W.DEG, fov_deg=40.0,
              res_x=40, res_y=30), (2.0, 6.0, 0.05), 300000),
    (W.Camera(M=0.5, S=0.1 * 0.25, Q=-2.0, r0=15.0, theta0=75 * W.DEG, fov_deg=40.0,
              res_x=24, res_y=18), (2.0, 6.0, 0.08), 120000),
]


@pytest.mark.parametrize("cam,ring,cap", RING_CAMS)
def test_ring_and_redshift_match_oracle(tracer, oracle, cam, ring, cap):
    """FP64: status (ring hits included), end state to 1e-9 and redshift factor to 1e-9
    against the oracle, outside the chaotic boundary band; FP32-mixed: the same
    classification on >= 99.9 % and redshift within 1e-5 on the rays both call hits."""
    r_in, r_out, hh = ring
    _setup(tracer, cam)
    got = to_numpy(tracer.trace_disk(r_in, r_out, hh, cap, 1.5e-4, 0))
    ref = oracle.trace_image_disk(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                  cam.res_x, cam.res_y, cap, 1.5e-4, r_in, r_out, hh)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y)
    assert_fp64_parity(got, ref, exclude=band, what="ring")
    hit = (ref["status"] == oracle.DISK) & ~band
    assert hit.sum() >= 10
    assert np.all(np.abs(got["z"][hit] - ref["z"][hit]) <= 1e-9 * np.abs(ref["z"][hit]))
    assert np.all(np.isnan(got["z"][ref["status"] != oracle.DISK]))
    assert np.all((ref["z"][hit] > 0.3) & (ref["z"][hit] < 3.0))
    mixed = to_numpy(tracer.trace_disk(r_in, r_out, hh, cap, 1.5e-4, 1))
    rep = mixed_report(mixed, ref, exclude=band)
    assert rep["agree"] >= 0.999, rep
    both = hit & (mixed["status"] == oracle.DISK)
    assert np.max(np.abs(mixed["z"][both] - ref["z"][both]) / ref["z"][both]) < 1e-5


def test_paper_numerics_match_oracle(g, tracer, oracle):
    """The listing's numerics -- forward-difference derivatives (delta = 1e-8), float32
    arguments and results, 0.1667 weights, v^phi = alpha -- on both sides.  The two
    evaluate g^{mu nu} by different formulas, and forward differences amplify their
    ~1e-16 rounding differences by 1/delta, so the tolerance is 1e-6 relative
    (the float32 outputs themselves are exact float32 values)."""
    flags = g.FLAGS_PAPER
    for cam in (W.Camera(0.5, 0.24, 0.0, 8.0, math.pi / 2, 75.0, 12, 9),
                W.sub_camera(W.MN_1000, 10, 8)):
        _setup(tracer, cam, flags=flags)
        got = to_numpy(tracer.trace(2000, 1.5e-4, 0))
        ref = oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg, cam.res_x,
                                 cam.res_y, 2000, 1.5e-4, flags=flags)
        assert_fp64_parity(got, ref, tol=1e-6, what="paper numerics")
        for k in ("t", "r", "th", "ph"):
            assert np.array_equal(got[k], got[k].astype(np.float32).astype(np.float64)), k
        _setup(tracer, cam)
        exact = to_numpy(tracer.trace(2000, 1.5e-4, 0))
        assert not np.array_equal(exact["r"], got["r"])
    # the listing's numerics are FP64 only
    tracer.set_options(flags=g.FLAG_FD_DERIVS)
    with pytest.raises(g.GeotraceError):
        tracer.trace(10, 1.5e-4, 1)


def test_euler_matches_oracle(g, tracer, oracle):
    cam = W.sub_camera(W.MN_1000, 9, 7)
    _setup(tracer, cam, flags=g.FLAG_EULER)
    got = to_numpy(tracer.trace(3000, 1.5e-4, 0))
    ref = oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg, cam.res_x,
                             cam.res_y, 3000, 1.5e-4, flags=oracle.FLAG_EULER)
    assert_fp64_parity(got, ref, what="euler")


def _orbits(n, seed, M=0.5):
    """Equatorial and inclined bound timelike orbits of Schwarzschild/Kerr started at
    r in [8M, 16M] with p_r = 0 and a little p_theta, H = -1/2 (E from the mass shell)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(16 * M, 32 * M, n)
    th = np.full(n, math.pi / 2) + rng.uniform(-0.2, 0.2, n)
    L = np.sqrt(M * r) / np.sqrt(1 - 3 * M / r) * rng.uniform(0.9, 1.05, n)
    pth = rng.uniform(-0.5, 0.5, n)
    return r, th, L, pth


def _mass_shell(oracle, M, S, r, th, L, pth):
    """p_t < 0 with g^{mu nu} p_mu p_nu = -1 for p = (p_t, 0, p_theta, L)."""
    g = oracle.metric_upper(M, S, 0.0, r, th)
    a, b = g[0, 0], 2 * g[0, 3] * L
    c = g[3, 3] * L * L + g[2, 2] * pth * pth + 1.0
    return (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)


def test_timelike_orbits_and_checkpoint_resume(g, tracer, oracle):
    """Massive particles (H = -1/2) from arbitrary states, FP64: 64 orbits of a Kerr
    spacetime against the oracle to 1e-9 (all state components), H kept to 1e-9; then
    the same run split into two calls -- the second resuming from the first's returned
    state -- equals one uninterrupted run bit for bit."""
    M, S = 0.5, 0.2
    r, th, L, pth = _orbits(64, 3)
    pt = np.array([_mass_shell(oracle, M, S, *x) for x in zip(r, th, L, pth)])
    init = {"t": np.zeros(64), "r": r, "th": th, "ph": np.zeros(64), "pt": pt,
            "pr": np.zeros(64), "pth": pth, "pph": L}
    tracer.set_spacetime(M, S, 0.0)
    tracer.set_options()
    dev = {k: torch.tensor(v, device="cuda") for k, v in init.items()}
    st = to_numpy(tracer.trace_states(dev, 1e9, 40000, 2e-3, 0))
    torch.cuda.synchronize()
    assert np.all(st["status"] == 2) and np.all(st["nsteps"] == 40000)
    got = {k: v.cpu().numpy() for k, v in dev.items()}
    for k in range(0, 64, 4):
        q0 = [init[x][k] for x in ("t", "r", "th", "ph")]
        p0 = [init[x][k] for x in ("pt", "pr", "pth", "pph")]
        qe, pe, s, ns, _ = oracle.trace_ray(M, S, 0.0, q0, p0, 1e9 / 1.5, 40000, 2e-3)
        want = np.concatenate([qe, pe])
        have = np.array([got[x][k] for x in ("t", "r", "th", "ph", "pt", "pr", "pth", "pph")])
        assert np.all(np.abs(have - want) <= 1e-9 * np.maximum(1, np.abs(want))), k
        assert abs(oracle.hamiltonian(M, S, 0.0, have[:4], have[4:]) + 0.5) < 1e-9
    # checkpoint: 2 x 20000 steps == 40000 steps
    dev2 = {k: torch.tensor(v, device="cuda") for k, v in init.items()}
    tracer.trace_states(dev2, 1e9, 20000, 2e-3, 0)
    st2 = to_numpy(tracer.trace_states(dev2, 1e9, 20000, 2e-3, 0))
    torch.cuda.synchronize()
    assert np.all(st2["nsteps"] == 20000)
    for k in init:
        assert np.array_equal(dev2[k].cpu().numpy(), got[k]), k


def test_camera_states_reproduce_the_camera_trace(g, tracer, oracle):
    """Null rays handed in as states (the oracle camera's initial data) follow the same
    arithmetic as the camera trace: equal to it to 1e-12 (the two cameras round
    differently), and escape at the given radius."""
    cam = W.sub_camera(W.MN_1000, 8, 6)
    _setup(tracer, cam)
    ref = to_numpy(tracer.trace(300000, 1.5e-4, 0))
    init = {k: [] for k in ("t", "r", "th", "ph", "pt", "pr", "pth", "pph")}
    for j in range(cam.res_y):
        for i in range(cam.res_x):
            q, p = oracle.camera_ray(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg,
                                     cam.res_x, cam.res_y, i, j)
            for k, v in zip(init, list(q) + list(p)):
                init[k].append(v)
    dev = {k: torch.tensor(v, device="cuda") for k, v in init.items()}
    st = to_numpy(tracer.trace_states(dev, 1.5 * cam.r0, 300000, 1.5e-4, 0))
    torch.cuda.synchronize()
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y)
    keep = ~band
    assert np.array_equal(st["status"][keep], ref["status"][keep])
    for k in ("t", "r", "th", "ph"):
        v = dev[k].cpu().numpy()
        assert np.all(np.abs(v[keep] - ref[k][keep]) <= 1e-9 * np.maximum(1, np.abs(ref[k][keep]))), k


def test_out_of_memory_is_reported_and_context_survives(g, tracer, oracle):
    """A request for more device memory than the GPU has (the host-copy staging of a
    100,000 x 100,000 image, 370 GB) fails cleanly with GT_ERR_OOM -- no fault, nothing
    allocated -- and the context keeps working."""
    lib, ctx = tracer.lib, tracer.ctx
    assert lib.gt_set_spacetime(ctx, 0.5, 0.24, 0.0) == 0
    assert lib.gt_set_camera(ctx, 15.0, 1.2, 75.0, 100000, 100000) == 0
    assert lib.gt_trace_host(ctx, 10, 1.5e-4, 0, None, None, None, None, None, None) == -4
    cam = W.Camera(0.5, 0.24, 0.0, 15.0, 1.2, 75.0, 6, 5)
    _setup(tracer, cam)
    got = to_numpy(tracer.trace(1000, 1.5e-4, 0))
    ref = oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg, cam.res_x,
                             cam.res_y, 1000, 1.5e-4)
    assert_fp64_parity(got, ref, what="after OOM")
