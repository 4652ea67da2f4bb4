"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 plain must match element by element to 1e-9 relative (per component, scaled by
max(1, |value|)) with identical status and step counts, outside a stated chaotic
band; the FP32-mixed path must agree on >= 99.9 % of classifications with end-angle
error <= 1e-3 rad.  Sizes keep the oracle to seconds while spanning several warps,
blocks and a ragged tail.
"""
import math

import numpy as np
import pytest

from paper_2310_15183_gb300 import workloads as W

from .parity import (assert_fp64_parity, mixed_report, neighbour_band, schwarzschild_band,
                     sensitive_rays, to_numpy)

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


def run_gpu(tracer, cam, n_steps, sp, mode=0, **opts):
    tracer.set_spacetime(cam.M, cam.S, cam.Q)
    tracer.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tracer.set_options(**opts)
    out = tracer.trace(n_steps, sp, mode)
    torch.cuda.synchronize()
    return to_numpy(out)


def run_oracle(oracle, cam, n_steps, sp, pixels=None, flags=0, **kw):
    return oracle.trace_image(cam.M, cam.S, cam.Q, cam.r0, cam.theta0, cam.fov_deg, cam.res_x,
                              cam.res_y, n_steps, sp, flags=flags, pixels=pixels, **kw)


SCHW = W.SCHW_64
MN = W.MN_1000
KERR = W.Camera(M=0.5, S=0.24, Q=0.0, r0=15.0, theta0=80 * W.DEG, fov_deg=30.0, res_x=20,
                res_y=15)


# ----------------------------------------------------------------- FP64 plain
def test_fp64_schwarzschild_literal_full_image(tracer, oracle):
    """64x64 Schwarzschild camera, 2000 steps (every ray MAXSTEPS), all 4096 rays."""
    got = run_gpu(tracer, SCHW, 2000, 1.5e-4)
    ref = run_oracle(oracle, SCHW, 2000, 1.5e-4)
    assert_fp64_parity(got, ref, what="schw64")
    assert np.all(ref["status"] == oracle.MAXSTEPS)


def test_fp64_schwarzschild_terminating(tracer, oracle):
    """24x20 Schwarzschild image with a step cap high enough for every ray to escape or
    fall in; photon-ring band |b - 3 sqrt(3) M| < 1e-3 M excluded."""
    cam = W.sub_camera(SCHW, 24, 20)
    got = run_gpu(tracer, cam, 400000, 1.5e-4)
    ref = run_oracle(oracle, cam, 400000, 1.5e-4, want_min_sin=True)
    band = schwarzschild_band(oracle, cam, cam.M) | (ref["min_sin"] < 1e-3)
    assert_fp64_parity(got, ref, exclude=band, what="schw T")
    st = ref["status"][~band]
    assert (st == oracle.HORIZON).sum() > 20 and (st == oracle.ESCAPED).sum() > 100


def test_fp64_kerr_terminating(tracer, oracle):
    """Kerr a = 0.96M at 80 deg inclination, narrow FOV so the shadow spans many pixels."""
    got = run_gpu(tracer, KERR, 500000, 1.5e-4)
    ref = run_oracle(oracle, KERR, 500000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], KERR.res_x, KERR.res_y) | (ref["min_sin"] < 1e-3)
    assert_fp64_parity(got, ref, exclude=band, what="kerr T")
    st = ref["status"][~band]
    assert (st == oracle.HORIZON).sum() > 10 and (st == oracle.ESCAPED).sum() > 10


def test_fp64_mn_literal(tracer, oracle):
    """Manko-Novikov (M=0.5, S=0.24, q=2), r0 = 30M, 80 deg, 20,000 steps, 24x16."""
    cam = W.sub_camera(MN, 24, 16)
    got = run_gpu(tracer, cam, 20000, 1.5e-4)
    ref = run_oracle(oracle, cam, 20000, 1.5e-4)
    assert_fp64_parity(got, ref, what="mn literal")


def test_fp64_mn_terminating(tracer, oracle):
    """Manko-Novikov with the listing's 500,000-step cap on a 10x8 image."""
    cam = W.sub_camera(MN, 10, 8)
    got = run_gpu(tracer, cam, 500000, 1.5e-4)
    ref = run_oracle(oracle, cam, 500000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    assert_fp64_parity(got, ref, exclude=band, what="mn T")


def test_fp64_range_trace_matches_full_image(tracer):
    """gt_trace_range over a ragged pixel range reproduces the full-image result bitwise."""
    cam = W.sub_camera(MN, 24, 16)
    full = run_gpu(tracer, cam, 3000, 1.5e-4)
    part = to_numpy(tracer.trace_range(37, 201, 3000, 1.5e-4))
    torch.cuda.synchronize()
    for k in ("t", "r", "th", "ph", "status", "nsteps"):
        assert np.array_equal(part[k], full[k][37:238]), k


def test_fp64_full_size_sampled(tracer, oracle):
    """The 1000x1000 Manko-Novikov camera at full size (ray range of 64 image rows, the
    FP64 benchmark leg's launch) against the oracle on 48 sampled pixels."""
    tracer.set_spacetime(MN.M, MN.S, MN.Q)
    tracer.set_camera(MN.r0, MN.theta0, MN.fov_deg, MN.res_x, MN.res_y)
    tracer.set_options()
    first, count = 468 * 1000, 64 * 1000
    got = to_numpy(tracer.trace_range(first, count, 20000, 1.5e-4))
    torch.cuda.synchronize()
    pix = first + W.sample_pixels(count, 48, seed=5)
    ref = run_oracle(oracle, MN, 20000, 1.5e-4, pixels=pix)
    sub = {k: v[pix - first] for k, v in got.items()}
    assert_fp64_parity(sub, ref, what="mn full sampled")


# ----------------------------------------------------------------- determinism
@pytest.mark.parametrize("cam,n_steps", [(W.sub_camera(SCHW, 24, 20), 400000),
                                         (W.sub_camera(MN, 24, 16), 3000)])
def test_bitwise_independent_of_launch_shape(tracer, cam, n_steps):
    """Same bits for every block size, grid size and persistent vs one-ray-per-thread."""
    base = run_gpu(tracer, cam, n_steps, 1.5e-4)
    for opts in (dict(block_size=32, blocks_per_sm=1), dict(block_size=256, blocks_per_sm=2),
                 dict(block_size=64, flags=4)):
        other = run_gpu(tracer, cam, n_steps, 1.5e-4, **opts)
        for k in ("t", "r", "th", "ph", "status", "nsteps"):
            assert np.array_equal(other[k], base[k]), (opts, k)


# ----------------------------------------------------------------- edge cases
@pytest.mark.parametrize("rx,ry", [(1, 1), (1, 7), (7, 1), (33, 17)])
def test_degenerate_and_ragged_images(tracer, oracle, rx, ry):
    cam = W.sub_camera(MN, rx, ry)
    got = run_gpu(tracer, cam, 1500, 1.5e-4)
    ref = run_oracle(oracle, cam, 1500, 1.5e-4)
    assert_fp64_parity(got, ref, what=f"{rx}x{ry}")


@pytest.mark.parametrize("mode", [0, 1])
def test_zero_steps_returns_camera_state(tracer, mode):
    cam = W.sub_camera(MN, 5, 3)
    got = run_gpu(tracer, cam, 0, 1.5e-4, mode)
    assert np.all(got["status"] == 2) and np.all(got["nsteps"] == 0)
    assert np.all(got["r"] == cam.r0) and np.all(got["th"] == cam.theta0)
    assert np.all(got["t"] == 0) and np.all(got["ph"] == 0)


def test_compat_flags_match_oracle(tracer, oracle):
    """The listing's 0.1667 weights and v^phi = alpha camera, both sides."""
    cam = W.Camera(M=0.5, S=0.24, Q=0.0, r0=15.0, theta0=1.1, fov_deg=75.0, res_x=9, res_y=7)
    got = run_gpu(tracer, cam, 5000, 1.5e-4, flags=1 | 2)
    ref = run_oracle(oracle, cam, 5000, 1.5e-4, flags=1 | 2)
    assert_fp64_parity(got, ref, what="compat")


def test_invalid_arguments(g, tracer):
    lib, ctx = tracer.lib, tracer.ctx
    assert lib.gt_set_spacetime(ctx, 0.5, 0.25, 0.0) == -1    # |S| >= M^2
    assert lib.gt_set_spacetime(ctx, 0.5, 0.0, 1.0) == -1     # q != 0 needs S != 0
    assert lib.gt_set_spacetime(ctx, -1.0, 0.0, 0.0) == -1
    assert lib.gt_set_camera(ctx, 15.0, 0.0, 75.0, 4, 4) == -1
    assert lib.gt_set_camera(ctx, 15.0, 1.0, 180.0, 4, 4) == -1
    assert lib.gt_set_camera(ctx, 15.0, 1.0, 75.0, 0, 4) == -1
    buf = torch.empty(64, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert lib.gt_trace(ctx, 10, 1.5e-4, 0, p, p, p, p, None, None) == -2  # not configured
    assert lib.gt_set_spacetime(ctx, 0.5, 0.24, 0.0) == 0
    assert lib.gt_set_camera(ctx, 15.0, 1.0, 75.0, 4, 4) == 0
    assert lib.gt_trace(ctx, 10, 0.0, 0, p, p, p, p, None, None) == -1     # sp <= 0
    assert lib.gt_trace(ctx, -1, 1e-4, 0, p, p, p, p, None, None) == -1    # n_steps < 0
    assert lib.gt_trace(ctx, 10, 1e-4, 7, p, p, p, p, None, None) == -1    # bad mode
    assert lib.gt_trace(ctx, 10, 1e-4, 0, p + 4, p, p, p, None, None) == -1  # misaligned
    assert lib.gt_trace_range(ctx, 10, 7, 10, 1e-4, 0, p, p, p, p, None, None) == -1
    # camera inside the ergoregion (g_tt >= 0 at r0 = 0.9 on the equator of a = 0.96M)
    assert lib.gt_set_camera(ctx, 0.9, math.pi / 2, 75.0, 4, 4) == 0
    assert lib.gt_trace(ctx, 10, 1e-4, 0, p, p, p, p, None, None) == -1
    assert lib.gt_sync(ctx) == 0


def test_watchdog_stops_long_launch_and_context_survives(g, tracer, oracle):
    """A launch that would run for minutes is stopped by the device watchdog: the call
    returns GT_ERR_TIMEOUT, every ray carries a status, and the context keeps working."""
    cam = W.sub_camera(MN, 256, 256)
    tracer.set_spacetime(cam.M, cam.S, cam.Q)
    tracer.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tracer.set_options(timeout_seconds=0.2)
    with pytest.raises(g.GeotraceError) as e:
        out = tracer.alloc_outputs(cam.n_rays)
        out["status"].fill_(99)
        tracer.trace(500000, 1.5e-4, 0, out=out)
    assert e.value.code == -5
    st = out["status"].cpu().numpy()
    assert np.all(st <= 4) and (st == 4).sum() > 0
    small = W.sub_camera(MN, 6, 5)
    got = run_gpu(tracer, small, 800, 1.5e-4)  # options reset to defaults here
    ref = run_oracle(oracle, small, 800, 1.5e-4)
    assert_fp64_parity(got, ref, what="after timeout")


def test_host_api_matches_device_api(tracer):
    cam = W.sub_camera(MN, 19, 11)
    dev = run_gpu(tracer, cam, 2500, 1.5e-4)
    host = tracer.trace_host(2500, 1.5e-4, 0)
    for k in ("t", "r", "th", "ph", "status", "nsteps"):
        assert np.array_equal(np.asarray(host[k]), dev[k]), k


def test_batch_matches_single_camera_traces(tracer, oracle):
    """One persistent launch over uneven cameras equals tracing each camera alone
    (bitwise for an all-Kerr batch); a mixed Kerr + Manko-Novikov batch matches the oracle."""
    cams = [W.Camera(0.5, 0.1, 0.0, 12.0, 0.7, 75.0, 13, 9),
            W.Camera(0.5, 0.2475, 0.0, 20.0, 1.5, 60.0, 5, 17),
            W.Camera(0.5, 0.0, 0.0, 9.0, 1.2, 75.0, 21, 3)]
    out = to_numpy(tracer.trace_batch(cams, 3000, 1.5e-4, 0))
    torch.cuda.synchronize()
    off = 0
    for c in cams:
        single = run_gpu(tracer, c, 3000, 1.5e-4)
        for k in ("t", "r", "th", "ph", "status", "nsteps"):
            assert np.array_equal(out[k][off:off + c.n_rays], single[k]), k
        off += c.n_rays
    mixed = cams + [W.Camera(0.5, 0.24, 2.0, 15.0, 1.3, 75.0, 7, 6)]
    out = to_numpy(tracer.trace_batch(mixed, 3000, 1.5e-4, 0))
    torch.cuda.synchronize()
    off = 0
    for c in mixed:
        ref = run_oracle(oracle, c, 3000, 1.5e-4)
        sub = {k: v[off:off + c.n_rays] for k, v in out.items()}
        assert_fp64_parity(sub, ref, what="batch")
        off += c.n_rays


# ----------------------------------------------------------------- FP32-mixed
def test_mixed_literal_mn(tracer, oracle):
    cam = W.sub_camera(MN, 24, 16)
    got = run_gpu(tracer, cam, 20000, 1.5e-4, mode=1)
    ref = run_oracle(oracle, cam, 20000, 1.5e-4)
    rep = mixed_report(got, ref)
    assert rep["agree"] == 1.0 and rep["max_angle"] < 1e-4, rep


@pytest.mark.parametrize("cam,n_steps,r_switch", [(W.sub_camera(SCHW, 24, 20), 400000, 0.0),
                                                  (KERR, 500000, 0.0), (KERR, 500000, 1.5),
                                                  (W.sub_camera(MN, 12, 10), 500000, 0.0)])
def test_mixed_terminating_classification_and_angle(tracer, oracle, cam, n_steps, r_switch):
    """Terminating rays, FP32-mixed against the oracle: Kerr without FP64 zone (the
    default), Kerr with one, and Manko-Novikov with its default 4M zone."""
    got = run_gpu(tracer, cam, n_steps, 1.5e-4, mode=1, r_switch=r_switch)
    ref = run_oracle(oracle, cam, n_steps, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    rep = mixed_report(got, ref, exclude=band)
    assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, rep


def test_mixed_zone_double_float_and_fp64(g, tracer, oracle):
    """The FP32-mixed zone of Manko-Novikov with its field in double-float (the default)
    and in FP64 (GT_FLAG_ZONE_FP64): both meet the mixed-precision criteria against the
    oracle on terminating rays; the zone statistics count every zone evaluation as FP64
    with the flag and a minority without it; and the two runs differ (the double-float
    field ran)."""
    cam = W.sub_camera(MN, 12, 10)
    ref = run_oracle(oracle, cam, 500000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    outs, stats = {}, {}
    for name, flags in (("df", 0), ("f64", g.FLAG_ZONE_FP64)):
        outs[name] = run_gpu(tracer, cam, 500000, 1.5e-4, mode=1, flags=flags)
        stats[name] = tracer.zone_stats()
        rep = mixed_report(outs[name], ref, exclude=band)
        assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, (name, rep)
    steps, f64 = stats["f64"]
    assert steps > 0 and f64 == 4 * steps, stats
    steps_df, f64_df = stats["df"]
    assert steps_df > 0 and f64_df < 0.5 * 4 * steps_df, stats
    assert not np.array_equal(outs["df"]["th"], outs["f64"]["th"], equal_nan=True)


def test_zone_double_float_tracks_the_fp64_zone(g, tracer):
    """A camera inside the Manko-Novikov zone (listing's spacetime, r0 = 3.8M < 4M, 64x64,
    2,000 steps, FP32-mixed): every ray takes its first step in the FP32 kernel and all
    later ones in the zone kernel, so the zone statistics count rays x 1,999 steps, all
    of them in double-float by default and all in FP64 with GT_FLAG_ZONE_FP64.  From the
    same first step, the double-float zone's end states stay within 1e-12 (relative) of
    the FP64 zone's: the double-float field and stage arithmetic carry ~2^-48 per
    operation (measured: max 5.6e-14 over the 4,096 rays)."""
    cam = W.Camera(M=0.5, S=0.24, Q=2.0, r0=1.9, theta0=80 * W.DEG, fov_deg=75.0,
                   res_x=64, res_y=64)
    n = 2000
    outs, stats = {}, {}
    for name, flags in (("df", 0), ("f64", g.FLAG_ZONE_FP64)):
        outs[name] = run_gpu(tracer, cam, n, 1.5e-4, mode=1, flags=flags)
        stats[name] = tracer.zone_stats()
    assert stats["df"] == (cam.n_rays * (n - 1), 0), stats
    assert stats["f64"] == (cam.n_rays * (n - 1), 4 * cam.n_rays * (n - 1)), stats
    assert np.array_equal(outs["df"]["status"], outs["f64"]["status"])
    assert np.array_equal(outs["df"]["nsteps"], outs["f64"]["nsteps"])
    for k in ("t", "r", "th", "ph"):
        a, b = outs["df"][k], outs["f64"][k]
        rel = np.abs(a - b) / np.maximum(1.0, np.abs(b))
        assert np.all(np.isfinite(a)) and rel.max() <= 1e-12, (k, float(rel.max()))
    assert not np.array_equal(outs["df"]["r"], outs["f64"]["r"])  # the double-float zone ran


def test_mixed_precise_mn_multipole_tails(g, tracer, oracle):
    """GT_FLAG_PRECISE_MN (closed-form multipole tails in the FP32 field): Manko-Novikov
    terminating rays against the oracle -- the same classification, and end angles of
    escaped rays two orders of magnitude closer than the mixed-precision bound."""
    cam = W.sub_camera(MN, 12, 10)
    ref = run_oracle(oracle, cam, 500000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    got = run_gpu(tracer, cam, 500000, 1.5e-4, mode=1, flags=g.FLAG_PRECISE_MN)
    rep = mixed_report(got, ref, exclude=band)
    assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-5, rep
    plain = run_gpu(tracer, cam, 500000, 1.5e-4, mode=1)
    assert not np.array_equal(plain["th"], got["th"])  # the other field form ran


def test_mixed_reprojection_interval(tracer, oracle):
    """H = 0 re-projection of p_r (FP64, every K steps): with K = 16 (re-projecting
    hundreds of times per ray) and with K beyond the step cap (never), the mixed path
    meets the same classification and angle criteria; the two runs differ, so the
    re-projection ran."""
    cam = KERR
    ref = run_oracle(oracle, cam, 500000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    outs = {}
    for k in (16, 1 << 30):
        outs[k] = run_gpu(tracer, cam, 500000, 1.5e-4, mode=1, reproject_every=k)
        rep = mixed_report(outs[k], ref, exclude=band)
        assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, (k, rep)
    assert not np.array_equal(outs[16]["th"], outs[1 << 30]["th"])


def test_mixed_full_size_sampled(tracer, oracle):
    """The benchmark launch: 1000x1000 Manko-Novikov, 20,000 steps, FP32-mixed, against
    the oracle on 64 sampled pixels."""
    got = run_gpu(tracer, MN, 20000, 1.5e-4, mode=1)
    pix = W.sample_pixels(MN.n_rays, 64, seed=11)
    ref = run_oracle(oracle, MN, 20000, 1.5e-4, pixels=pix)
    sub = {k: v[pix] for k, v in got.items()}
    rep = mixed_report(sub, ref)
    assert rep["agree"] == 1.0 and rep["max_angle"] < 1e-4, rep
    for k in ("t", "r"):
        assert np.max(np.abs(sub[k] - ref[k]) / np.abs(ref[k])) < 1e-4


# ----------------------------------------------------------------- autotuner and graphs
def test_autotuner_picks_valid_shape_caches_it_and_keeps_bits(g, tracer, tmp_path):
    cam = W.sub_camera(MN, 96, 64)
    base = run_gpu(tracer, cam, 2500, 1.5e-4, mode=0)
    cache = str(tmp_path / "tune.txt")
    b, k, rpt, v = tracer.autotune(0, trial_rays=4096, trial_steps=200, cache_path=cache)
    assert b in (64, 128, 192, 256) and 1 <= k <= 8 and rpt == 1 and v > 0
    assert open(cache).read().count("|") == 1
    b2, k2, rpt2, v2 = tracer.autotune(0, trial_rays=4096, trial_steps=200, cache_path=cache)
    assert (b2, k2, rpt2) == (b, k, rpt)
    out = to_numpy(tracer.trace(2500, 1.5e-4, 0))  # tuned shape kept in the context
    torch.cuda.synchronize()
    for key in ("t", "r", "th", "ph", "status", "nsteps"):
        assert np.array_equal(out[key], base[key]), key


def test_two_rays_per_thread_is_bitwise_equal_and_tuned(g, tracer, tmp_path):
    """The FP32 rounds kernel with two rays per thread runs the same arithmetic per ray:
    bitwise equal to one ray per thread, for the literal workload and for terminating rays
    that park in and return from an FP64 zone; the autotuner searches it for FP32-mixed."""
    for cam, n_steps, rsw in ((W.sub_camera(MN, 24, 16), 20000, 0.0),
                              (KERR, 300000, 1.5), (W.sub_camera(MN, 10, 8), 300000, 0.0)):
        one = run_gpu(tracer, cam, n_steps, 1.5e-4, mode=1, r_switch=rsw)
        two = run_gpu(tracer, cam, n_steps, 1.5e-4, mode=1, r_switch=rsw, rays_per_thread=2)
        for k in ("t", "r", "th", "ph", "status", "nsteps"):
            assert np.array_equal(one[k], two[k]), (cam, k)
    cam = W.sub_camera(MN, 96, 64)
    tracer.set_spacetime(cam.M, cam.S, cam.Q)
    tracer.set_camera(cam.r0, cam.theta0, cam.fov_deg, cam.res_x, cam.res_y)
    tracer.set_options()
    b, k, rpt, v = tracer.autotune(1, trial_rays=4096, trial_steps=200,
                                   cache_path=str(tmp_path / "tune1.txt"))
    assert rpt in (1, 2) and v > 0
    assert open(str(tmp_path / "tune1.txt")).read().split("|")[1].split()[2] == str(rpt)


def test_graph_launch_replays_the_batch(g, tracer, oracle):
    """GT_FLAG_GRAPH: the batched trace replayed from a cached CUDA graph -- FP64 bitwise
    equal to the direct launch, twice in a row; FP32-mixed (rounds under a conditional
    WHILE node) bitwise equal to the host-driven rounds and within the mixed-precision
    criteria of FP64."""
    cams = [W.Camera(0.5, 0.1, 0.0, 12.0, 0.7, 75.0, 13, 9),
            W.Camera(0.5, 0.2475, 0.0, 20.0, 1.5, 60.0, 5, 17),
            W.Camera(0.5, 0.24, 0.0, 15.0, 80 * W.DEG, 30.0, 12, 10)]
    tracer.set_options()
    direct = to_numpy(tracer.trace_batch(cams, 300000, 1.5e-4, 0))
    # an explicit FP64 zone (Kerr has none by default) so that rays park and resume
    tracer.set_options(flags=g.FLAG_GRAPH, r_switch=1.5)
    out = tracer.alloc_outputs(sum(c.n_rays for c in cams))
    for _ in range(2):
        for v in out.values():
            v.zero_()
        got = to_numpy(tracer.trace_batch(cams, 300000, 1.5e-4, 0, out=out))
        torch.cuda.synchronize()
        for key in ("t", "r", "th", "ph", "status", "nsteps"):
            assert np.array_equal(got[key], direct[key]), key
    mixed = to_numpy(tracer.trace_batch(cams, 300000, 1.5e-4, 1))
    torch.cuda.synchronize()
    tracer.set_options(r_switch=1.5)
    rounds = to_numpy(tracer.trace_batch(cams, 300000, 1.5e-4, 1))
    torch.cuda.synchronize()
    for key in ("t", "r", "th", "ph", "status", "nsteps"):  # same kernels, same bits
        assert np.array_equal(mixed[key], rounds[key]), key
    off = 0
    for c in cams:
        sl = slice(off, off + c.n_rays)
        band = neighbour_band(direct["status"][sl], c.res_x, c.res_y)
        rep = mixed_report({k: v[sl] for k, v in mixed.items()},
                           {k: v[sl] for k, v in direct.items()}, exclude=band)
        assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, rep
        off += c.n_rays


def test_pixel_list_trace_matches_full_image(tracer):
    """gt_trace_pixels (compact outputs) reproduces the full-image result bitwise, in both
    modes (FP32-mixed parks and resumes rays by their list position)."""
    cam = W.sub_camera(W.SCHW_64, 40, 30)
    pix = W.sample_pixels(cam.n_rays, 173, seed=9)
    for mode, n_steps in ((0, 400000), (1, 400000)):
        # explicit FP64 zone: mixed rays park and resume (Kerr has none by default)
        full = run_gpu(tracer, cam, n_steps, 1.5e-4, mode=mode, r_switch=1.5)
        sub = to_numpy(tracer.trace_pixels(torch.tensor(pix, device="cuda"), n_steps, 1.5e-4, mode))
        torch.cuda.synchronize()
        for k in ("t", "r", "th", "ph", "status", "nsteps"):
            assert np.array_equal(sub[k], full[k][pix]), (mode, k)


# ----------------------------------------------------------------- per-ray initial data
def kerr_rmin(M, a, r0, p, th0, n_grid=4000):
    """min over r in (r_+, r0] of R(r)/(E^2 r^4), R the Kerr radial potential of the ray's
    constants of motion E = -p_t, L = p_phi and Carter constant K (dense geometric grid)."""
    E, L = -p[0], p[3]
    K = p[2] ** 2 + np.cos(th0) ** 2 * (-a * a * E * E + L * L / np.sin(th0) ** 2)
    rp = M + np.sqrt(M * M - a * a)
    r = np.exp(np.linspace(np.log(rp * 1.0001), np.log(r0), n_grid))
    R = (E * (r * r + a * a) - a * L) ** 2 - (r * r - 2 * M * r + a * a) * ((L - a * E) ** 2 + K)
    return float(np.min(R / (E * E * r ** 4)))


def _oracle_rays(oracle, M, r0, al, be, spin, q, th0, n_steps, sp):
    from concurrent.futures import ThreadPoolExecutor

    def one(k):
        S = spin[k] * M * M
        q0, p0 = oracle.camera_dir(M, S, q[k], r0, th0[k], al[k], be[k])
        qe, pe, st, ns, ms = oracle.trace_ray(M, S, q[k], q0, p0, r0, n_steps, sp)
        return qe, st, ns, ms, p0
    with ThreadPoolExecutor(max_workers=16) as ex:
        res = list(ex.map(one, range(len(al))))
    out = {k: np.array([x[0][i] for x in res]) for i, k in enumerate(("t", "r", "th", "ph"))}
    out["status"] = np.array([x[1] for x in res], np.uint8)
    out["nsteps"] = np.array([x[2] for x in res], np.uint32)
    out["min_sin"] = np.array([x[3] for x in res])
    out["p0"] = np.array([x[4] for x in res])
    return out


def test_per_ray_trace_matches_oracle(tracer, oracle):
    """gt_trace_rays (the surrogate's label generator: spacetime and camera per ray) against
    the oracle's per-ray camera and integrator, FP64: 200 rays over the training ranges
    (a/M in [0, 0.99], inclination 5-90 deg, 40 of them Manko-Novikov with q in [-2, 2]),
    element-wise 1e-9 with equal status and step count at a 3,000-step cap; then the Kerr
    rays to termination, outside the photon-ring band and axis crossings."""
    M, r0, sp = 0.5, 15.0, 1.5e-4
    al, be, spin, q, th0 = W.surrogate_samples(200, seed=77, M=M, r0=r0)
    rng = np.random.Generator(np.random.PCG64(78))
    spin[:40] = rng.uniform(0.1, 0.99, 40)  # Manko-Novikov needs S != 0
    q[:40] = rng.uniform(-2.0, 2.0, 40)
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in (al, be, spin, q, th0)]
    got = to_numpy(tracer.trace_rays(*dev, M, r0, 3000, sp, 0))
    torch.cuda.synchronize()
    ref = _oracle_rays(oracle, M, r0, al, be, spin, q, th0, 3000, sp)
    assert_fp64_parity(got, ref, what="per-ray 3000")
    kerr = slice(40, 200)
    args = [x[kerr] for x in (al, be, spin, q, th0)]
    got = to_numpy(tracer.trace_rays(*[d[kerr] for d in dev], M, r0, 400000, sp, 0))
    torch.cuda.synchronize()
    ref = _oracle_rays(oracle, M, r0, *args, 400000, sp)
    band = np.array([abs(kerr_rmin(M, a * M, r0, p, t)) < 1e-3
                     for a, p, t in zip(args[2], ref["p0"], args[4])]) | (ref["min_sin"] < 1e-3)
    assert_fp64_parity(got, ref, exclude=band, what="per-ray terminating")
    st = ref["status"][~band]
    assert (st == oracle.HORIZON).sum() > 5 and (st == oracle.ESCAPED).sum() > 50


@pytest.mark.parametrize("mode", [0, 1])
def test_overflowing_step_is_nonfinite_and_keeps_the_camera_state(tracer, oracle, mode):
    """A finite but enormous step_precision makes the first step overflow: every ray ends
    as NONFINITE after 1 step with its initial state, as in the oracle."""
    for cam in (W.Camera(0.5, 0.0, 0.0, 15.0, 1.2, 75.0, 5, 5),
                W.Camera(0.5, 0.24, 0.0, 15.0, 1.2, 75.0, 5, 5),
                W.Camera(0.5, 0.24, 2.0, 15.0, 1.2, 75.0, 5, 5)):
        got = run_gpu(tracer, cam, 100, 1e200, mode=mode)
        ref = run_oracle(oracle, cam, 100, 1e200)
        assert np.all(ref["status"] == oracle.NONFINITE) and np.all(ref["nsteps"] == 1)
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["nsteps"], ref["nsteps"])
        for k in ("t", "r", "th", "ph"):
            assert np.max(np.abs(got[k] - ref[k])) <= 1e-15 * max(1.0, np.max(np.abs(ref[k]))), k


# ----------------------------------------------------------------- Manko-Novikov zoo
ZOO = [(q, S) for q in (-2.0, 0.0, 2.0) for S in (0.1 * 0.25, 0.98 * 0.25)]


@pytest.mark.parametrize("q,S", ZOO)
def test_fp64_mn_zoo(tracer, oracle, q, S):
    """The spacetimes of the paper's shadow zoo (q in {-2, 0, 2} x S in {0.1M^2, 0.98M^2};
    q = 0 is Kerr): FP64 against the oracle on a 10x8 image from the listing's viewpoint
    r0 = 16M, 80 deg, FOV 60 deg, to a 250,000-step cap (rays escape, fall in or stay
    trapped), outside the chaotic boundary band and axis crossings; then FP32-mixed with
    the same classification and 1e-3 rad.  Manko-Novikov has chaotic regions (Sec. 5): rays
    whose oracle end state moves by more than 1e-10 under a 1e-13 change of the initial p_r
    are excluded as well (their two correct FP64 integrations part beyond 1e-9)."""
    cam = W.Camera(M=0.5, S=S, Q=q, r0=8.0, theta0=80 * W.DEG, fov_deg=60.0, res_x=10, res_y=8)
    got = run_gpu(tracer, cam, 250000, 1.5e-4)
    ref = run_oracle(oracle, cam, 250000, 1.5e-4, want_min_sin=True)
    band = neighbour_band(ref["status"], cam.res_x, cam.res_y) | (ref["min_sin"] < 1e-3)
    band |= sensitive_rays(oracle, cam, 250000, 1.5e-4, ref)
    assert band.sum() < 3 * cam.res_x * cam.res_y // 4
    assert_fp64_parity(got, ref, exclude=band, what=f"zoo q={q} S={S}")
    mixed = run_gpu(tracer, cam, 250000, 1.5e-4, mode=1)
    rep = mixed_report(mixed, ref, exclude=band)
    assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, rep
