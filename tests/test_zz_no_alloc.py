"""gt_trace_batch_noalloc -- the batched trace for callers that cannot allocate device
memory (its scratch is a static device array of the library) -- must give the same
rays as gt_trace_batch, call after call.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes

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


def _descs(g, cams):
    arr = (g.CameraDesc * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = g.CameraDesc(c.M, c.S, c.Q, c.r0, c.theta0, c.fov_deg, c.res_x, c.res_y)
    return arr


def _noalloc(g, cams, n_steps, sp, mode):
    lib = g.load_library()
    n = sum(c.n_rays for c in cams)
    out = {k: torch.full((n,), -7.0, dtype=torch.float64, device="cuda") for k in ("t", "r", "th", "ph")}
    out["status"] = torch.full((n,), 99, dtype=torch.uint8, device="cuda")
    out["nsteps"] = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.gt_trace_batch_noalloc(0, ctypes.c_void_p(stream.cuda_stream), _descs(g, cams),
                                    len(cams), int(n_steps), float(sp), int(mode),
                                    *[ctypes.c_void_p(out[k].data_ptr())
                                      for k in ("t", "r", "th", "ph", "status", "nsteps")])
    assert rc == 0
    torch.cuda.synchronize()
    return to_numpy(out)


def _with_context(g, cams, n_steps, sp, mode):
    tr = g.Tracer(0)
    try:
        out = tr.trace_batch(cams, n_steps, sp, mode)
        torch.cuda.synchronize()
        return to_numpy(out)
    finally:
        tr.close()


CALLS = [
    # two FP64 calls in a row with different batches: the second must not see the
    # first's queue counter or descriptors
    ([W.Camera(0.5, 0.1, 0.0, 12.0, 0.7, 75.0, 13, 9),
      W.Camera(0.5, 0.24, 2.0, 15.0, 1.3, 75.0, 7, 6),
      W.Camera(0.5, 0.0, 0.0, 9.0, 1.2, 75.0, 21, 3)], 3000),
    ([W.Camera(0.5, 0.2475, 0.0, 20.0, 1.5, 60.0, 5, 17),
      W.Camera(0.5, 0.24, 0.0, 15.0, 80 * W.DEG, 30.0, 12, 10)], 400000),
]


def test_noalloc_batch_matches_allocating_batch_twice_in_a_row(g):
    for cams, n_steps in CALLS:
        got = _noalloc(g, cams, n_steps, 1.5e-4, 0)
        want = _with_context(g, cams, n_steps, 1.5e-4, 0)
        assert_fp64_parity(got, want, what="noalloc vs gt_trace_batch")
        assert np.all(got["status"] <= 3)


def test_noalloc_mixed_mode_within_mixed_tolerance(g):
    """FP32-mixed runs its FP64 zone inline here, so it is compared with the
    reduced-precision criteria: same classification, end angles within 1e-3 rad."""
    cams, n_steps = CALLS[1]
    got = _noalloc(g, cams, n_steps, 1.5e-4, 1)
    want = _with_context(g, cams, n_steps, 1.5e-4, 0)
    band = np.concatenate([neighbour_band(want["status"][o:o + c.n_rays], c.res_x, c.res_y)
                           for c, o in zip(cams, np.cumsum([0] + [c.n_rays for c in cams]))])
    rep = mixed_report(got, want, exclude=band)
    assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, rep


def test_noalloc_mixed_mode_inline_fp64_zone(g):
    """A Manko-Novikov camera (whose 4M FP64 zone the FP32-mixed kernel enters inline
    here, converting the ray state to FP64 and back) batched with a Kerr camera, so the
    per-camera kernel variant runs; against gt_trace_batch's FP64 result with the
    reduced-precision criteria outside the chaotic boundary band."""
    cams = [W.Camera(0.5, 0.24, 2.0, 15.0, 80 * W.DEG, 30.0, 10, 8),
            W.Camera(0.5, 0.24, 0.0, 15.0, 80 * W.DEG, 30.0, 9, 7)]
    n_steps = 200000
    got = _noalloc(g, cams, n_steps, 1.5e-4, 1)
    want = _with_context(g, cams, n_steps, 1.5e-4, 0)
    offs = np.cumsum([0] + [c.n_rays for c in cams])
    band = np.concatenate([neighbour_band(want["status"][o:o + c.n_rays], c.res_x, c.res_y)
                           for c, o in zip(cams, offs)])
    rep = mixed_report(got, want, exclude=band)
    assert rep["agree"] >= 0.999 and rep["max_angle_escaped"] <= 1e-3, rep
    mn = slice(0, cams[0].n_rays)
    # the MN rays did reach the zone: some were captured or are still inside it
    assert np.any((want["status"][mn] == 1) | (want["r"][mn] < 4 * cams[0].M))


def test_noalloc_rejects_batches_beyond_its_static_scratch(g):
    lib = g.load_library()
    cams = [W.Camera(0.5, 0.1, 0.0, 12.0, 0.7, 75.0, 2, 2)] * 65
    buf = torch.empty(4 * 65, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = lib.gt_trace_batch_noalloc(0, None, _descs(g, cams), 65, 100, 1.5e-4, 0,
                                    p, p, p, p, None, None)
    assert rc == -1
