"""The synthetic workloads carry the values the paper prints (tests/golden/paper_parameters.json)."""
import json
import math
import os

import numpy as np

from paper_2310_15183_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def g(key):
    return GOLD[key]["value"]


def test_mn_workload_uses_listing_constants():
    c = W.MN_1000
    assert (c.M, c.S, c.Q) == (g("mass_M"), g("spin_S"), g("quadrupole_q"))
    assert (c.fov_deg, c.res_x, c.res_y) == (g("fov_deg"), g("res_x"), g("res_y"))
    assert W.WORKLOADS["mn1000"].step_precision == g("step_precision")
    assert W.WORKLOADS["mn1000_T"].n_steps == g("n_steps_listing")


def test_batch_cameras_seeded_and_in_range():
    a = W.batch_cameras()
    b = W.batch_cameras()
    assert a == b and len(a) == 64
    for c in a:
        assert 128 <= c.res_x <= 1024 and c.res_x == c.res_y
        assert 0 <= c.S / c.M <= 0.99 * c.M
        assert 5 * W.DEG <= c.theta0 <= 90 * W.DEG
        assert 15 * c.M <= c.r0 <= 50 * c.M
    assert W.batch_cameras(seed=1) != a


def test_pixel_sample_and_surrogate_draws():
    s = W.sample_pixels(10 ** 6, 500, 7)
    assert s.size == 500 and np.all(np.diff(s) > 0) and s[-1] < 10 ** 6
    al, be, a, q, th = W.surrogate_samples(1000)
    V = math.tan(0.5 * 75 * W.DEG) / 15.0
    assert np.all(np.abs(be) <= V) and np.all(q == 0) and np.all((a >= 0) & (a <= 0.99))
