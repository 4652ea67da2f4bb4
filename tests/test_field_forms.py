"""The Manko-Novikov field's reverse-sweep derivatives (what the kernels run) against the
forward dual-number derivatives of the same expressions, on the host: both are exact to
rounding, so in double they agree to ~1e-13 (~1e-12 for the FP32 kernels' closed-form
multipole tails, against dual numbers that keep the direct differences); in float the
reverse sweep must be no less accurate than the forward form, and both must overflow at
the same points."""
import json
import os
import subprocess

import pytest

from paper_2310_15183_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_reverse_sweep_matches_dual_numbers(tmp_path):
    exe = str(tmp_path / "field_forms")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + cuda_inc,
                    os.path.join(HERE, "field_forms.cpp"), "-o", exe], check=True)
    res = json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    assert res["points"] >= 3000 and res["points_f32"] >= 3000
    assert res["reverse_vs_forward_f64"] < 1e-11, res
    # the closed-form multipole tails of the FP32 kernels, evaluated in double
    assert res["tail_form_vs_forward_f64"] < 1e-10, res
    assert res["finite_mismatch"] == 0, res
    assert res["f32_vs_f64"] < 2e-3 and res["f32_vs_f64"] <= 1.5 * res["f32_forward_vs_f64"], res


def test_multipole_tail_closed_form_against_the_series():
    """The closed forms the FP32 kernels use with GT_FLAG_PRECISE_MN for the Manko-Novikov
    sums, Sa - 1 = -t^3 N(t)/(1 + s Q(t)) and Sb + 1 = -t^3 N(-t)/(1 + s' Q(-t)), against the
    Legendre series they stand for, summed term by term to convergence (t = 1/R,
    u = x y / R, R^2 = x^2 + y^2 - 1; the full sums are 1/(x - y) and 1/(x + y))."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(2310))
    for _ in range(200):
        x = 1.0 + rng.uniform(0.5, 30.0)
        y = rng.uniform(-0.999, 0.999)
        R = np.sqrt(x * x + y * y - 1.0)
        t, u = 1.0 / R, x * y / R
        P = [1.0, u]
        for l in range(1, 400):
            P.append(((2 * l + 1) * u * P[l] - l * P[l - 1]) / (l + 1))
        terms = np.array([P[l] * t ** (l + 1) for l in range(401)])
        alt = terms * (-1.0) ** np.arange(401)
        # the series do sum to 1/(x - y) and 1/(x + y)
        assert abs(terms.sum() - 1.0 / (x - y)) < 1e-12 * (1.0 / (x - y))
        assert abs(alt.sum() - 1.0 / (x + y)) < 1e-12 * (1.0 / (x + y))
        Ea_series = -(x - y) * terms[3:].sum()  # Sa - 1
        Eb_series = (x + y) * alt[3:].sum()     # Sb + 1 (Sb = -(x + y) sum_{l<=2} (-1)^l ...)
        P2, P3 = P[2], P[3]
        c4 = P2 * P2 - 4 * u * u * P2 + 2 * P2 + u * u
        c5 = 2 * u * P2 * (1 - P2)
        c6 = P2 * P2
        N = lambda tt: 2 * P3 - c4 * tt - c5 * tt ** 2 - c6 * tt ** 3
        Q = lambda tt: 1 + u * tt + P2 * tt ** 2
        Ea = -t ** 3 * N(t) / (1 + (x - y) * t * Q(t))
        Eb = -t ** 3 * N(-t) / (1 + (x + y) * t * Q(-t))
        scale = t ** 4 * (x + 1)
        assert abs(Ea - Ea_series) < 1e-10 * scale, (x, y, Ea, Ea_series)
        assert abs(Eb - Eb_series) < 1e-10 * scale, (x, y, Eb, Eb_series)


def test_compensated_update_error_bound(tmp_path):
    """The FP32-mixed state update (low part first, then Fast2Sum) stays within
    sum_k (u |d_k| + u^2 |hi_k|) of the exact sum -- including a momentum driven through
    zero, where hi is the smaller term -- and keeps |lo| <= ulp(hi)/2 (<= ulp(hi) at a zero
    crossing, where Fast2Sum's precondition can fail for a step)."""
    exe = str(tmp_path / "compensated_sum")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off",
                    os.path.join(HERE, "compensated_sum.cpp"), "-o", exe], check=True)
    res = json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    for name, (ratio, lo) in res.items():
        assert ratio <= 1.0, (name, res)
        assert lo <= (1.0 if name == "zero_crossing" else 0.5), (name, res)


def test_double_float_zone_arithmetic_and_rates(tmp_path):
    """The double-float arithmetic of the FP32-mixed zone (csrc/df.cuh) against long double:
    sum, sum under cancellation, product, reciprocal and inverse square root within a few
    u^2 (u = 2^-24) of the result, exp within 2^-45 over [-69, 87], the stage rotation of
    sin/cos within 4 u^2 for angles up to 1/16; and the Manko-Novikov
    rates evaluated in double-float (zone_df.cuh) at random points of the zone of eight
    spacetimes, where its range check accepts them, against long double: within ~64x the
    error of the same evaluation in double at the median and the 99th percentile (the
    ratio of the two precisions, 2^5), below 1e-6 of the largest rate everywhere, with the
    range check accepting most of the zone and of the listing's trapped-ray shell; and the
    Kerr rates in double-float over r_+ < r < 5M likewise."""
    exe = str(tmp_path / "df_arith")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-I" + cuda_inc,
                    os.path.join(HERE, "df_arith.cpp"), "-o", exe], check=True)
    res = json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    u2 = 2.0 ** -48
    assert res["add"] <= 3 * u2 and res["add_cancel"] <= 3 * u2, res
    assert res["mul"] <= 5 * u2, res
    assert res["rcp"] <= 4 * u2 and res["rsqrt"] <= 6 * u2, res
    assert res["exp"] <= 2.0 ** -45, res
    assert res["rotate_abs"] <= 4 * u2 and res["rotate_refused"] == 0, res
    assert res["zone_points_df"] >= 0.85 * res["zone_points"], res
    assert res["shell_points_df"] >= 0.85 * res["shell_points"], res
    assert res["rates_df_median"] <= 64 * res["rates_f64_median"], res
    assert res["rates_df_p99"] <= 64 * res["rates_f64_p99"], res
    assert res["rates_df_max"] < 1e-6, res
    # Kerr (a zone set with r_switch): double-float keeps ~1e-14 of the largest rate at the
    # median; within 10 % of r_+ the cancellation in Delta = r (r - 2M) + a^2, which FP64
    # takes through one exactly rounded FMA, costs it up to ~1e-10
    assert res["kerr_points"] >= 70000, res
    assert res["kerr_df_median"] <= 64 * res["kerr_f64_median"], res
    assert res["kerr_df_p99"] < 1e-11 and res["kerr_df_max"] < 1e-9, res
