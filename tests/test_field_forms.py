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
