"""Pins of the oracle's exit tests against the radial null geodesic of Schwarzschild.

A radial light ray (L = 0, theta = pi/2) in Schwarzschild has E = -p_t conserved and
dr/dtau = +-E exactly (the null condition gives p_r = +-E/f with f = 1 - 2M/r and
dq^r/dtau = f p_r), while dq^t/dtau = E/f.  The step of the listing's propagation
kernel, h = sp/|dq^t/dtau| = sp f(r)/E, therefore depends on r alone, and the exact
flow moves r by +-E h per step: the step at which each exit test first fires follows
from the scalar recurrence r_{n+1} = r_n +- 6 w sp f(r_n), w the RK4 weight.  RK4 on
the full 8-dimensional system reproduces that count, so each of the paper's exit
constants -- the horizon factor 3e-5 on the step, the escape radius 1.5 r0 and the
listing's 0.1667 weight -- is pinned to the step: a factor 10 in the horizon constant
moves the capture by ~15,000 steps, 1.4 r0 instead of 1.5 r0 the escape by ~7,000, and
the 0.1667 weight the escape by 7 steps.

The last test pins the NONFINITE branch the paper does not have (a step whose result is
not finite ends the ray and keeps its last finite state).
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
M = GOLD["mass_M"]["value"]
SP = GOLD["step_precision"]["value"]
HORIZON = GOLD["horizon_factor"]["value"]
ESCAPE = GOLD["escape_factor"]["value"]
W_LISTING = GOLD["rk4_weight_listing"]["value"]
R0 = 10.0  # camera at 20M


def f(r):
    return 1.0 - 2.0 * M / r


def radial_state(sign, r):
    """Radial null ray at (0, r, pi/2, 0) with E = 1; sign -1 ingoing, +1 outgoing."""
    return np.array([0.0, r, math.pi / 2, 0.0]), np.array([-1.0, sign / f(r), 0.0, 0.0])


def exit_step(sign, r_start, horizon=HORIZON, escape=ESCAPE, w=1.0 / 6.0, sp=SP):
    """(status, step) of the first exit of the scalar recurrence of the exact flow,
    tested in the listing's order: escape first, then the collapsed step."""
    r, n = r_start, 0
    while True:
        h = sp * f(r)
        r += sign * 6.0 * w * h
        n += 1
        if r > escape * r_start:
            return 0, n
        if h < sp * horizon:
            return 1, n


def test_horizon_exit_step_of_radial_infall(oracle):
    q, p = radial_state(-1, R0)
    _, _, st, ns, _ = oracle.trace_ray(M, 0.0, 0.0, q, p, R0, 10 ** 7, SP)
    want_st, want_n = exit_step(-1, R0)
    assert st == oracle.HORIZON == want_st
    assert abs(ns - want_n) <= 1, (ns, want_n)
    # the constant is what fixes the step: a factor of 10 either way is far off
    for other in (HORIZON * 10, HORIZON / 10):
        assert abs(ns - exit_step(-1, R0, horizon=other)[1]) > 5000


def test_escape_exit_step_of_radial_outgoing(oracle):
    q, p = radial_state(+1, R0)
    qe, _, st, ns, _ = oracle.trace_ray(M, 0.0, 0.0, q, p, R0, 10 ** 7, SP)
    want_st, want_n = exit_step(+1, R0)
    assert st == oracle.ESCAPED == want_st
    assert abs(ns - want_n) <= 1, (ns, want_n)
    # no interpolation to the escape radius: the end state is the first one beyond it
    assert ESCAPE * R0 < qe[1] < ESCAPE * R0 + 2 * SP
    assert abs(ns - exit_step(+1, R0, escape=1.4)[1]) > 1000


@pytest.mark.parametrize("sign", [+1, -1])
def test_listing_weight_shifts_the_exit_step(oracle, sign):
    """The listing's 0.1667 weights (6 x 0.1667 = 1.0002) advance r 0.02 % faster per step."""
    q, p = radial_state(sign, R0)
    _, _, st, ns, _ = oracle.trace_ray(M, 0.0, 0.0, q, p, R0, 10 ** 7, SP,
                                       flags=oracle.FLAG_COMPAT_WEIGHTS)
    want_st, want_n = exit_step(sign, R0, w=W_LISTING)
    exact_n = exit_step(sign, R0)[1]
    assert st == want_st and abs(ns - want_n) <= 1, (ns, want_n)
    assert exact_n - want_n >= 5  # the weight is visible in the step count


@pytest.mark.parametrize("S,Q", [(0.0, 0.0), (0.24, 0.0), (0.24, 2.0)])
def test_nonfinite_step_keeps_last_finite_state(oracle, S, Q):
    """A step whose result is not finite ends the ray as NONFINITE at that step and keeps
    the state before it: (a) a state on the axis with L != 0 (1/sin^2 theta = inf in the
    first stage); (b) a finite step_precision so large that the first step overflows."""
    q = np.array([0.0, 10.0, 0.0, 0.0])
    p = np.array([-1.0, 0.1, 0.0, 0.5])
    qe, pe, st, ns, _ = oracle.trace_ray(M, S, Q, q, p, 10.0, 100, SP)
    assert st == oracle.NONFINITE and ns == 1
    assert np.array_equal(qe, q) and np.array_equal(pe, p)
    q0, p0 = oracle.camera_ray(M, S, Q, 15.0, 1.2, 75.0, 5, 5, 2, 1)
    for sp in (1e200, 1.7e308):
        qe, pe, st, ns, _ = oracle.trace_ray(M, S, Q, q0, p0, 15.0, 100, sp)
        assert st == oracle.NONFINITE and ns == 1
        assert np.array_equal(qe, q0) and np.array_equal(pe, p0)
