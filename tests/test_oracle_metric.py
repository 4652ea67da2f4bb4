"""Pins of the oracle's spacetimes (Sec. 2.2) against facts other than its own formulas.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong
sign, a swapped index, a mis-read garbled formula) fails it.
"""
import numpy as np
import pytest

M, S = 0.5, 0.24

# points outside the horizon, off the axis
PTS = [(2.3, 0.7), (10.0, 1.2), (1.5, 0.3), (4.0, 1.5707963267948966), (25.0, 2.8), (1.2, 1.9)]


def test_kerr_a0_is_schwarzschild(oracle):
    """Kerr with S = 0 is the textbook Schwarzschild metric (Eq. schwMetric)."""
    for r, th in PTS:
        g = oracle.metric_lower(M, 0.0, 0.0, r, th)
        f = 1.0 - 2.0 * M / r
        want = np.diag([-f, 1.0 / f, r * r, (r * np.sin(th)) ** 2])
        np.testing.assert_allclose(g, want, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("Q", [0.0, 2.0, -2.0])
def test_inverse_is_inverse(oracle, Q):
    """g_{mu nu} g^{nu sigma} = delta (lower and upper metric are written independently)."""
    for r, th in PTS:
        if Q != 0.0 and r < 1.2:
            continue
        gl = oracle.metric_lower(M, S, Q, r, th)
        gu = oracle.metric_upper(M, S, Q, r, th)
        np.testing.assert_allclose(gl @ gu, np.eye(4), atol=1e-12)


def _richardson_fd(fun, x, h):
    """Central differences with one Richardson step: error O(h^4)."""
    d1 = (fun(x + h) - fun(x - h)) / (2 * h)
    d2 = (fun(x + h / 2) - fun(x - h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("Q", [0.0, 2.0])
def test_derivatives_three_routes(oracle, Q):
    """d_r, d_theta g^{mu nu}: the integrator's route (Kerr: hand-derived closed form,
    Manko-Novikov: complex step) agrees with Richardson-extrapolated finite differences
    of the metric values, and for Kerr also with complex step."""
    for r, th in PTS:
        if Q != 0.0 and r < 1.2:
            continue
        d = oracle.dmetric_upper(M, S, Q, r, th, 0)
        fd_r = _richardson_fd(lambda x: oracle.metric_upper(M, S, Q, x, th), r, 1e-3 * r)
        fd_t = _richardson_fd(lambda x: oracle.metric_upper(M, S, Q, r, x), th, 1e-3)
        scale = np.max(np.abs(d)) + 1.0
        np.testing.assert_allclose(d[1], fd_r, atol=2e-8 * scale)
        np.testing.assert_allclose(d[2], fd_t, atol=2e-8 * scale)
        assert np.all(d[0] == 0) and np.all(d[3] == 0)
        if Q == 0.0:
            dcs = oracle.dmetric_upper(M, S, Q, r, th, 1)
            np.testing.assert_allclose(d, dcs, rtol=1e-12, atol=1e-13 * scale)


def test_mn_at_q0_is_kerr(oracle):
    """Manko-Novikov with q = 0 reduces exactly to Kerr (Sec. 2.2.3: the deviation q
    is measured from Kerr).  This pins the Kerr g_{t phi} sign reading, B as a sum of
    squares and the gamma' reading all at once."""
    for s in (0.05, 0.24, -0.2, 0.2499):
        for r, th in PTS:
            gk = oracle.metric_upper(M, s, 0.0, r, th)
            gm = oracle.mn_metric_upper(M, s, 0.0, r, th)
            np.testing.assert_allclose(gm, gk, rtol=1e-11, atol=1e-13)
            gkl = oracle.metric_lower(M, s, 0.0, r, th)
            gml = oracle.mn_metric_lower(M, s, 0.0, r, th)
            np.testing.assert_allclose(gml, gkl, rtol=1e-11, atol=1e-13)


def test_mn_constants_match_kerr_horizon(oracle):
    """k = sqrt(M^2 - a^2): the Manko-Novikov horizon x = 1 sits at Kerr's r_+ = M + k."""
    for s in (0.05, 0.24, -0.2):
        F = oracle.mn_fields(M, s, 2.0, 5.0, 1.0)
        a = s / M
        assert abs(F["k"] - np.sqrt(M * M - a * a)) < 1e-15
        assert abs(F["beta"] - 2.0 * M ** 3 / F["k"] ** 3) < 1e-12 * F["beta"]


@pytest.mark.parametrize("Q", [2.0, -2.0, 0.5])
def test_mn_asymptotically_flat(oracle, Q):
    """f -> 1 - 2M/r, omega -> 0, e^{2 gamma} -> 1 far away (a literal product B would
    give f -> -1/(2 alpha y))."""
    for th in (0.4, 1.1, 2.5):
        for r in (1e3, 1e5):
            F = oracle.mn_fields(M, S, Q, r, th)
            assert abs(F["f"] - (1.0 - 2.0 * M / r)) < 10 * (M / r) ** 2
            assert abs(F["omega"]) < 10 * M * M / r
            assert abs(F["e2gamma"] - 1.0) < 10 * (M / r) ** 2


@pytest.mark.parametrize("Q", [2.0, -2.0])
def test_mn_axis_regular(oracle, Q):
    """e^{2 gamma} = 1 on the symmetry axis (elementary flatness).  The printed
    gamma' without the (-1)^{2-l} reading gives e^{2 gamma} ~ 1e-317 there."""
    for r in (1.5, 3.0, 20.0):
        for th in (1e-7, np.pi - 1e-7):
            F = oracle.mn_fields(M, S, Q, r, th)
            assert abs(F["e2gamma"] - 1.0) < 1e-9


@pytest.mark.parametrize("Q", [2.0, -2.0])
def test_mn_equatorial_reflection(oracle, Q):
    """The spacetime is reflection symmetric about the equator."""
    for r, th in PTS:
        if r < 1.2:
            continue
        g1 = oracle.metric_upper(M, S, Q, r, th)
        g2 = oracle.metric_upper(M, S, Q, r, np.pi - th)
        np.testing.assert_allclose(g1, g2, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("Q", [2.0, -2.0, 0.7])
def test_mn_quadrupole_shift(oracle, Q):
    """q is the quadrupole deviation from Kerr (Sec. 2.2.3): the mass quadrupole moves
    by -q M^3, so far away f_q - f_0 = 2 q M^3 P_2(cos theta)/r^3 + O(r^-4).  The sign
    also fixes the paper's statement that q > 0 is oblate and q < 0 prolate."""
    for th in (0.3, 1.2, 2.0):
        c = np.cos(th)
        P2 = (3 * c * c - 1) / 2

        def coef(r):
            d = oracle.mn_fields(M, S, Q, r, th)["f"] - oracle.mn_fields(M, S, 0.0, r, th)["f"]
            return d * r ** 3 / (2 * P2)

        lim = 2 * coef(2000.0) - coef(1000.0)  # remove the 1/r correction
        assert abs(lim - Q * M ** 3) < 2e-4 * abs(Q) * M ** 3
