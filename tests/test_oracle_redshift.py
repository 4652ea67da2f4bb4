"""Pins of the oracle's ring emitter and redshift (Sec. 3.3.3), its paper-numerics
variants (forward-difference derivatives, float32 I/O) and the explicit Euler
integrator of Sec. 3.1.1.

Closed forms used (Bardeen, Press & Teukolsky 1972, equatorial circular orbits of Kerr,
prograde, G = c = 1):
    E = (r^1.5 - 2 M r^0.5 + a M^0.5) / (r^0.75 sqrt(r^1.5 - 3 M r^0.5 + 2 a M^0.5)),
    L = M^0.5 (r^2 - 2 a M^0.5 r^0.5 + a^2) / (r^0.75 sqrt(r^1.5 - 3 M r^0.5 + 2 a M^0.5)),
    Omega = M^0.5 / (r^1.5 + a M^0.5),   u^t = (r^1.5 + a M^0.5) / (r^0.75 sqrt(...)),
and the redshift of a photon of impact parameter b = L_ph/E_ph reaching a static
observer at r0 (equatorial): z = u^t (1 - b Omega) sqrt(-g_tt(r0)).
"""
import math

import numpy as np
import pytest

M = 0.5


def bpt(a, r):
    s = math.sqrt(r ** 1.5 - 3 * M * r ** 0.5 + 2 * a * M ** 0.5)
    E = (r ** 1.5 - 2 * M * r ** 0.5 + a * M ** 0.5) / (r ** 0.75 * s)
    L = M ** 0.5 * (r * r - 2 * a * M ** 0.5 * r ** 0.5 + a * a) / (r ** 0.75 * s)
    Om = M ** 0.5 / (r ** 1.5 + a * M ** 0.5)
    ut = (r ** 1.5 + a * M ** 0.5) / (r ** 0.75 * s)
    return E, L, Om, ut


@pytest.mark.parametrize("a", [0.0, 0.24, 0.45, 0.49])
def test_ring_emitter_is_the_bardeen_circular_orbit(oracle, a):
    """Equatorial Kerr: the emitter momentum (from d_r g^{mu nu} and the quadratic for
    p_phi) equals (-E, 0, 0, L) of the prograde circular orbit, for r outside the photon
    orbit; and it is a unit timelike covector."""
    for r in (3.1, 4.0, 6.0, 10.0, 25.0):
        if r ** 1.5 - 3 * M * r ** 0.5 + 2 * a * M ** 0.5 <= 0:
            continue
        E, L, _, _ = bpt(a, r)
        p = oracle.circular_orbit(M, a * M, 0.0, r, math.pi / 2)
        assert abs(p[0] + E) < 1e-12 and abs(p[3] - L) < 1e-11 * max(1, L), (a, r, p, E, L)
        assert p[1] == 0 and p[2] == 0
        g = oracle.metric_upper(M, a * M, 0.0, r, math.pi / 2)
        assert abs(p @ g @ p + 1.0) < 1e-12


def test_ring_emitter_of_manko_novikov_reduces_to_kerr(oracle):
    """At q -> 0 the Manko-Novikov emitter tends to the Kerr one (q = 1e-9, complex-step
    derivatives) and at q = 2 it is still a unit timelike prograde orbit."""
    S = 0.24
    for r in (4.0, 8.0):
        pk = oracle.circular_orbit(M, S, 0.0, r, math.pi / 2)
        pm = oracle.circular_orbit(M, S, 1e-9, r, math.pi / 2)
        assert np.max(np.abs(pk - pm)) < 1e-7
        p2 = oracle.circular_orbit(M, S, 2.0, r, math.pi / 2)
        g = oracle.metric_upper(M, S, 2.0, r, math.pi / 2)
        assert abs(p2 @ g @ p2 + 1.0) < 1e-12 and p2[3] > 0


@pytest.mark.parametrize("a", [0.0, 0.45])
def test_redshift_closed_form(oracle, a):
    """A photon of impact parameter b at the ring (equatorial, any radial momentum
    consistent with H = 0) is shifted by z = u^t (1 - b Omega) sqrt(-g_tt(r0))."""
    r0, th0 = 15.0, math.pi / 2
    gl0 = oracle.metric_lower(M, a * M, 0.0, r0, th0)
    for r in (4.0, 7.0, 12.0):
        _, _, Om, ut = bpt(a, r)
        for b in (-6.0, 0.0, 2.5, 5.0):
            # momentum (p_t, p_r, 0, p_phi) with p_t = 1 (the backward ray), L = b, H = 0
            g = oracle.metric_upper(M, a * M, 0.0, r, math.pi / 2)
            pt, pph = 1.0, -b
            rest = g[0, 0] * pt * pt + 2 * g[0, 3] * pt * pph + g[3, 3] * pph * pph
            if rest >= 0:
                continue
            pr = math.sqrt(-rest / g[1, 1])
            z = oracle.redshift(M, a * M, 0.0, r0, th0, [0, r, math.pi / 2, 0], [pt, pr, 0, pph])
            want = ut * (1 - b * Om) * math.sqrt(-gl0[0, 0])
            assert abs(z - want) < 1e-12 * want, (r, b, z, want)


def test_ring_hit_of_radial_infall(oracle):
    """A radial ray falling onto a ring of outer radius r_out ends as DISK at the first
    step with r <= r_out (recurrence of the exact flow, as in the exit-constant pins),
    and its redshift is the b = 0 closed form."""
    sp, r0, r_out = 1.5e-4, 10.0, 6.0
    f = lambda r: 1 - 2 * M / r
    out = oracle.trace_image_disk(M, 0.0, 0.0, r0, math.pi / 2, 1e-6, 1, 1, 10 ** 7, sp,
                                  3.0, r_out, 0.1)
    r, n = r0, 0
    while r > r_out:
        r -= 6 * (1 / 6) * sp * f(r)
        n += 1
    assert out["status"][0] == oracle.DISK and abs(int(out["nsteps"][0]) - n) <= 1
    ut = 1 / math.sqrt(1 - 3 * M / out["r"][0])
    assert abs(out["z"][0] - ut * math.sqrt(f(r0))) < 1e-9


def test_forward_difference_derivatives_are_close_to_exact(oracle):
    """The listing's forward differences (delta = 1e-8) differ from the exact derivatives
    by O(delta) truncation plus rounding amplified by 1/delta (~1e-8 relative in the
    rates); over 2,000 far-field steps the end states differ by 1e-12 to 1e-9 -- not zero
    (the derivatives are different), not more than the rates' error allows."""
    for (S, Q) in ((0.24, 0.0), (0.24, 2.0)):
        q, p = oracle.camera_ray(M, S, Q, 15.0, 1.2, 75.0, 5, 5, 2, 1)
        exact = oracle.trace_ray(M, S, Q, q, p, 15.0, 2000, 1.5e-4)
        fd = oracle.trace_ray(M, S, Q, q, p, 15.0, 2000, 1.5e-4, flags=oracle.FLAG_FD_DERIVS)
        rel = np.max(np.abs(fd[0] - exact[0]) / np.maximum(1, np.abs(exact[0])))
        assert 1e-14 < rel < 1e-6, rel


def test_float32_io_rounds_arguments_and_outputs(oracle):
    """With float32 I/O the outputs are float32 values and the run equals the double one
    started from the float32-rounded state of the float32-rounded spacetime."""
    S = 0.24  # not a float32 number
    out = oracle.trace_image(M, S, 0.0, 15.0, 1.2, 75.0, 3, 3, 500, 1.5e-4,
                             flags=oracle.FLAG_F32_IO)
    for k in ("t", "r", "th", "ph"):
        assert np.array_equal(out[k], out[k].astype(np.float32).astype(np.float64))
    S32 = float(np.float32(S))
    q, p = oracle.camera_ray(M, S32, 0.0, 15.0, 1.2, 75.0, 3, 3, 1, 1)
    q32, p32 = q.astype(np.float32).astype(np.float64), p.astype(np.float32).astype(np.float64)
    qe = oracle.trace_ray(M, S32, 0.0, q32, p32, 15.0, 500, 1.5e-4)[0]
    assert np.array_equal(qe.astype(np.float32).astype(np.float64),
                          np.array([out[k][4] for k in ("t", "r", "th", "ph")]))


def test_euler_is_first_order_and_rk4_fourth(oracle):
    """Drift of the Hamiltonian H = 1/2 g^{mu nu} p_mu p_nu (exactly -1/2 along the flow)
    over a fixed span of coordinate time on a timelike Schwarzschild orbit: halving the
    step halves Euler's drift (first order, Sec. 3.1.1) and cuts RK4's by at least 2^3.7
    (fourth order, Sec. 3.1.2; ~2^4.7 is measured at these steps)."""
    r = 12.0
    f = 1 - 2 * M / r
    L = math.sqrt(M * r) / math.sqrt(1 - 3 * M / r) * 1.1  # a slightly eccentric orbit
    E = math.sqrt(f * (1 + L * L / (r * r)))
    q = [0.0, r, math.pi / 2, 0.0]
    p = [-E, 0.0, 0.0, L]
    assert abs(oracle.hamiltonian(M, 0.0, 0.0, q, p) + 0.5) < 1e-14
    T = 3000.0  # coordinate time (each step advances t by about sp)

    def drift(sp, flags):
        qe, pe, st, _, _ = oracle.trace_ray(M, 0.0, 0.0, q, p, 1e9, int(round(T / sp)), sp,
                                            flags=flags)
        assert st == oracle.MAXSTEPS
        return abs(oracle.hamiltonian(M, 0.0, 0.0, qe, pe) + 0.5)

    euler = math.log2(drift(0.1, oracle.FLAG_EULER) / drift(0.05, oracle.FLAG_EULER))
    rk4 = math.log2(drift(4.0, 0) / drift(2.0, 0))
    assert abs(euler - 1.0) < 0.1 and rk4 > 3.7, (euler, rk4)
