"""Timelike orbits (Sec. 3.2.1 "Orbits"): the oracle's periapsis precession against the
closed-form quadrature of Schwarzschild geodesics.

With M = 1 units, an equatorial bound orbit of semi-latus rectum p and eccentricity e
(r = p M / (1 + e cos chi)) has L^2 = p^2 M^2 / (p - 3 - e^2) and
E^2 = ((p - 2)^2 - 4 e^2) / (p (p - 3 - e^2)), and its azimuth advances per radial period
by Delta phi = 2 int_0^pi sqrt(p / (p - 6 - 2 e cos chi)) dchi (Cutler, Kennefick &
Poisson 1994) -- 2 pi plus the relativistic precession, ~6 pi M/p for large p.
"""
import math

import numpy as np
import pytest

M = 0.5


def orbit_constants(p, e):
    L = p * M / math.sqrt(p - 3 - e * e)
    E = math.sqrt(((p - 2) ** 2 - 4 * e * e) / (p * (p - 3 - e * e)))
    return E, L


def delta_phi(p, e):
    from scipy.integrate import quad
    v, _ = quad(lambda c: math.sqrt(p / (p - 6 - 2 * e * math.cos(c))), 0.0, math.pi,
                epsabs=1e-14, epsrel=1e-13)
    return 2 * v


@pytest.mark.parametrize("p,e", [(12.0, 0.2), (20.0, 0.5), (9.0, 0.3)])
def test_periapsis_precession_matches_quadrature(oracle, p, e):
    E, L = orbit_constants(p, e)
    rp = p * M / (1 + e)
    q0 = np.array([0.0, rp, math.pi / 2, 0.0])
    p0 = np.array([-E, 0.0, 0.0, L])
    assert abs(oracle.hamiltonian(M, 0.0, 0.0, q0, p0) + 0.5) < 1e-13  # timelike, H = -1/2
    sp = 2e-3
    ra = p * M / (1 - e)
    period = 2 * math.pi * ((rp + ra) / 2) ** 1.5 / math.sqrt(M) * 2.0  # > one radial period
    n = int(period / sp)
    path = oracle.trace_path(M, 0.0, 0.0, q0, p0, 1e9, n, sp)
    pr = path[:, 5]
    # the next periapsis: p_r crosses zero from below after the apoapsis
    k = np.flatnonzero((pr[:-1] < 0) & (pr[1:] >= 0))
    assert k.size >= 1
    i = k[0]
    # quadratic through three states around the crossing: phi as a function of p_r
    sl = slice(i - 1, i + 2)
    coef = np.polyfit(pr[sl], path[sl, 3], 2)
    phi_peri = np.polyval(coef, 0.0)
    want = delta_phi(p, e)
    assert abs(phi_peri - want) < 1e-7 * want, (phi_peri, want)
    assert want - 2 * math.pi > 0.1 * (6 * math.pi / p)  # a precession is there to measure
