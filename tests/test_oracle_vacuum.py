"""Vacuum pin of the oracle's Manko-Novikov metric: R_{mu nu} = 0.

Sec. 2.2.3 states that the Manko-Novikov spacetime is a stationary, axisymmetric
vacuum solution of Einstein's equations.  The Ricci tensor is built here from the
oracle's lower metric by nested Richardson finite differences -- a route that shares
nothing with the oracle's formulas -- so this pins f, omega and gamma (including the
coefficients that vanish on the axis and at infinity, which the flatness and
regularity pins cannot see).  A planted mistake in gamma' shows the test's reach.
"""
import numpy as np
import pytest

M, S = 0.5, 0.24


def _d1(fun, x, h):
    a = (fun(x + h) - fun(x - h)) / (2 * h)
    b = (fun(x + h / 2) - fun(x - h / 2)) / h
    return (4 * b - a) / 3


def _christoffel(glow, r, th, h=1e-3):
    g = glow(r, th)
    gi = np.linalg.inv(g)
    dg = np.zeros((4, 4, 4))
    dg[1] = _d1(lambda x: glow(x, th), r, h * r)
    dg[2] = _d1(lambda x: glow(r, x), th, h)
    # Gamma^a_{mn} = 1/2 g^{ab} (d_m g_{bn} + d_n g_{bm} - d_b g_{mn})
    t = dg.transpose(1, 0, 2) + dg.transpose(1, 2, 0) - dg  # [b, m, n]
    return 0.5 * np.einsum("ab,bmn->amn", gi, t)


def _ricci(glow, r, th, h2=2e-3):
    G = _christoffel(glow, r, th)
    dG = np.zeros((4, 4, 4, 4))
    dG[1] = _d1(lambda x: _christoffel(glow, x, th), r, h2 * r)
    dG[2] = _d1(lambda x: _christoffel(glow, r, x), th, h2)
    # R_{mn} = d_a G^a_{mn} - d_n G^a_{ma} + G^a_{ab} G^b_{mn} - G^a_{nb} G^b_{ma}
    R = (np.einsum("aamn->mn", dG) - np.einsum("nama->mn", dG)
         + np.einsum("aab,bmn->mn", G, G) - np.einsum("anb,bma->mn", G, G))
    return R, np.max(np.abs(G)) ** 2


PTS = [(2.3, 0.7), (1.3, 1.2), (4.0, 0.4), (6.0, 2.2)]


@pytest.mark.parametrize("Q", [0.0, 2.0, -1.0])
def test_ricci_flat(oracle, Q):
    glow = lambda r, th: oracle.metric_lower(M, S, Q, r, th)  # noqa: E731
    for r, th in PTS:
        R, scale = _ricci(glow, r, th)
        assert np.max(np.abs(R)) < 1e-6 * scale, (r, th, np.max(np.abs(R)) / scale)


def test_ricci_detects_planted_gamma_mistake(oracle):
    """Change the 3 beta^2/(2 R^6) coefficient of gamma' to beta^2/R^6 (a plausible
    misreading) by rescaling g_rr and g_theta_theta: the vacuum test must fail."""
    Q = 2.0
    F0 = oracle.mn_fields(M, S, Q, 3.0, 1.0)
    k, beta = F0["k"], F0["beta"]

    def glow(r, th):
        g = oracle.metric_lower(M, S, Q, r, th).copy()
        x, y = (r - M) / k, np.cos(th)
        R = np.sqrt(x * x + y * y - 1)
        u = x * y / R
        P2, P3 = (3 * u * u - 1) / 2, (5 * u ** 3 - 3 * u) / 2
        wrong = np.exp(2 * (-0.5) * beta ** 2 / R ** 6 * (P3 * P3 - P2 * P2))
        g[1, 1] *= wrong
        g[2, 2] *= wrong
        return g

    worst = max(np.max(np.abs(R)) / s for R, s in (_ricci(glow, r, th) for r, th in PTS))
    assert worst > 1e-3
