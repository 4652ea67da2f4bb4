"""Pins of the oracle's RK4 propagation (Sec. 3.1.2 and the listing's propagation
kernel) against closed forms, exact quadratures, conservation laws, symmetry and
convergence order."""
import numpy as np
import pytest
from scipy import integrate

M = 0.5
BC = 3 * np.sqrt(3) * M  # Schwarzschild critical impact parameter


# --------------------------------------------------------------------------- helpers
def _carter(a, q, p):
    """Carter constant of a null geodesic in Kerr (Sec. 2.2.2 mentions it)."""
    th = q[2]
    E, L = -p[0], p[3]
    return p[2] ** 2 + np.cos(th) ** 2 * (-a * a * E * E + L * L / np.sin(th) ** 2)


def _schw_quadratures(b, u_in, u_out):
    """Exact equatorial Schwarzschild null orbit: total phi sweep and |t| elapsed going
    from u_in = 1/r_start inward to the turning point and back out to u_out = 1/r_end.
    (du/dphi)^2 = 1/b^2 - u^2 (1 - 2 M u);  dt/dphi = 1/(b u^2 (1 - 2 M u))."""
    roots = np.roots([2 * M, -1.0, 0.0, 1.0 / b ** 2])
    real = np.sort(roots[np.abs(roots.imag) < 1e-12].real)
    um = min(x for x in real if x > u_in)
    others = [x for x in real if x != um]
    assert len(others) == 2

    def g(u):  # (1/b^2 - u^2 + 2Mu^3)/(um - u) = -2M (u - u1)(u - u2), no cancellation
        return -2 * M * (u - others[0]) * (u - others[1])

    phi = t = 0.0
    for lo in (u_in, u_out):
        phi += integrate.quad(lambda u: 1.0 / np.sqrt(g(u)), lo, um, weight="alg",
                              wvar=(0, -0.5), epsabs=1e-14, epsrel=1e-14, limit=200)[0]
        t += integrate.quad(lambda u: 1.0 / (b * u * u * (1 - 2 * M * u) * np.sqrt(g(u))),
                            lo, um, weight="alg", wvar=(0, -0.5), epsabs=1e-13, epsrel=1e-14,
                            limit=200)[0]
    return phi, t


# --------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("S,Q", [(0.24, 0.0), (0.24, 2.0)])
def test_energy_and_angular_momentum_bitwise_constant(oracle, S, Q):
    """p_t and p_phi have identically zero rates (the metric depends on r, theta only),
    so E = -p_t and L_z = p_phi never change, bit for bit."""
    q0, p0 = oracle.camera_ray(M, S, Q, 15.0, 80 * np.pi / 180, 75.0, 32, 32, 17, 14)
    path = oracle.trace_path(M, S, Q, q0, p0, 15.0, 3000, 1.5e-4)
    assert len(path) == 3001
    assert np.all(path[:, 4] == p0[0]) and np.all(path[:, 7] == p0[3])


@pytest.mark.parametrize("S,Q", [(0.24, 0.0), (0.24, 2.0), (0.0, 0.0)])
def test_hamiltonian_drift_is_fourth_order(oracle, S, Q):
    """H = 0 is not preserved by RK4; its drift over a fixed coordinate-time span
    shrinks 16x per halving of step_precision (order 4).  A derivative inconsistent
    with the metric would leave an O(1) drift that does not shrink."""
    q0, p0 = oracle.camera_ray(M, S, Q, 15.0, 80 * np.pi / 180, 75.0, 64, 64, 36, 32)
    drifts = []
    for sp in (0.08, 0.04, 0.02):
        n = int(round(16 / sp))
        qe, pe, _, _, _ = oracle.trace_ray(M, S, Q, q0, p0, 15.0, n, sp)
        drifts.append(abs(oracle.hamiltonian(M, S, Q, qe, pe)))
    r1, r2 = drifts[0] / drifts[1], drifts[1] / drifts[2]
    assert 11 < r1 < 22 and 11 < r2 < 22, drifts


def test_carter_constant_conserved_kerr(oracle):
    """Kerr keeps the Carter constant (Sec. 2.2.2); its RK4 drift is fourth order and
    tiny at the paper's step_precision."""
    S = 0.24
    a = S / M
    q0, p0 = oracle.camera_ray(M, S, 0.0, 15.0, 80 * np.pi / 180, 75.0, 64, 64, 42, 27)
    K0 = _carter(a, q0, p0)
    drifts = []
    for sp in (0.08, 0.04):
        qe, pe, _, _, _ = oracle.trace_ray(M, S, 0.0, q0, p0, 15.0, int(round(16 / sp)), sp)
        drifts.append(abs(_carter(a, qe, pe) - K0))
    assert 11 < drifts[0] / drifts[1] < 22
    qe, pe, st, ns, _ = oracle.trace_ray(M, S, 0.0, q0, p0, 15.0, 400000, 1.5e-4)
    assert st == oracle.ESCAPED
    assert abs(_carter(a, qe, pe) - K0) < 1e-10 * abs(K0)
    assert abs(oracle.hamiltonian(M, S, 0.0, qe, pe)) < 1e-11


# --------------------------------------------------------------------------- closed forms
def test_schwarzschild_equatorial_end_state_matches_quadrature(oracle):
    """Equatorial Schwarzschild rays (a 1-row camera at theta0 = pi/2, r0 = 20M): the
    oracle's end phi and t equal the exact orbit integrals to 1e-9, with the end
    radius taken from the oracle; the classification follows b vs 3 sqrt(3) M."""
    r0, resX = 10.0, 15
    out = oracle.trace_image(M, 0.0, 0.0, r0, np.pi / 2, 75.0, resX, 1, 400000, 1.5e-4,
                             want_p=True)
    checked = 0
    for i in range(resX):
        p = out["p"][i]
        b = abs(p[3] / p[0])
        assert abs(out["th"][i] - np.pi / 2) < 1e-12
        if abs(b - BC) < 1e-3 * M:
            continue
        if b < BC:
            assert out["status"][i] == oracle.HORIZON
            continue
        assert out["status"][i] == oracle.ESCAPED
        assert 1.5 * r0 < out["r"][i] < 1.5 * r0 + 1e-3
        phi, t = _schw_quadratures(b, 1.0 / r0, 1.0 / out["r"][i])
        assert abs(abs(out["ph"][i]) - phi) < 1e-9, (i, out["ph"][i], phi)
        assert np.sign(out["ph"][i]) == np.sign(i - (resX - 1) / 2)
        assert abs(-out["t"][i] - t) < 1e-9 * t
        checked += 1
    assert checked >= 6


def test_weak_field_deflection(oracle):
    """Far from the hole the bending is 4M/b to first order (finite-distance form,
    per leg (M/b)(sqrt(1-w^2) + sqrt((1-w)/(1+w)) + w/sqrt(1-w^2)), w = b/R, which
    tends to 2M/b per leg as R -> infinity)."""
    r0, fov = 2000.0, 6.0
    out = oracle.trace_image(M, 0.0, 0.0, r0, np.pi / 2, fov, 9, 1, 200000, 0.25,
                             pixels=[8, 6], want_p=True)
    for k in range(2):
        p = out["p"][k]
        b = abs(p[3] / p[0])
        assert out["status"][k] == oracle.ESCAPED and b > 100 * M
        dphi = 0.0
        for R in (r0, out["r"][k]):
            w = b / R
            dphi += np.pi / 2 - np.arcsin(w) + (M / b) * (
                np.sqrt(1 - w * w) + np.sqrt((1 - w) / (1 + w)) + w / np.sqrt(1 - w * w))
        # first-order formula; the O((M/b)^2) remainder is ~ (15 pi/4)(M/b)^2
        assert abs(abs(out["ph"][k]) - dphi) < 20 * (M / b) ** 2


def test_photon_sphere_instability(oracle):
    """A photon on the r = 3M circular orbit stays there, and a small radial offset
    grows like cosh(t / (3 sqrt(3) M)) (the orbit's Lyapunov rate in coordinate time)."""
    r = 3 * M * (1 + 1e-9)
    q = np.array([0.0, r, np.pi / 2, 0.0])
    f = 1 - 2 * M / r
    L = BC
    # p_t from H = 0 with p_r = p_theta = 0:  p_t^2 / f = L^2 / r^2
    p = np.array([-np.sqrt(f) * L / r, 0.0, 0.0, L])
    sp = 1e-3
    path = oracle.trace_path(M, 0.0, 0.0, q, p, 100.0, 60000, sp)
    t, dr = path[:, 0], path[:, 1] - 3 * M
    lam = 1 / (3 * np.sqrt(3) * M)
    i1, i2 = np.searchsorted(t, 20.0), np.searchsorted(t, 40.0)
    assert abs(dr[i1]) < 1e-4
    rate = np.log(abs(dr[i2]) / abs(dr[i1])) / (t[i2] - t[i1])
    assert abs(rate / lam - 1) < 0.02, rate / lam


@pytest.mark.slow
def test_kerr_classification_from_radial_potential(oracle):
    """Kerr (a = 0.96M, theta0 = 80 deg): HORIZON exactly for the rays whose radial
    potential has no turning point between r_+ and r0 (exact, from the initial
    constants of motion); rays within a thin band of the critical curve are excluded."""
    S, r0, th0 = 0.24, 15.0, 80 * np.pi / 180
    a = S / M
    rp = M + np.sqrt(M * M - a * a)
    res, fov = 9, 30.0
    pix = [(i, j) for j in range(res) for i in range(res)]
    out = oracle.trace_image(M, S, 0.0, r0, th0, fov, res, res, 500000, 1.5e-4,
                             pixels=[j * res + i for i, j in pix], want_p=True)
    P = np.polynomial.polynomial
    n_cap = n_esc = 0
    for k, (i, j) in enumerate(pix):
        q0, p0 = oracle.camera_ray(M, S, 0.0, r0, th0, fov, res, res, i, j)
        E, L = -p0[0], p0[3]
        K = p0[2] ** 2 + np.cos(th0) ** 2 * (-a * a * E * E + L * L / np.sin(th0) ** 2)
        # R(r) = (E r^2 + (a^2 E - a L))^2 - (r^2 - 2 M r + a^2)((L - a E)^2 + K)
        W = [a * a * E - a * L, 0.0, E]
        Rpoly = P.polysub(P.polymul(W, W), P.polymul([a * a, -2 * M, 1.0], [(L - a * E) ** 2 + K]))
        rs = np.linspace(rp * 1.0001, r0, 20001)
        Rv = P.polyval(rs, Rpoly) / (E * E * rs ** 4)
        if abs(Rv.min()) < 1e-3:
            continue  # photon-ring band
        captured = Rv.min() > 0
        assert out["status"][k] == (oracle.HORIZON if captured else oracle.ESCAPED), (i, j)
        n_cap += captured
        n_esc += not captured
        assert np.all(out["p"][k][[0, 3]] == p0[[0, 3]])
    assert n_cap >= 10 and n_esc >= 10, (n_cap, n_esc)


@pytest.mark.parametrize("S,Q", [(0.24, 2.0), (0.24, 0.0)])
def test_equatorial_mirror_symmetry_of_image(oracle, S, Q):
    """theta0 = pi/2: pixel rows j and resY-1-j end mirrored in theta, equal otherwise."""
    resX, resY = 3, 4
    out = oracle.trace_image(M, S, Q, 15.0, np.pi / 2, 75.0, resX, resY, 4000, 1.5e-4)
    for j in range(resY):
        for i in range(resX):
            k, km = j * resX + i, (resY - 1 - j) * resX + i
            assert abs(out["th"][k] + out["th"][km] - np.pi) < 1e-11
            for key in ("t", "r", "ph"):
                assert abs(out[key][k] - out[key][km]) < 1e-11 * max(1, abs(out[key][k]))
            assert out["status"][k] == out["status"][km]


# --------------------------------------------------------------------------- brute force
def _end_at_radius(oracle, S, Q, q0, p0, r0, sp):
    """End state of an escaping ray interpolated (cubic Hermite in the step parameter)
    to exactly r = 1.5 r0, removing the step-size dependent overshoot."""
    _, _, st, n, _ = oracle.trace_ray(M, S, Q, q0, p0, r0, 10 ** 7, sp)
    assert st == oracle.ESCAPED
    qa, pa, _, _, _ = oracle.trace_ray(M, S, Q, q0, p0, r0, n - 1, sp)
    qb, pb, _, _, _ = oracle.trace_ray(M, S, Q, qa, pa, r0, 1, sp)
    dqa, _ = oracle.vector_field(M, S, Q, qa, pa)
    dqb, _ = oracle.vector_field(M, S, Q, qb, pb)
    h = abs(sp / dqa[0])
    target = 1.5 * r0

    def herm(s, y0, y1, d0, d1):
        return ((2 * s ** 3 - 3 * s ** 2 + 1) * y0 + (s ** 3 - 2 * s ** 2 + s) * h * d0
                + (-2 * s ** 3 + 3 * s ** 2) * y1 + (s ** 3 - s ** 2) * h * d1)

    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if herm(mid, qa[1], qb[1], dqa[1], dqb[1]) < target:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)
    return np.array([herm(s, qa[m], qb[m], dqa[m], dqb[m]) for m in (0, 2, 3)])


@pytest.mark.parametrize("S,Q", [(0.24, 2.0), (0.24, 0.0)])
def test_small_step_brute_force_converges(oracle, S, Q):
    """The run at step_precision sp agrees with a 16x finer brute-force run, both
    interpolated to r = 1.5 r0, to O(sp^4) (tiny images, as the oracle must finish)."""
    r0, th0 = 15.0, 80 * np.pi / 180
    for i, j in [(13, 5), (2, 9), (15, 15)]:
        q0, p0 = oracle.camera_ray(M, S, Q, r0, th0, 75.0, 16, 16, i, j)
        coarse = _end_at_radius(oracle, S, Q, q0, p0, r0, 2e-3)
        fine = _end_at_radius(oracle, S, Q, q0, p0, r0, 2e-3 / 16)
        assert np.max(np.abs(coarse - fine)) < 1e-8, (i, j, coarse - fine)


def test_compat_weights_are_first_order_off(oracle):
    """The listing's 0.1667 weights sum to 1.0002: the end state moves by O(2e-4)
    relative to exact 1/6 -- a check that the flag is wired and that 1/6 is the default."""
    q0, p0 = oracle.camera_ray(M, 0.24, 0.0, 15.0, 1.2, 75.0, 8, 8, 6, 2)
    qa, _, _, _, _ = oracle.trace_ray(M, 0.24, 0.0, q0, p0, 15.0, 2000, 1.5e-4)
    qb, _, _, _, _ = oracle.trace_ray(M, 0.24, 0.0, q0, p0, 15.0, 2000, 1.5e-4,
                                      oracle.FLAG_COMPAT_WEIGHTS)
    dt = abs(qa[0] - qb[0]) / abs(qa[0])
    assert 1e-4 < dt < 4e-4


def test_maxsteps_and_zero_steps(oracle):
    """n_steps = 0 returns the initial state as MAXSTEPS; the literal 2000-step run of
    the 64x64 Schwarzschild camera stops every ray as MAXSTEPS near t = -0.3."""
    q0, p0 = oracle.camera_ray(M, 0.0, 0.0, 10.0, np.pi / 2, 75.0, 64, 64, 3, 60)
    qe, pe, st, n, _ = oracle.trace_ray(M, 0.0, 0.0, q0, p0, 10.0, 0, 1.5e-4)
    assert st == oracle.MAXSTEPS and n == 0 and np.all(qe == q0) and np.all(pe == p0)
    out = oracle.trace_image(M, 0.0, 0.0, 10.0, np.pi / 2, 75.0, 64, 64, 2000, 1.5e-4,
                             pixels=np.arange(0, 4096, 97))
    assert np.all(out["status"] == oracle.MAXSTEPS) and np.all(out["nsteps"] == 2000)
    assert np.all(np.abs(out["t"] + 0.3) < 1e-3)
