"""Pins of the oracle's camera (appendix listing initial-data block, Sec. 3.3.1)."""
import numpy as np
import pytest

CASES = [  # (M, S, Q, r0, theta0)
    (0.5, 0.0, 0.0, 10.0, np.pi / 2),
    (0.5, 0.24, 2.0, 15.0, 80 * np.pi / 180),
    (0.5, 0.2475, 0.0, 20.0, 0.3),
    (0.5, 0.24, -2.0, 12.0, 2.0),
]


@pytest.mark.parametrize("M,S,Q,r0,th0", CASES)
def test_initial_momentum_is_null_and_normalised(oracle, M, S, Q, r0, th0):
    """H(q0, p0) = 0 (light-like, Sec. 3.3.1) and v^t = g^{t nu} p_nu = -1 (the
    rescaling of Sec. 3.3.1), checked with the inverse metric, which the camera
    itself never uses."""
    resX, resY = 7, 5
    for i in range(resX):
        for j in range(resY):
            q, p = oracle.camera_ray(M, S, Q, r0, th0, 75.0, resX, resY, i, j)
            assert list(q) == [0.0, r0, th0, 0.0]
            gu = oracle.metric_upper(M, S, Q, r0, th0)
            v = gu @ p
            assert abs(v[0] + 1.0) < 1e-13
            assert abs(0.5 * p @ gu @ p) < 1e-13 * (p @ p)


@pytest.mark.parametrize("M,S,Q,r0,th0", CASES)
def test_pixel_directions_are_the_listing_linspaces(oracle, M, S, Q, r0, th0):
    """v^theta/(-v^r) and v^phi sin(theta0)/(-v^r) are numpy.linspace(-V, V, resY)[j]
    and numpy.linspace(-H, H, resX)[i] with V = tan(FOV/2)/r0, H = atan(tan V resX/resY)."""
    fov, resX, resY = 75.0, 9, 4
    V = np.tan(0.5 * fov / 180 * np.pi) / r0
    H = np.arctan(np.tan(V) * resX / resY)
    al, be = np.linspace(-H, H, resX), np.linspace(-V, V, resY)
    gu = oracle.metric_upper(M, S, Q, r0, th0)
    for i in range(resX):
        for j in range(resY):
            _, p = oracle.camera_ray(M, S, Q, r0, th0, fov, resX, resY, i, j)
            v = gu @ p
            assert v[1] < 0
            assert abs(v[2] / -v[1] - be[j]) < 1e-13
            assert abs(v[3] * np.sin(th0) / -v[1] - al[i]) < 1e-13


def test_flat_space_limit(oracle):
    """With M -> 0 the quadratic has the Minkowski root T = -sqrt(1 + r0^2 (beta^2 + alpha^2))."""
    M, r0, th0, fov, res = 1e-14, 7.0, 1.1, 60.0, 5
    V = np.tan(0.5 * fov / 180 * np.pi) / r0
    for i, j in [(0, 0), (2, 3), (4, 1)]:
        q, p = oracle.camera_ray(M, 0.0, 0.0, r0, th0, fov, res, res, i, j)
        al, be = np.linspace(-V, V, res)[i], np.linspace(-V, V, res)[j]
        T = -np.sqrt(1 + r0 ** 2 * (be ** 2 + al ** 2))
        want = np.array([1.0, -1.0 / -T, r0 ** 2 * be / -T, r0 ** 2 * np.sin(th0) * al / -T])
        np.testing.assert_allclose(p, want, rtol=1e-12, atol=1e-14)


def test_single_pixel_is_on_axis_of_view(oracle):
    """A 1x1 camera looks straight at the hole (alpha = beta = 0)."""
    q, p = oracle.camera_ray(0.5, 0.24, 2.0, 15.0, 1.2, 75.0, 1, 1, 0, 0)
    assert p[2] == 0.0
    gu = oracle.metric_upper(0.5, 0.24, 2.0, 15.0, 1.2)
    assert abs((gu @ p)[3]) < 1e-15


def test_equatorial_camera_mirror(oracle):
    """At theta0 = pi/2, rows j and resY-1-j have opposite p_theta and equal p_t, p_r, p_phi."""
    resX, resY = 4, 6
    for i in range(resX):
        for j in range(resY):
            _, p1 = oracle.camera_ray(0.5, 0.24, 2.0, 15.0, np.pi / 2, 75.0, resX, resY, i, j)
            _, p2 = oracle.camera_ray(0.5, 0.24, 2.0, 15.0, np.pi / 2, 75.0, resX, resY, i,
                                      resY - 1 - j)
            assert p1[2] == -p2[2]
            np.testing.assert_allclose(p1[[0, 1, 3]], p2[[0, 1, 3]], rtol=1e-15)


def test_compat_camera_flag_matches_at_equator(oracle):
    """The listing's v^phi = alpha equals the default alpha/sin(theta0) at theta0 = pi/2."""
    for i, j in [(0, 0), (3, 2)]:
        _, p1 = oracle.camera_ray(0.5, 0.24, 0.0, 15.0, np.pi / 2, 75.0, 5, 5, i, j, 0)
        _, p2 = oracle.camera_ray(0.5, 0.24, 0.0, 15.0, np.pi / 2, 75.0, 5, 5, i, j,
                                  oracle.FLAG_COMPAT_CAMERA)
        np.testing.assert_allclose(p1, p2, rtol=1e-15)


@pytest.mark.parametrize("bad", [
    dict(M=0.0), dict(S=0.25), dict(S=0.0, Q=1.0), dict(r0=0.0), dict(th0=0.0),
    dict(fov=180.0), dict(resX=0),
])
def test_invalid_arguments_rejected(oracle, bad):
    kw = dict(M=0.5, S=0.24, Q=0.0, r0=15.0, th0=1.0, fov=75.0, resX=4, resY=4)
    kw.update(bad)
    with pytest.raises(ValueError):
        oracle.camera_ray(kw["M"], kw["S"], kw["Q"], kw["r0"], kw["th0"], kw["fov"],
                          kw["resX"], kw["resY"], 0, 0)


@pytest.mark.parametrize("M,S,Q,r0,th0", CASES)
def test_direction_camera_is_null_normalised_and_points_where_asked(oracle, M, S, Q, r0, th0):
    """The per-ray form (direction (alpha, beta) instead of a pixel index, used for the
    surrogate's training rays): H = 0, v^t = -1, and v^theta/(-v^r) = beta,
    v^phi sin(theta0)/(-v^r) = alpha, checked with the inverse metric."""
    rng = np.random.default_rng(4)
    gu = oracle.metric_upper(M, S, Q, r0, th0)
    for al, be in rng.uniform(-0.05, 0.05, (20, 2)):
        q, p = oracle.camera_dir(M, S, Q, r0, th0, al, be)
        assert list(q) == [0.0, r0, th0, 0.0]
        v = gu @ p
        assert abs(v[0] + 1.0) < 1e-13
        assert abs(0.5 * p @ gu @ p) < 1e-13 * (p @ p)
        assert abs(v[2] / -v[1] - be) < 1e-13 and abs(v[3] * np.sin(th0) / -v[1] - al) < 1e-13
