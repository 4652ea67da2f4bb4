"""Pins of the CPU reference network used to check the GPU surrogate's gradients."""
import numpy as np

from oracle import mlp


def _batch(n=64, seed=3):
    rng = np.random.default_rng(seed)
    al, be = rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, n)
    sp, q, th = rng.uniform(0, 0.99, n), np.zeros(n), rng.uniform(0.1, 1.5, n)
    X0 = mlp.features(al, be, sp, q, th)
    st = rng.integers(0, 2, n)
    y, d = mlp.labels(st, rng.uniform(0.1, 3.0, n), rng.uniform(-3, 3, n))
    return X0, y, d


def test_fp64_gradient_matches_finite_differences():
    """The analytic backward pass of the exact (unrounded) network against central
    differences on a sample of parameters from every layer."""
    p = mlp.init_params(7)
    X0, y, d = _batch()
    loss, g, _ = mlp.loss_and_grad(p, X0, y, d, 10.0, bf=False)
    rng = np.random.default_rng(0)
    ws, bs = mlp.split(np.arange(p.size))
    idx = []
    for w, b in zip(ws, bs):
        idx += list(rng.choice(w.ravel()[np.nonzero(w.ravel() % 16 < 10)[0]] if w.shape[1] == 16
                               else w.ravel(), 4, replace=False)) + list(rng.choice(b, 2))
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X0, y, d, 10.0, bf=False)[0] -
              mlp.loss_and_grad(pm, X0, y, d, 10.0, bf=False)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.0e38])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6
    assert r[3] == 1.0 and r[4] == -2.5


def test_features_cover_unit_range():
    X = mlp.features([-0.0491, 0.0491], [-0.05, 0.05], [0.0, 0.99], [0, 0],
                     [5 * np.pi / 180, np.pi / 2])
    assert np.allclose(X[:, 2], [-1, 1]) and np.allclose(X[:, 4], [-1, 1])
    assert np.all(np.abs(X[:, :2]) < 1.01)
    # polar columns: rho and a unit (cos psi, sin psi); cos/sin of theta0
    assert np.allclose(X[:, 5], np.hypot(X[:, 0], X[:, 1]))
    assert np.allclose(X[:, 6] ** 2 + X[:, 7] ** 2, 1.0)
    assert np.allclose(X[:, 8] ** 2 + X[:, 9] ** 2, 1.0) and np.all(X[:, 10:] == 0)


def test_f16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 1.0 + 2 ** -10, -2.5, 65504.0])
    r = mlp.f16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -9
    assert r[3] == 1.0 + 2 ** -10 and r[4] == -2.5 and r[5] == 65504.0


def test_rounded_network_stays_close_to_exact():
    """The 16-bit rounding points perturb the loss and gradient only slightly (a
    transposed or misplaced rounding would not)."""
    p = mlp.init_params(4)
    rng = np.random.Generator(np.random.PCG64(8))
    X0 = mlp.features(rng.uniform(-0.04, 0.04, 64), rng.uniform(-0.04, 0.04, 64),
                      rng.uniform(0, 0.99, 64), np.zeros(64), rng.uniform(0.1, 1.5, 64))
    y = (rng.uniform(size=64) < 0.5).astype(float)
    d = np.stack([np.ones(64), np.zeros(64), np.zeros(64)], 1) * y[:, None]
    l0, g0, _ = mlp.loss_and_grad(p, X0, y, d, 10.0, bf=False)
    l1, g1, _ = mlp.loss_and_grad(p, X0, y, d, 10.0, bf=True)
    assert abs(l1 - l0) < 1e-2 * abs(l0)
    assert np.linalg.norm(g1 - g0) < 2e-2 * np.linalg.norm(g0)
