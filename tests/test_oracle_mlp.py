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


def test_split_product_error_bound():
    """The split-precision product x_hi w_hi + x_lo w_hi + x_hi w_lo (hi = bf16(v),
    lo = bf16(v - hi)) is within 2^-15 sum_k |x_k||w_k| of the exact product: each pair
    carries its value to 2^-17 and the dropped x_lo w_lo is at most 2^-16 of |x||w|.
    A single bf16 product is not (its error is ~2^-9)."""
    rng = np.random.default_rng(8)
    A = rng.normal(0, 1, (64, 256)) * np.exp(rng.uniform(-3, 3, (64, 1)))
    Wt = rng.normal(0, 0.06, (48, 256))
    exact = A @ Wt.T
    scale = np.abs(A) @ np.abs(Wt).T
    err = np.abs(mlp.split_product(A, Wt) - exact)
    assert np.all(err <= 2.0 ** -15 * scale)
    plain = np.abs(mlp.bf16(A) @ mlp.bf16(Wt).T - exact)
    assert np.max(plain / scale) > 2.0 ** -11
    hi, lo = mlp.split_bf16(A)
    assert np.all(np.abs(hi + lo - A) <= 2.0 ** -16 * np.abs(A))
