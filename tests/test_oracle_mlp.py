"""Pins of the FP64 surrogate network of the oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp


def small(seed=0, sizes=(25, 7, 6, 4)):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mlp.n_params(list(sizes))) * 0.3
    x = rng.uniform(-1, 1, (11, 5))
    t = rng.standard_normal((11, sizes[-1]))
    return list(sizes), theta, x, t


def test_silu_derivative_against_finite_differences():
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.dsilu(z))) < 1e-9


def test_gradient_against_central_differences():
    sizes, theta, x, t = small()
    L, g = mlp.loss_and_grad(theta, sizes, x, t)
    assert abs(L - mlp.loss(theta, sizes, x, t)) < 1e-14
    h = 1e-6
    # every parameter of this small network (all weight and bias blocks)
    fd = np.empty_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (mlp.loss(theta + e, sizes, x, t) - mlp.loss(theta - e, sizes, x, t)) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-8 * max(1.0, np.max(np.abs(g)))


def test_output_bias_stationary_at_target_mean():
    sizes, theta, x, t = small(1)
    layers = mlp.unflatten(theta, sizes)
    W, b = layers[-1]
    layers[-1] = (np.zeros_like(W), t.mean(axis=0))
    th = mlp.flatten(layers)
    _, g = mlp.loss_and_grad(th, sizes, x, t)
    nb = sizes[-1]
    assert np.max(np.abs(g[-nb:])) < 1e-14


def test_linear_network_reduces_to_least_squares():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (60, 5))
    t = rng.standard_normal((60, 3))
    A = np.hstack([mlp.embed(x), np.ones((60, 1))])
    sol, *_ = np.linalg.lstsq(A, t, rcond=None)
    W, b = sol[:25].T, sol[25]
    theta = mlp.flatten([(W, b)])
    L, g = mlp.loss_and_grad(theta, [25, 3], x, t)
    assert np.max(np.abs(g)) < 1e-12
    assert abs(L - np.sum((A @ sol - t) ** 2) / t.size) < 1e-13


def test_targets_and_loops_round_trip():
    rng = np.random.default_rng(5)
    parity = np.array([1, 1, -1, -1, 1])
    pairs = mlp.pair_list(parity)
    assert pairs == [(0, 0), (0, 1), (0, 4), (1, 1), (1, 4), (2, 2), (2, 3), (3, 3), (4, 4)]
    a = rng.standard_normal((2, 7, 5, 5))
    a = a + np.swapaxes(a, -1, -2)
    mask = np.outer(parity, parity) > 0
    a = a * mask
    y = mlp.targets(a[0], a[1], 0.3, pairs)
    assert y.shape == (7, 2 * len(pairs))
    assert np.allclose(mlp.loops_from_outputs(y, 0.3, pairs, 5), a, rtol=0, atol=1e-14)


def test_features_scaling():
    f = mlp.features([np.pi, -np.pi / 2], [0.0, np.pi], 0.1, -0.225, -0.9)
    assert np.allclose(f, [[1, 0, 0, 0, 0], [-0.5, 1, 0, 0, 0]])


def test_embedding_values():
    x = np.array([[1.0, -0.5, 0.5, 2.0, -1.0]])
    e = mlp.embed(x)[0]
    assert e.shape == (25,)
    assert np.allclose(e[:5], x[0])
    for k in range(1, 5):
        c0, s0, c1, s1 = e[5 + 4 * (k - 1):9 + 4 * (k - 1)]
        assert np.isclose(c0, (-1) ** k) and abs(s0) < 1e-12          # x0 = 1: k pi
        assert np.isclose(c1, np.cos(-k * np.pi / 2)) and np.isclose(s1, np.sin(-k * np.pi / 2))
    assert np.allclose(e[21:], [0.25, 0.125, 1.0, -0.5])
