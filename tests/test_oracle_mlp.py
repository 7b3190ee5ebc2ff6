"""Pins of the FP64 network oracle (oracle/mlp.py) against things fixed
independently of its backward pass: central finite differences of the loss,
a network whose output is known in closed form, the first Adam step (which
moves every parameter by lr * g / (|g| + eps)), and a learnable toy
regression whose loss must fall."""
import numpy as np
import pytest

import oracle.mlp as M
from paper_2503_20605_gb300 import inputs as I

SMALL = (3, 7, 5, 6, 4)


def _data(S, n_out, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(20, 160, S), rng.uniform(8, 24, S), 10 ** rng.uniform(-1, 1, S)], axis=1)
    y = rng.normal(1.0, 0.3, (S, n_out))
    return x, y


def test_features():
    u = M.features(np.array([[90.0, 16.0, 1.0], [160.0, 24.0, 10.0], [20.0, 8.0, 0.1]]))
    np.testing.assert_allclose(u, [[0, 0, 0], [1, 1, 1], [-1, -1, -1]], atol=1e-15)


def test_param_count_and_init():
    assert M.n_params() == 3 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 64 + 64 == 149056
    p = I.mlp_init(0)
    assert p.dtype == np.float32 and p.size == M.n_params()
    (W0, b0), _, _, (W3, b3) = M.unpack(p.astype(np.float64))
    assert np.all(np.abs(W0) <= 1 / np.sqrt(3)) and np.all(b0 == 0) and np.all(b3 == 1)


@pytest.mark.parametrize("sizes,S", [(SMALL, 5), (M.SIZES, 3)])
def test_gradient_matches_central_differences(sizes, S):
    rng = np.random.default_rng(1)
    p = I.mlp_init(2, sizes).astype(np.float64) + rng.normal(0, 0.05, M.n_params(sizes))
    x, y = _data(S, sizes[-1], 3)
    g = M.grad(p, x, y, sizes)
    idx = np.arange(p.size) if p.size < 400 else rng.choice(p.size, 60, replace=False)
    # include the first and last entries of every layer's W and b
    bounds = np.cumsum([0] + [s for i, o in zip(sizes[:-1], sizes[1:]) for s in (o * i, o)])
    idx = np.unique(np.concatenate([idx, bounds[:-1], bounds[1:] - 1]))
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (M.loss(p + e, x, y, sizes) - M.loss(p - e, x, y, sizes)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, np.abs(g).max()) + 1e-8 * abs(g[k]), (k, fd, g[k])


def test_closed_form_output():
    # hidden weights zero: h_l = tanh(b_l) for l >= 2, output = W3 tanh(b2) + b3
    sizes = SMALL
    rng = np.random.default_rng(4)
    p = rng.normal(0, 1, M.n_params(sizes))
    layers = M.unpack(p, sizes)
    layers[1][0][:] = 0
    layers[2][0][:] = 0
    x, _ = _data(4, sizes[-1], 5)
    yhat, _ = M.forward(p, x, sizes)
    (W3, b3), (_, b2) = layers[3], layers[2]
    np.testing.assert_allclose(yhat, np.tile(W3 @ np.tanh(b2) + b3, (4, 1)), rtol=1e-14)


def test_first_adam_step():
    rng = np.random.default_rng(6)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1e-3, 50)
    opt = M.Adam(50, lr=1e-3)
    q = opt.step(p, g)
    np.testing.assert_allclose(p - q, 1e-3 * g / (np.abs(g) + M.EPS), rtol=1e-9)


def test_training_reduces_loss():
    sizes = (3, 16, 16, 16, 4)
    x, _ = _data(64, 4, 7)
    u = M.features(x)
    y = np.stack([1 + 0.3 * u[:, 0], 1 - 0.2 * u[:, 1], 1 + 0.1 * u[:, 0] * u[:, 1], 1 + 0.1 * u[:, 2]], axis=1)
    p = I.mlp_init(8, sizes).astype(np.float64)
    opt = M.Adam(p.size, lr=1e-2)
    l0 = M.loss(p, x, y, sizes)
    for _ in range(300):
        p = opt.step(p, M.grad(p, x, y, sizes))
    assert M.loss(p, x, y, sizes) < 0.05 * l0
