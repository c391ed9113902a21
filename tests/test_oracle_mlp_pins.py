"""Pins of the indicator oracle (oracle/mlp.py): finite-difference gradients,
closed-form loss, and the feature layout on hand-built states."""
import math

import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    f_in = 40
    P = mlp.init_params(f_in, seed=1)
    for key in P:
        P[key] = P[key] + 0.05 * rng.normal(size=P[key].shape)  # nonzero biases
    X = rng.normal(size=(17, f_in))
    y = (rng.uniform(size=17) < 0.3).astype(float)
    a = 3.0
    cache = mlp.forward(P, X)
    g = mlp.backward(P, X, cache, y, a)
    h = 1e-6
    for key in P:
        flat = P[key].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for j in idx:
            old = flat[j]
            flat[j] = old + h
            lp = mlp.loss(mlp.forward(P, X)["logit"], y, a)
            flat[j] = old - h
            lm = mlp.loss(mlp.forward(P, X)["logit"], y, a)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (key, j, fd, an)


def test_loss_at_zero_logit():
    y = np.array([1.0, 0.0, 1.0, 0.0, 0.0])
    a = 4.0
    ref = np.mean(a * y * math.log(2) + (1 - y) * math.log(2))
    assert abs(mlp.loss(np.zeros(5), y, a) - ref) < 1e-15


def _const_state(n, N, U):
    w = np.zeros((n, n, n, 5, N))
    w[..., 0] = U
    return w


def test_features_constant_state():
    g = 1.4
    rho, v, p = 1.3, np.array([0.3, -0.4, 0.2]), 0.8
    U = np.array([rho, rho * v[0], rho * v[1], rho * v[2], p / (g - 1) + 0.5 * rho * v @ v])
    w = _const_state(3, 10, U)
    X = mlp.features(w, 2, g)
    assert X.shape == (27, mlp.n_features_padded(2))
    c = math.sqrt(g * p / rho)
    own = 5 * 9
    assert np.all(X[:, :own] == 0)
    assert np.allclose(X[:, own], math.log(rho), atol=1e-15)
    assert np.allclose(X[:, own + 1], np.linalg.norm(v) / c, atol=1e-14)
    assert np.all(np.abs(X[:, own + 2:]) < 1e-15)


def test_features_neighbour_offsets_and_scales():
    g = 1.4
    U = np.array([1.0, 0.1, 0.0, 0.0, 2.0])
    w = _const_state(4, 4, U)
    # one cell at (iz, iy, ix) = (1, 2, 3) gets a larger density mean
    w[1, 2, 3, 0, 0] = 1.5
    w[1, 2, 2, 4, 2] = 0.6  # a high mode (l = 2) of the energy of cell (1,2,2)
    X = mlp.features(w, 1, g)
    own, extra = 5 * 3, 2 + 5  # log rho, Mach, then the five excursion bounds
    offs = mlp.neighbour_offsets()
    cell = (1 * 4 + 2) * 4 + 2  # (iz, iy, ix) = (1, 2, 2): its +x neighbour is the changed cell
    j = offs.index((0, 0, 1))
    assert abs(X[cell, own + extra + 5 * j + 0] - 0.5 / 1.0) < 1e-15
    assert abs(X[cell, own + extra + 5 * j + 4]) < 1e-15
    # energy high mode l=2 of cell (1,2,2) scaled by |E|
    assert abs(X[cell, 4 * 3 + 1] - 0.6 / 2.0) < 1e-15
    # its excursion bound: mode 2 is sqrt(3) xi_y, whose largest |value| on S
    # is sqrt(3) (the GLL end points of S_y)
    assert abs(X[cell, own + 2 + 4] - 0.6 * math.sqrt(3) / 2.0) < 1e-15
    assert np.all(X[cell, own + 2: own + 6] == 0)
    # the changed cell sees every neighbour at -0.5 / 1.5 in density
    cc = (1 * 4 + 2) * 4 + 3
    for j in range(26):
        assert abs(X[cc, own + extra + 5 * j] - (-0.5 / 1.5)) < 1e-15
