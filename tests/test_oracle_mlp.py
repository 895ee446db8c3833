"""Pins of the learned-correction oracle (oracle/mlp.py): gradients against
finite differences, Adam's first step in closed form, the residual label's
asymptotic order, and closed forms of the quadrupole features."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_param_count():
    assert mlp.n_params() == 12 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 9347


def test_gelu_and_its_derivative():
    z = np.linspace(-4, 4, 41)
    ref = np.array([0.5 * v * (1 + math.tanh(math.sqrt(2 / math.pi) * (v + 0.044715 * v ** 3)))
                    for v in z])
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=1e-15, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def test_backward_matches_finite_differences():
    g = np.random.default_rng(4)
    theta = mlp.init(7)
    X = g.normal(0, 1, (32, 12))
    Y = g.normal(0, 0.1, (32, 3))
    L, grad = mlp.backward(theta, X, Y)
    assert L == pytest.approx(mlp.loss(theta, X, Y), rel=1e-15)
    idx = g.choice(len(theta), 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (mlp.loss(theta + e, X, Y) - mlp.loss(theta - e, X, Y)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-7 * max(1e-3, abs(grad[k])) + 1e-10


def test_adam_first_step_closed_form():
    """After one step from zero moments the update is lr g / (|g| + eps)."""
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    t1, m, v = mlp.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_label_falls_as_third_power():
    """The multipole error of a cell relative to G M / R^2 is octupole order:
    (w/R)^3 for unequal masses; a single particle has no residual."""
    g = np.random.default_rng(2)
    xs = g.uniform(0, 0.01, (5, 3))
    ms = g.uniform(0.5, 1.5, 5)
    M = ms.sum()
    com = (ms[:, None] * xs).sum(0) / M
    dd = xs - com
    d2 = (dd ** 2).sum(1)
    Q = np.array([np.sum(ms * (3 * dd[:, 0] ** 2 - d2)), np.sum(ms * (3 * dd[:, 1] ** 2 - d2)),
                  np.sum(ms * (3 * dd[:, 2] ** 2 - d2)), np.sum(ms * 3 * dd[:, 0] * dd[:, 1]),
                  np.sum(ms * 3 * dd[:, 0] * dd[:, 2]), np.sum(ms * 3 * dd[:, 1] * dd[:, 2])])
    u = np.array([0.3, 0.5, 0.81]) / np.linalg.norm([0.3, 0.5, 0.81])
    mags = [np.linalg.norm(mlp.label(com + R * u, M, com, Q, xs, ms)) for R in (0.1, 0.2, 0.4)]
    for a, b in zip(mags, mags[1:]):
        assert 7.0 < a / b < 9.2
    one = mlp.label(np.array([1.0, 2.0, 3.0]), 2.0, np.zeros(3), np.zeros(6), np.zeros((1, 3)),
                    np.array([2.0]))
    assert np.max(np.abs(one)) < 1e-13


def test_quadrupole_features_closed_form():
    """Two equal masses at +-s/2 on the x axis: Q/(M w^2) = s^2/(2 w^2)
    diag(1, -1/2, -1/2); a target on the y axis sees r.Q.r = -s^2/(4 w^2)."""
    s, w, m = 0.6, 2.0, 1.5
    xs = np.array([[-s / 2, 0, 0], [s / 2, 0, 0]])
    M = 2 * m
    Q = np.array([m * s * s, -m * s * s / 2, -m * s * s / 2, 0.0, 0.0, 0.0])
    f = mlp.features(np.array([0.0, 10.0, 0.0]), M, np.zeros(3), Q, np.array([0.1, 0.0, 0.0]), w, 2)
    k = s * s / (2 * w * w)
    np.testing.assert_allclose(f[:3], [0, 1, 0], atol=1e-15)
    assert f[3] == pytest.approx(0.2)
    assert f[4] == pytest.approx(math.log10(2))
    np.testing.assert_allclose(f[5:8], [-0.05, 0, 0], atol=1e-15)
    assert f[8] == pytest.approx(-k / 2)
    assert f[9] == pytest.approx(k / 2)
    assert f[10] == pytest.approx(1.5 * k * k)
    assert f[11] == pytest.approx(k ** 3 / 4)
