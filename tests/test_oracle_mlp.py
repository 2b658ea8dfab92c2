"""Pins of the network oracle (oracle/mlp.py) against mathematics, not
against itself: central finite differences of the loss, a hand-built network
with a known output, the cross-entropy at a zero logit, and Adam's closed form
under a constant gradient."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def _batch(seed, B=24, fin=12):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, fin))
    Y = np.stack([rng.uniform(0, 1, B), rng.integers(0, 2, B).astype(float)], axis=1)
    mask = (rng.uniform(0, 1, B) < 0.7).astype(float)
    return X, Y, mask


def test_param_count():
    assert M.n_params() == 12 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 2 + 2 == 9282


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_central_differences(seed):
    """Every coordinate of the backward pass against (L(t+e) - L(t-e)) / 2e,
    e = 1e-6 (the loss is piecewise smooth; a kink within e of a sample is a
    measure-zero event for random weights)."""
    theta = M.init_params(100 + seed)
    theta[-2:] = [0.3, -0.2]
    X, Y, mask = _batch(seed)
    lam, kappa = 0.3, 4.0
    _, g = M.loss_grad(theta, X, Y, mask, lam, kappa)
    eps = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        t = theta.copy()
        t[i] += eps
        lp = M.loss(t, X, Y, mask, lam, kappa)
        t[i] -= 2 * eps
        lm = M.loss(t, X, Y, mask, lam, kappa)
        fd[i] = (lp - lm) / (2 * eps)
    err = np.abs(fd - g)
    assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)
    assert err.max() <= 1e-7 + 1e-5 * np.abs(g).max()


def test_hand_built_network():
    """sizes (1,2,2,2,2): h1 = (relu(x), relu(-x)), identity hidden layers,
    o0 = h1_0 - h1_1 + 0.5 = x + 0.5, o1 = 2(h1_0 + h1_1) - 1 = 2|x| - 1."""
    sizes = (1, 2, 2, 2, 2)
    parts = [np.array([1.0, -1.0]), np.zeros(2),
             np.eye(2).ravel(), np.zeros(2),
             np.eye(2).ravel(), np.zeros(2),
             np.array([1.0, -1.0, 2.0, 2.0]), np.array([0.5, -1.0])]
    theta = np.concatenate(parts)
    assert theta.size == M.n_params(sizes)
    x = np.array([[-1.5], [0.0], [0.25], [3.0]])
    o = M.forward(theta, x, sizes)
    np.testing.assert_array_equal(o[:, 0], x[:, 0] + 0.5)
    np.testing.assert_array_equal(o[:, 1], 2 * np.abs(x[:, 0]) - 1)


def test_cross_entropy_at_zero_logit():
    """With mask 0 the loss is lam * BCE(sigmoid(o1), y1); at o1 = 0 it is
    lam * log 2 whatever y1 is; its o1-gradient is lam * (1/2 - y1) / B."""
    sizes = (1, 2, 2, 2, 2)
    theta = np.zeros(M.n_params(sizes))
    X = np.array([[0.3], [-0.7]])
    Y = np.array([[0.5, 1.0], [0.2, 0.0]])
    lam = 0.25
    L_, g = M.loss_grad(theta, X, Y, np.zeros(2), lam, sizes=sizes)
    assert L_ == pytest.approx(lam * math.log(2.0), rel=1e-15)
    # the output bias b3[1] is the last parameter
    assert g[-1] == pytest.approx(lam * ((0.5 - 1.0) + (0.5 - 0.0)) / 2, abs=1e-17)


def test_asymmetric_regression_term():
    """mask 1, lam 0: under-prediction by e costs kappa e^2, over-prediction e^2."""
    sizes = (1, 2, 2, 2, 2)
    theta = np.zeros(M.n_params(sizes))
    theta[-2] = 0.4                       # o0 = 0.4 for every input
    X = np.zeros((2, 1))
    Y = np.array([[0.5, 0.0], [0.1, 0.0]])
    L_ = M.loss(theta, X, Y, np.ones(2), lam=0.0, kappa=4.0, sizes=sizes)
    assert L_ == pytest.approx((4.0 * 0.1 ** 2 + 0.3 ** 2) / 2, rel=1e-14)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2, so every step moves theta by lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th0 = np.array([1.0, 2.0, 3.0, 4.0])
    opt = M.Adam(4, lr=1e-2)
    th = th0.copy()
    for _ in range(25):
        th = opt.step(th, g)
    expect = th0 - 25 * 1e-2 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(th, expect, rtol=0, atol=1e-12)


def test_training_reduces_loss():
    """A few hundred Adam steps on a smooth target bring the loss down by an
    order of magnitude (the backward pass points downhill)."""
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (256, 12))
    Y = np.stack([0.5 + 0.3 * np.tanh(X[:, 0] - X[:, 3]), (X[:, 1] > 0).astype(float)], 1)
    mask = np.ones(256)
    theta = M.init_params(3)
    opt = M.Adam(theta.size, lr=3e-3)
    l0 = M.loss(theta, X, Y, mask)
    for _ in range(300):
        _, g = M.loss_grad(theta, X, Y, mask)
        theta = opt.step(theta, g)
    assert M.loss(theta, X, Y, mask) < 0.1 * l0
