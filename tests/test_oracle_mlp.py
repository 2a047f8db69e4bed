"""Pins for the FP64 oracle of the learned warm start (MLP forward, Gaussian
NLL loss and gradient, Adam).  CPU only."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _net(dims, seed=0):
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(1, len(dims)):
        ps.append(rng.normal(0, 1.0 / math.sqrt(dims[l - 1]), size=dims[l] * dims[l - 1]))
        ps.append(rng.normal(0, 0.1, size=dims[l]))
    return np.concatenate(ps)


def test_param_count():
    assert O.mlp_num_params([36, 256, 256, 256, 300]) == 36 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 300 + 300


def test_gelu_forward_matches_erf_definition():
    from scipy.special import erf

    dims = [1, 1]
    # identity-like single linear layer: no activation on the output
    params = np.array([2.0, 0.5])
    out = O.mlp_forward(dims, params, [0.0], [1.0], np.array([[3.0]]))
    assert out[0, 0] == pytest.approx(6.5)
    # one hidden unit: y = GELU(z) through an identity output layer
    dims = [1, 1, 1]
    for z in [-2.0, -0.3, 0.0, 0.7, 3.0]:
        params = np.array([1.0, 0.0, 1.0, 0.0])
        y = O.mlp_forward(dims, params, [0.0], [1.0], np.array([[z]]))[0, 0]
        assert y == pytest.approx(0.5 * z * (1 + erf(z / math.sqrt(2))), rel=1e-14, abs=1e-16)


def test_input_normalisation():
    dims = [2, 1]
    params = np.array([1.0, 1.0, 0.0])
    y = O.mlp_forward(dims, params, [1.0, -2.0], [2.0, 4.0], np.array([[3.0, 2.0]]))
    assert y[0, 0] == pytest.approx((3 - 1) / 2 + (2 + 2) / 4)


def test_zero_network_loss_closed_form():
    # mu = 0 and s = 0 everywhere: loss = mean over samples of 0.5 ||t||^2
    dims = [3, 4, 6]  # n_mu = 4, nu = 2 -> 2 scales
    params = np.zeros(O.mlp_num_params(dims))
    rng = np.random.default_rng(1)
    X = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 4))
    loss, g = O.mlp_loss_grad(dims, params, np.zeros(3), np.ones(3), X, T, 2)
    assert loss == pytest.approx(0.5 * np.sum(T ** 2) / 5, rel=1e-14)


def test_gradient_matches_central_finite_differences():
    dims = [4, 6, 5, 9]  # n_mu = 6, nu = 2: 3 scales
    params = _net(dims, 2)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(7, 4))
    T = rng.normal(size=(7, 6))
    xm, xs = rng.normal(size=4), 0.5 + rng.random(4)
    loss, g = O.mlp_loss_grad(dims, params, xm, xs, X, T, 2)
    h = 1e-6
    fd = np.zeros_like(params)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = h
        lp, _ = O.mlp_loss_grad(dims, params + e, xm, xs, X, T, 2)
        lm, _ = O.mlp_loss_grad(dims, params - e, xm, xs, X, T, 2)
        fd[i] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_adam_first_step_moves_by_learning_rate_times_sign():
    # after one step m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    p0 = p.copy()
    O.mlp_adam(p, g, m, v, 1, lr=0.01)
    np.testing.assert_allclose(p0 - p, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_bias_correction_second_step():
    p = np.array([0.0])
    m = np.zeros(1)
    v = np.zeros(1)
    O.mlp_adam(p, np.array([1.0]), m, v, 1, lr=0.1)
    O.mlp_adam(p, np.array([3.0]), m, v, 2, lr=0.1)
    m2 = 0.9 * 0.1 * 1.0 + 0.1 * 3.0
    v2 = 0.999 * 0.001 * 1.0 + 0.001 * 9.0
    step2 = 0.1 * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert p[0] == pytest.approx(-0.1 * 1.0 / (1.0 + 1e-8) - step2, rel=1e-12)
