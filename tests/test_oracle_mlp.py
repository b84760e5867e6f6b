"""Pins of the FP64 surrogate-MLP reference: backpropagation against central finite
differences, closed forms of special networks, SiLU, the first Adam step, bf16 rounding."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(1)
    theta = M.init(3) * 0.7 + rng.normal(0, 0.05, M.N_PARAMS)
    X = rng.normal(0, 1, (9, 5))
    T = rng.normal(0, 1, (9, 3))
    loss, g = M.loss_and_grad(theta, X, T)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    # every tensor is probed: biases and the padded-free weight blocks
    idx = np.unique(np.concatenate([idx, [0, 5 * 64, 5 * 64 + 64, M.N_PARAMS - 1, M.N_PARAMS - 4]]))
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, X, T)[0] - M.loss_and_grad(theta - e, X, T)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_zero_weights_give_the_bias_closed_form():
    """With all weights zero the output is b3 and only the biases of the last layer learn."""
    p = M.unpack(np.zeros(M.N_PARAMS))
    p["b1"][:] = 0.3
    p["b2"][:] = -0.2
    p["b3"][:] = [1.0, -2.0, 0.5]
    theta = M.pack(p)
    X = np.random.default_rng(0).normal(size=(4, 5))
    assert np.allclose(M.forward(theta, X), [[1.0, -2.0, 0.5]] * 4)
    T = np.zeros((4, 3))
    loss, g = M.loss_and_grad(theta, X, T)
    assert loss == pytest.approx((1 + 4 + 0.25) / 3)
    gp = M.unpack(g)
    assert np.allclose(gp["b3"], 2 * np.array([1.0, -2.0, 0.5]) / 3)
    assert np.allclose(gp["W1"], 0) and np.allclose(gp["W2"], 0)
    # W3 sees the constant hidden activation silu(b2) = silu(-0.2)
    assert np.allclose(gp["W3"], np.outer(2 * np.array([1.0, -2.0, 0.5]) / 3,
                                          np.full(64, -0.2 / (1 + np.exp(0.2)))))


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 41)
    assert np.allclose(M.silu(z), z * 0.5 * (1 + np.tanh(z / 2)))
    h = 1e-6
    assert np.allclose(M.dsilu(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), atol=1e-8)
    assert M.silu(0.0) == 0.0 and M.dsilu(0.0) == 0.5


def test_first_adam_step_moves_each_parameter_by_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-12)
    assert np.allclose(th, -0.01 * np.sign(g), atol=1e-9)


def test_bf16_rounding():
    assert M.bf16(1.0) == 1.0
    assert M.bf16(1.0 + 2 ** -9) == 1.0               # ties to even
    assert M.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = np.random.default_rng(2).normal(size=1000)
    assert np.max(np.abs(M.bf16(x) / x - 1)) <= 2 ** -8 + 1e-12
