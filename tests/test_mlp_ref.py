"""Pins of the FP64 reference of the proposal network (no GPU)."""
import math

import numpy as np

from oracle import mlp_ref as R


def test_parameter_count():
    # 6*128+128 + 3*(128*128+128) + 128*4+4
    assert R.param_count() == 50948


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    assert abs(R.gelu(np.array([0.0]))[0]) == 0.0
    # Phi(x) + Phi(-x) = 1  =>  gelu(x) - gelu(-x) = x
    assert np.allclose(R.gelu(x) - R.gelu(-x), x, atol=1e-15)
    assert abs(R.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-6
    assert np.allclose((R.gelu(x + h) - R.gelu(x - h)) / (2 * h), R.gelu_grad(x), atol=1e-8)


def test_loss_at_zero_output_is_log2_plus_squares():
    p = np.zeros(R.param_count())
    x = np.random.default_rng(0).normal(size=(5, 6))
    t = np.array([[0.3, 0.2, 1.0, 0.5]] * 5)
    loss, g = R.loss_grad(p, x, t)
    assert abs(loss - (0.09 + 0.04 + 0.25 + math.log(2))) < 1e-14


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.3, R.param_count())
    x = rng.normal(size=(7, 6))
    t = np.column_stack([rng.uniform(0, 0.5, 7), rng.uniform(-0.5, 0.5, 7), rng.integers(0, 2, 7),
                         rng.uniform(0, 1, 7)])
    mask = np.array([1, 1, 0, 1, 1, 0, 1], float)
    _, g = R.loss_grad(p, x, t, mask)
    idx = rng.choice(p.size, 60, replace=False)
    idx = np.concatenate([idx, [0, 767, 768, 895, p.size - 1, p.size - 5]])
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (R.loss_grad(pp, x, t, mask)[0] - R.loss_grad(pm, x, t, mask)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, g[k])


def test_first_adamw_step_is_signed_learning_rate():
    """At t = 1 the bias-corrected moments are g and g^2, so without decay
    every weight moves by lr * g/(|g| + eps)."""
    rng = np.random.default_rng(2)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = R.adamw(p, np.zeros(100), np.zeros(100), g, 1, lr=0.01, eps=1e-12)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-12)
    p2, _, _ = R.adamw(p, np.zeros(100), np.zeros(100), g, 1, lr=0.01, eps=1e-12, wd=0.5)
    assert np.allclose(p2, p - 0.01 * (np.sign(g) + 0.5 * p), atol=1e-12)
