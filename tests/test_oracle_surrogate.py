"""Pins of the surrogate network's oracle: the gradient against central finite
differences of the loss, GELU against its definition through the normal CDF,
BF16 rounding against torch's conversion, Adam against a hand-derived first step."""
import math

import numpy as np

from oracle import surrogate as S


def test_gelu_is_z_times_normal_cdf():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 61)
    assert np.abs(S.gelu(z) - z * norm.cdf(z)).max() < 1e-15
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.abs(fd - S.gelu_grad(z)).max() < 1e-8


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(0).normal(size=1000).astype(np.float32) * 10
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16_round(x), ref)


def test_gradient_matches_central_differences():
    d_in, H, B = 5, 16, 7
    rng = np.random.default_rng(1)
    p = S.init_params(d_in, H, seed=2)
    p += rng.normal(0, 0.05, p.size)  # nonzero biases
    X = rng.uniform(-0.5, 0.5, (B, d_in))
    t = rng.normal(size=B)
    loss, g = S.loss_grad(p, X, t, d_in, H)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(p.size)
        e[i] = h
        fd = (S.loss_grad(p + e, X, t, d_in, H)[0] - S.loss_grad(p - e, X, t, d_in, H)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_moves_each_parameter_by_lr():
    # first step: m = (1-b1) g, v = (1-b2) g^2; bias correction gives m/c1 = g, v/c2 = g^2
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = S.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p, -0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)
