"""Pins of the learned-potential oracle (oracle/mlp.py) against calculus and libraries:

* the loss computed from window-pattern counts equals the loss with the network run
  on every window of every configuration (the definition);
* the back-propagated gradient equals central finite differences of the loss;
* BF16 rounding against torch's float32 -> bfloat16 conversion and hand-worked ties;
* GELU and its derivative against scipy's normal CDF and finite differences;
* one Adam step against the update written out for a scalar.
"""
import math

import numpy as np
import pytest
import scipy.special

from oracle import mlp


def random_batch(n, L, seed):
    g = np.random.default_rng(seed)
    W = (L + 63) // 64
    words = np.zeros((n, W), dtype=np.uint64)
    for r in range(n):
        occ = g.choice(L, size=L // 2, replace=False)
        for i in occ:
            words[r, i // 64] |= np.uint64(1) << np.uint64(i % 64)
    labels = g.integers(0, 2, n).astype(np.uint8)
    return words, labels


def test_counted_loss_equals_direct_loss():
    theta = mlp.init_params(3).astype(np.float64)
    theta += np.random.default_rng(1).normal(0, 0.05, theta.size)
    for L in (20, 70):
        words, labels = random_batch(5, L, L)
        loss, _ = mlp.loss_and_grad(theta, words, labels, L)
        assert abs(loss - mlp.loss_direct(theta, words, labels, L)) < 1e-10


def test_window_counts_sum_to_L():
    words, _ = random_batch(7, 37, 2)
    c = mlp.window_counts(words, 37)
    assert np.all(c.sum(axis=1) == 37)
    # every configuration with N particles: each site is the centre of one window
    centre_bit = (np.arange(512) >> 4) & 1
    assert np.all(c @ centre_bit == 37 // 2)


def test_gradient_against_finite_differences():
    L = 24
    words, labels = random_batch(6, L, 5)
    theta = mlp.init_params(9).astype(np.float64)
    theta += np.random.default_rng(2).normal(0, 0.1, theta.size)
    _, grad = mlp.loss_and_grad(theta, words, labels, L)
    offsets, k = {}, 0
    for name, shape in mlp.SIZES:
        offsets[name] = (k, int(np.prod(shape)))
        k += int(np.prod(shape))
    g = np.random.default_rng(0)
    idx = []
    for name, (k0, n) in offsets.items():
        idx += list(k0 + g.choice(n, size=min(n, 6), replace=False))
    h = 1e-5
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, words, labels, L)[0] - mlp.loss_and_grad(tm, words, labels, L)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, grad[i])


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(4)
    x = np.concatenate([g.normal(0, 3, 5000), g.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, -2.5]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want.astype(np.float64))
    # ties go to the even mantissa: 1 + 2^-8 is half way between 1 and 1 + 2^-7
    assert mlp.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert mlp.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


def test_gelu_and_derivative():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(mlp.gelu(x), x * scipy.special.ndtr(x), rtol=1e-13, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_adam_step_written_out():
    theta = np.array([0.5], dtype=np.float32)
    g = np.array([0.2])
    th, m, v = mlp.adam(theta, g, np.zeros(1), np.zeros(1), 1, 0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    assert abs(float(th[0]) - (0.5 - 0.01 * 0.2 / (0.2 + 1e-8))) < 1e-7
    assert abs(float(m[0]) - 0.02) < 1e-8 and abs(float(v[0]) - 0.001 * 0.04) < 1e-11   # float32 state
