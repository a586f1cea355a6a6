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


def _f32_evaluation(theta, words, labels, L, seed):
    """The network evaluated in FP32 the way a GPU may: FP32 activations (correctly
    rounded GELU), BF16 operands rounded from them, FP32 matrix products and FP32 sums in
    a shuffled order.  Independent of loss_and_grad except for the shared definitions."""
    f = np.float32
    P = mlp.unpack(theta)
    X = mlp.patterns().astype(f)
    bf = lambda a: mlp.bf16(np.asarray(a, dtype=f)).astype(f)
    Z1 = mlp.layer1_f32(theta).astype(f)
    H1 = mlp.gelu(Z1.astype(np.float64)).astype(f)
    Z2 = (bf(H1) @ bf(P["W2"]).T).astype(f) + P["b2"].astype(f)
    H2 = mlp.gelu(Z2.astype(np.float64)).astype(f)
    Phi = (bf(H2) @ bf(P["W3"])).astype(f) + f(P["b3"])
    counts = mlp.window_counts(words, L).astype(f)
    y = np.asarray(labels, dtype=f)
    n = y.size
    z = f(0.5) * (counts @ Phi) + f(P["c"])
    loss = float(np.mean((np.logaddexp(0.0, z.astype(np.float64)) - y * z).astype(f)))
    dz = ((f(1) / (f(1) + np.exp(-z))) - y) / f(n)
    order = np.random.default_rng(seed).permutation(n)
    dPhi = f(0.5) * (counts[order].T @ dz[order])
    g = {}
    g["c"] = np.array(dz[order].sum(dtype=f))
    g["b3"] = np.array(dPhi[::-1].sum(dtype=f))
    g["W3"] = bf(H2).T @ dPhi
    dZ2 = (np.outer(dPhi, bf(P["W3"])) * mlp.gelu_grad(Z2.astype(np.float64)).astype(f)).astype(f)
    g["W2"] = bf(dZ2).T @ bf(H1)
    g["b2"] = dZ2[::-1].sum(axis=0, dtype=f)
    dH1 = bf(dZ2) @ bf(P["W2"])
    dZ1 = (dH1 * mlp.gelu_grad(Z1.astype(np.float64)).astype(f)).astype(f)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0, dtype=f)
    return loss, mlp.pack(g)


@pytest.mark.parametrize("L,n,seed", [(20, 300, 1), (70, 200, 2), (128, 150, 3)])
def test_grad_tolerance_covers_an_fp32_evaluation(L, n, seed):
    # the element-wise parity tolerance (twice the first-order running error bound of an
    # FP32 / BF16 evaluation) holds for an FP32 evaluation with its own rounding, order
    # and BF16 decisions
    theta = (mlp.init_params(7) + np.random.default_rng(L).normal(0, 0.05, mlp.N_PARAMS)).astype(np.float32)
    words, labels = random_batch(n, L, seed)
    loss, g = mlp.loss_and_grad(theta, words, labels, L, bf=True)
    tol_loss, tol = mlp.grad_tolerance(theta, words, labels, L)
    l32, g32 = _f32_evaluation(theta, words, labels, L, seed)
    assert abs(l32 - loss) <= tol_loss
    bad = np.abs(g32 - g) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:10], (np.abs(g32 - g) / tol).max())
    # the FP32 evaluation really does differ (it is not the oracle itself)
    assert np.abs(g32 - g).max() > 0


def test_grad_tolerance_rejects_planted_mistakes():
    # mistakes a kernel could make fail the element-wise check: a sign in one W1 or b1
    # element, a transposed W2 gradient, a dropped b3 term, a missing 1/2 in dPhi
    L, n = 40, 200
    theta = (mlp.init_params(11) + np.random.default_rng(4).normal(0, 0.05, mlp.N_PARAMS)).astype(np.float32)
    words, labels = random_batch(n, L, 9)
    _, g = mlp.loss_and_grad(theta, words, labels, L, bf=True)
    _, tol = mlp.grad_tolerance(theta, words, labels, L)
    off = {}
    k = 0
    for name, shape in mlp.SIZES:
        off[name] = (k, int(np.prod(shape)))
        k += int(np.prod(shape))

    def rejected(h):
        return bool((np.abs(h - g) > tol).any())

    for name in ("W1", "b1", "W3"):
        k0, m = off[name]
        i = k0 + int(np.argmax(np.abs(g[k0:k0 + m])))
        h = g.copy()
        h[i] = -h[i]
        assert rejected(h), name
    # W1: most elements are far above their tolerance, so a sign error anywhere is seen
    k0, m = off["W1"]
    assert np.mean(np.abs(g[k0:k0 + m]) > tol[k0:k0 + m]) > 0.8
    h = g.copy()
    k0, m = off["W2"]
    h[k0:k0 + m] = g[k0:k0 + m].reshape(128, 128).T.reshape(-1)
    assert rejected(h)
    h = g.copy()
    h[off["b3"][0]] = 0.0
    assert rejected(h)
    h = g.copy()
    k0, m = off["W3"]
    h[k0:k0 + m] *= 2.0
    assert rejected(h)
