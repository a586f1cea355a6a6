"""CPU oracle of the learned guiding potential (test infrastructure only; nothing in the
product package imports this module).

The potential is U(C) = sum_i phi(w_i(C)), w_i(C) the 9 sites i-4..i+4 (mod L) read as
a 9-bit pattern (bit k = site i-4+k), with phi a small MLP 9 -> 128 -> 128 -> 1 (GELU).
It is trained as a classifier between configurations drawn from the time-averaged
(ancestral) distribution p_ave (label 1) and from the end-of-interval distribution
p_end (label 0) of a biased population (Sec. 2.2, eqs. Opave and Opend).  For the SSEP
the tilted generator is symmetric, so p_end ~ v and p_ave ~ v^2 with v its top
eigenvector, and the Bayes logit ln(p_ave/p_end) = ln v + const is U/2 of the optimal
(Doob) control.  The logit of a configuration is therefore
    z(C) = (1/2) sum_i phi(w_i(C)) + c,
and the loss is the mean binary cross-entropy softplus(z) - y z.

Because a window has only 512 possible patterns, z(C) = (1/2) sum_p n_p(C) Phi_p + c with
Phi_p = phi(pattern p) and n_p(C) the number of windows of C showing pattern p: the
network is evaluated once per pattern, and dL/dPhi_p = (1/2) sum_n dz_n n_p(C_n).

Parameter vector (float32, this order): W1[128][9], b1[128], W2[128][128], b2[128],
W3[128], b3, c.  Products on the GPU take BF16 inputs and FP32 accumulation; with
bf16=True this oracle rounds the same operands to BF16 (round to nearest even) and
accumulates in FP64.
"""
import math

import numpy as np

H = 128
SIZES = (("W1", (H, 9)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", ()), ("c", ()))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def init_params(seed):
    """Deterministic initial parameters (uniform +-1/sqrt(fan_in)); biases zero."""
    g = np.random.default_rng(seed)
    p = {"W1": g.uniform(-1, 1, (H, 9)) / 3.0, "b1": np.zeros(H),
         "W2": g.uniform(-1, 1, (H, H)) / math.sqrt(H), "b2": np.zeros(H),
         "W3": g.uniform(-1, 1, H) / math.sqrt(H), "b3": np.zeros(()), "c": np.zeros(())}
    return pack(p).astype(np.float32)


def bf16(x):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def patterns():
    """The 512 window patterns as rows of 9 bits."""
    p = np.arange(512)
    return ((p[:, None] >> np.arange(9)[None, :]) & 1).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    return cdf + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, bf=False):
    """Phi (512,) and the saved activations."""
    P = unpack(theta)
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    X = patterns()
    Z1 = X @ r(P["W1"]).T + P["b1"]
    H1 = gelu(Z1)
    Z2 = r(H1) @ r(P["W2"]).T + P["b2"]
    H2 = gelu(Z2)
    Phi = r(H2) @ r(P["W3"]) + P["b3"]
    return Phi, dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def window_counts(words, L):
    """n_p(C) for each configuration: (n, 512) counts.  words: (n, W) uint64."""
    words = np.atleast_2d(np.asarray(words, dtype=np.uint64))
    n = words.shape[0]
    sites = np.zeros((n, L), dtype=np.int64)
    for i in range(L):
        sites[:, i] = (words[:, i // 64] >> np.uint64(i % 64)) & np.uint64(1)
    counts = np.zeros((n, 512), dtype=np.int64)
    for i in range(L):
        pat = np.zeros(n, dtype=np.int64)
        for k in range(9):
            pat |= sites[:, (i - 4 + k) % L] << k
        np.add.at(counts, (np.arange(n), pat), 1)
    return counts


def loss_and_grad(theta, words, labels, L, bf=False):
    """Mean BCE loss over the batch and its gradient with respect to theta."""
    P = unpack(theta)
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    Phi, A = forward(theta, bf)
    counts = window_counts(words, L).astype(np.float64)
    y = np.asarray(labels, dtype=np.float64)
    B = y.size
    z = 0.5 * counts @ Phi + P["c"]
    loss = float(np.mean(np.logaddexp(0.0, z) - y * z))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / B
    dPhi = 0.5 * counts.T @ dz
    g = {}
    g["c"] = np.array(dz.sum())
    g["b3"] = np.array(dPhi.sum())
    g["W3"] = r(A["H2"]).T @ dPhi
    dZ2 = np.outer(dPhi, r(P["W3"])) * gelu_grad(A["Z2"])
    g["W2"] = r(dZ2).T @ r(A["H1"])
    g["b2"] = dZ2.sum(axis=0)
    dH1 = r(dZ2) @ r(P["W2"])
    dZ1 = dH1 * gelu_grad(A["Z1"])
    g["W1"] = dZ1.T @ A["X"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, pack(g)


def loss_direct(theta, words, labels, L):
    """The same loss with the network run on every window of every configuration (no
    pattern counting), FP64: the definition the counted form must equal."""
    P = unpack(theta)
    words = np.atleast_2d(np.asarray(words, dtype=np.uint64))
    y = np.asarray(labels, dtype=np.float64)
    tot = 0.0
    for n in range(words.shape[0]):
        sites = [int((int(words[n, i // 64]) >> (i % 64)) & 1) for i in range(L)]
        z = P["c"]
        for i in range(L):
            x = np.array([sites[(i - 4 + k) % L] for k in range(9)], dtype=np.float64)
            h1 = gelu(P["W1"] @ x + P["b1"])
            h2 = gelu(P["W2"] @ h1 + P["b2"])
            z = z + 0.5 * (P["W3"] @ h2 + P["b3"])
        tot += math.log1p(math.exp(-abs(z))) + max(z, 0.0) - y[n] * z
    return tot / words.shape[0]


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), FP64 arithmetic on FP32 state; returns new state."""
    theta = np.asarray(theta, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta.astype(np.float32), m.astype(np.float32), v.astype(np.float32)
