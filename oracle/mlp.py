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
accumulates in FP64, except the 9-input first layer, whose FP32 sum (in the GPU's order)
decides the BF16 codes of the first hidden layer.  running_error_bound / grad_tolerance
give the element-wise tolerance of an FP32 evaluation against these values.
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
    # with BF16 operands, Z1 is formed in FP32 in the GPU's order: GELU(Z1) is rounded to
    # a BF16 code, a decision both sides must take in the same precision
    Z1 = layer1_f32(theta) if bf else X @ P["W1"].T + P["b1"]
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


# ---------------------------------------------------------------------------
# Element-wise tolerance of an FP32 / BF16 evaluation of loss_and_grad(bf=True).
#
# The GPU evaluates the same network with every product's operands rounded to BF16
# (from FP32 values), products accumulated in FP32 (tensor cores or FP32 cores), and
# GELU, GELU', exp and log1p in FP32.  Against the FP64 values of loss_and_grad its
# results differ by (i) the FP32 rounding of every sum, at most gamma(n) = n u / (1 - n u)
# times the sum of the magnitudes of its n terms (u = 2^-24, the standard a-priori
# bound of a recursive sum in any order), (ii) a few ulp in each FP32 elementary
# function, and (iii) at a BF16 operand whose exact value lies within the error of its
# FP32 input of a rounding tie, one BF16 ulp (the two sides may round to different
# neighbours; away from a tie both round to the same BF16 value and the error is
# absorbed).  running_error_bound propagates these through the network to first order
# (each error times the magnitude of the derivative it meets); the tolerance of the
# parity tests is twice this bound, the factor covering the neglected second-order
# terms.
# ---------------------------------------------------------------------------
U32 = 2.0 ** -24


def _gamma(n):
    n = np.asarray(n, dtype=np.float64)
    return n * U32 / (1.0 - n * U32)


def _gamma_mma(k):
    """Accumulation bound of a K-term product on the tensor cores: K/16 steps of
    m16n8k16, each adding 16 exact BF16 products to the FP32 accumulator with at most a
    few units of rounding (three counted), plus the epilogue."""
    return _gamma(3 * (k // 16) + 4)


def layer1_f32(theta):
    """Z1 in FP32 in the order the GPU forms it (b1, then the BF16 weights of the set
    input bits in increasing k, each add rounded): the one FP32 value whose BF16 rounding
    (after GELU) the two sides must decide alike."""
    P = unpack(theta)
    X = patterns()
    bW1 = bf16(P["W1"]).astype(np.float32)
    z = np.broadcast_to(P["b1"].astype(np.float32), (512, H)).copy()
    for k in range(9):
        on = X[:, k] > 0
        z[on] = z[on] + bW1[:, k][None, :]
    return z.astype(np.float64)


def _bf16_ulp(x):
    """One BF16 ulp at |x| (8 significant bits), 2^-133 at 0."""
    a = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), 2.0 ** -126)
    return np.ldexp(1.0, (np.floor(np.log2(a)) - 7).astype(np.int64))


def _bf16_flip(x, e):
    """Error of the BF16 rounding of a value known to within e: where a rounding tie lies
    within e + |float32(x) - x| of x the two sides may take different neighbours, which
    differ by the BF16 ulp at the tie, at most that at |x|; elsewhere 0."""
    x = np.asarray(x, dtype=np.float64)
    ulp = _bf16_ulp(x)
    a = np.abs(x)
    mid = (np.floor(a / ulp - 0.5) + 0.5) * ulp       # the nearest tie at or below |x|
    d = np.minimum(np.abs(a - mid), np.abs(mid + ulp - a))
    near = d <= np.asarray(e, dtype=np.float64) + U32 * a + 1e-300
    return np.where(near, ulp, 0.0)


def _gelu_second(x):
    return np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi) * (2.0 - x * x)


def _gelu_fn_err(x):
    """Error of an FP32 GELU evaluated as 0.5 x erfc(-x / sqrt 2) (erfc to a few ulp, no
    cancellation): a few roundings relative to |GELU(x)|, plus the relative error u of the
    argument -x / sqrt 2 met by the derivative of erfc."""
    return 8.0 * U32 * (np.abs(gelu(x)) + np.abs(x) * np.abs(x) * np.exp(-0.5 * x * x))


def _gelu_grad_fn_err(x):
    """Error of an FP32 GELU' evaluated as 0.5 erfc(-x / sqrt 2) + x exp(-x^2/2) / sqrt(2 pi):
    a few roundings of each term plus the relative error x^2 u of the exponent's argument."""
    ax = np.abs(x)
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    return 8.0 * U32 * (cdf + ax * np.exp(-0.5 * x * x) * (1.0 + x * x))


def _forward_bound(theta):
    """Values and first-order error bounds of the forward pass (see the comment above)."""
    P = unpack(theta)
    X = patterns()
    bW1, bW2, bW3 = bf16(P["W1"]), bf16(P["W2"]), bf16(P["W3"])
    b1, b2, b3, c = P["b1"], P["b2"], P["b3"], P["c"]
    # forward
    Z1 = layer1_f32(theta)
    e_Z1 = np.zeros_like(Z1)
    H1 = gelu(Z1)
    e_H1 = np.abs(gelu_grad(Z1)) * e_Z1 + _gelu_fn_err(Z1)
    rH1 = bf16(H1)
    e_rH1 = _bf16_flip(H1, e_H1)
    Z2 = rH1 @ bW2.T + b2
    e_Z2 = e_rH1 @ np.abs(bW2).T + _gamma_mma(H) * (np.abs(rH1) @ np.abs(bW2).T + np.abs(b2))
    H2 = gelu(Z2)
    e_H2 = np.abs(gelu_grad(Z2)) * e_Z2 + _gelu_fn_err(Z2)
    rH2 = bf16(H2)
    e_rH2 = _bf16_flip(H2, e_H2)
    Phi = rH2 @ bW3 + b3
    e_Phi = e_rH2 @ np.abs(bW3) + _gamma(H + 2) * (np.abs(rH2) @ np.abs(bW3) + abs(b3))
    return dict(P=P, X=X, bW2=bW2, bW3=bW3, Z1=Z1, e_Z1=e_Z1, rH1=rH1, e_rH1=e_rH1, Z2=Z2,
                e_Z2=e_Z2, rH2=rH2, e_rH2=e_rH2, Phi=Phi, e_Phi=e_Phi)


def phi_tolerance(theta):
    """Element-wise tolerance of an FP32 / BF16 evaluation of forward(bf=True)'s Phi:
    twice its first-order running error bound."""
    return 2.0 * _forward_bound(theta)["e_Phi"]


def running_error_bound(theta, words, labels, L):
    """(loss bound, gradient bound) of an FP32 / BF16 evaluation, element-wise, to first
    order (see the comment above); the arrays match loss_and_grad's outputs."""
    f = _forward_bound(theta)
    P, X, bW2, bW3 = f["P"], f["X"], f["bW2"], f["bW3"]
    c = P["c"]
    Z1, e_Z1, rH1, e_rH1 = f["Z1"], f["e_Z1"], f["rH1"], f["e_rH1"]
    Z2, e_Z2, rH2, e_rH2 = f["Z2"], f["e_Z2"], f["rH2"], f["e_rH2"]
    Phi, e_Phi = f["Phi"], f["e_Phi"]
    # logits and loss
    counts = window_counts(words, L).astype(np.float64)
    y = np.asarray(labels, dtype=np.float64)
    n = y.size
    z = 0.5 * counts @ Phi + c
    e_z = 0.5 * counts @ e_Phi + _gamma(L + 2) * (0.5 * counts @ np.abs(Phi) + abs(c))
    e_loss = float(np.mean(e_z + 6.0 * U32 * (np.abs(z) + 1.0)))
    sig = 1.0 / (1.0 + np.exp(-z))
    dz = (sig - y) / n
    e_dz = (0.25 * e_z + 6.0 * U32) / n
    # back-propagation
    e_grad = {}
    adz = np.abs(dz)
    e_grad["c"] = np.array(e_dz.sum() + _gamma(n + 1) * adz.sum())
    ntot = counts.sum(axis=0)
    dPhi = 0.5 * counts.T @ dz
    e_dPhi = 0.5 * counts.T @ e_dz + _gamma(ntot + n + 1) * (0.5 * counts.T @ adz)
    adPhi = np.abs(dPhi)
    e_grad["b3"] = np.array(e_dPhi.sum() + _gamma(2 * 512) * adPhi.sum())
    e_grad["W3"] = e_rH2.T @ adPhi + np.abs(rH2).T @ e_dPhi + _gamma(2 * 512) * (np.abs(rH2).T @ adPhi)
    g2 = gelu_grad(Z2)
    dZ2 = np.outer(dPhi, bW3) * g2
    e_dZ2 = (np.outer(e_dPhi, np.abs(bW3)) * np.abs(g2)
             + np.outer(adPhi, np.abs(bW3)) * (np.abs(_gelu_second(Z2)) * e_Z2 + _gelu_grad_fn_err(Z2))
             + 3.0 * U32 * np.abs(dZ2))
    rdZ2 = bf16(dZ2)
    e_rdZ2 = _bf16_flip(dZ2, e_dZ2)
    arH1, ardZ2 = np.abs(rH1), np.abs(rdZ2)
    e_grad["W2"] = (e_rdZ2.T @ arH1 + ardZ2.T @ e_rH1 + e_rdZ2.T @ e_rH1
                    + _gamma_mma(512) * (ardZ2.T @ arH1))
    e_grad["b2"] = e_dZ2.sum(axis=0) + _gamma(2 * 512) * np.abs(dZ2).sum(axis=0)
    dH1 = rdZ2 @ bW2
    e_dH1 = e_rdZ2 @ np.abs(bW2) + _gamma_mma(H) * (ardZ2 @ np.abs(bW2))
    g1 = gelu_grad(Z1)
    dZ1 = dH1 * g1
    e_dZ1 = (e_dH1 * np.abs(g1) + np.abs(dH1) * (np.abs(_gelu_second(Z1)) * e_Z1 + _gelu_grad_fn_err(Z1))
             + U32 * np.abs(dZ1))
    e_grad["b1"] = e_dZ1.sum(axis=0) + _gamma(2 * 512) * np.abs(dZ1).sum(axis=0)
    e_grad["W1"] = e_dZ1.T @ X + _gamma(2 * 512) * (np.abs(dZ1).T @ X)
    return e_loss, pack(e_grad)


def grad_tolerance(theta, words, labels, L):
    """The parity tolerance: twice the first-order running error bound, element-wise."""
    e_loss, e_grad = running_error_bound(theta, words, labels, L)
    return 2.0 * e_loss, 2.0 * e_grad
