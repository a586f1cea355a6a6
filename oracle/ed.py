"""Exact diagonalisation of the tilted SSEP generator (test infrastructure only).

psi(s) = lim (1/t) ln < exp(-s K_t) >_0 (Sec. 2.1, eqs. biastraj and psi-z) is the
largest eigenvalue of the tilted generator built from eq. (P-Theta): every
transition C -> C' is multiplied by exp(-s) (each hop adds one to K), and the
diagonal holds minus the escape rate r(C).  For the SSEP (Sec. 3.1: a particle
hops with rate 1 to each empty neighbour on a ring) the rates are symmetric, so
the tilted generator is a real symmetric matrix.

Used only for small rings (C(L, N) states, L <= 14 in the tests).
"""
import itertools
import math

import numpy as np
import scipy.linalg


def basis(L, N):
    """All configurations with N particles on L sites, as integer bitmasks
    (site i = bit i), in increasing order."""
    out = []
    for occ in itertools.combinations(range(L), N):
        m = 0
        for i in occ:
            m |= 1 << i
        out.append(m)
    return np.array(sorted(out), dtype=np.int64)


def hops(L, mask):
    """(new_mask) for every allowed hop out of `mask` (Sec. 3.1 rules)."""
    res = []
    for i in range(L):
        j = (i + 1) % L
        a = (mask >> i) & 1
        b = (mask >> j) & 1
        if a != b:
            res.append(mask ^ (1 << i) ^ (1 << j))
    return res


def generator_parts(L, N):
    """Return (A, r, states): A[y, x] = number of hops x -> y (0/1), r = escape rates."""
    states = basis(L, N)
    index = {int(m): k for k, m in enumerate(states)}
    n = len(states)
    A = np.zeros((n, n))
    r = np.zeros(n)
    for x, m in enumerate(states):
        hs = hops(L, int(m))
        r[x] = len(hs)
        for m2 in hs:
            A[index[m2], x] += 1.0
    return A, r, states


def tilted_generator(L, N, s):
    A, r, _ = generator_parts(L, N)
    return math.exp(-s) * A - np.diag(r)


def psi_exact(L, N, s):
    """Largest eigenvalue of the (symmetric) tilted generator."""
    H = tilted_generator(L, N, s)
    return float(np.linalg.eigvalsh(H)[-1])


def psi_power(L, N, s, iters=20000, tol=1e-14):
    """The same eigenvalue by power iteration on H + c I (c = L makes every entry
    non-negative, so the Perron vector is the one reached); a check independent of
    the LAPACK routine."""
    H = tilted_generator(L, N, s)
    c = float(L)
    B = H + c * np.eye(H.shape[0])
    v = np.ones(H.shape[0])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = B @ v
        lam_new = float(v @ w)
        v = w / np.linalg.norm(w)
        if abs(lam_new - lam) < tol * max(1.0, abs(lam_new)):
            lam = lam_new
            break
        lam = lam_new
    return lam - c


def transient_generating_function(L, N, x0_mask, dt, z):
    """Exact E[ z^(hops in [0, dt]) ; C_dt = y | C_0 = x0 ] for all y: the column x0
    of expm(dt (z A - diag r)).  Returns (values, states)."""
    A, r, states = generator_parts(L, N)
    G = z * A - np.diag(r)
    E = scipy.linalg.expm(dt * G)
    x = int(np.nonzero(states == x0_mask)[0][0])
    return E[:, x], states
