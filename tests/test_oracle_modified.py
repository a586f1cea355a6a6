"""Pins of the oracle's MODIFIED dynamics (Sec. 3.2, eq. def-ups-ssep) and [iid]
selection (Sec. 4.1), against what the mathematics fixes:

* the modified process has generator e^-s (A - diag r); its weight exp(-(1-e^-s) A),
  A = integral of r, adds -(1-e^-s) diag r, so E[Upsilon 1{C_dt = y} | C_0] is the
  exact tilted transient expm(dt (e^-s A - diag r)) (ED module);
* the specified FP32 exponential against FP64 exp;
* the psi term from quantised weights against the FP64 definition;
* psi_hat against exact diagonalisation, and against the plain estimator;
* [iid] ancestors against a brute force with exact integers.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import ed


def mask_of(row):
    m = 0
    for i, v in enumerate(row):
        if v:
            m |= 1 << i
    return m


def test_weight_exp_against_fp64():
    rng = np.random.default_rng(3)
    F = 47
    xs = list(-rng.exponential(3.0, size=4000)) + [0.0, -1e-9, -1e-6, -0.5, -30.0, -80.0]
    for x in xs:
        x = float(np.float32(x))
        got = oracle.weight_exp(x, F)
        exact = math.ldexp(math.exp(x), F)
        assert abs(got - exact) <= 2e-7 * exact + 1.0, (x, got, exact)


@pytest.mark.parametrize("L,N,x0,dt,s", [(6, 3, 0b000111, 0.6, 0.4), (5, 2, 0b00101, 0.5, -0.5)])
def test_modified_weight_gives_tilted_transient(L, N, x0, dt, s):
    n = 200000
    start = np.array([(x0 >> i) & 1 for i in range(L)], dtype=np.uint8)
    out, dK, A = oracle.evolve_sites_modified(L, np.tile(start, (n, 1)), dt, s, beta=2, seed=99)
    c = -math.expm1(-s)
    ups = np.exp(-c * A.astype(np.float64))
    states = ed.basis(L, N)
    idx = {int(m): k for k, m in enumerate(states)}
    ends = np.array([idx[mask_of(r)] for r in out])
    H = ed.tilted_generator(L, N, s)
    exact = scipy.linalg.expm(dt * H)[:, int(np.nonzero(states == x0)[0][0])]
    for y in range(len(states)):
        vals = ups * (ends == y)
        assert abs(vals.mean() - exact[y]) <= 5 * vals.std() / math.sqrt(n) + 1e-12, y
    # the activity and the rate-scaled hop law: mean hops = E[int e^-s r dt]
    assert abs(dK.mean() - math.exp(-s) * A.mean()) <= 5 * dK.std() / math.sqrt(n)


@pytest.mark.parametrize("s", [0.2, -0.3, 1e-4])
def test_modified_psi_term_against_definition(s):
    rng = np.random.default_rng(11)
    A = rng.gamma(4.0, 1.0, size=5000).astype(np.float32)
    spec = oracle.psi_term_modified(s, A)
    c = -math.expm1(-s)
    ref = A.min() if s >= 0 else A.max()
    exact = -c * float(ref) + math.log(math.fsum(math.exp(-c * (float(a) - float(ref))) for a in A) / A.size)
    # FP32 weights: a few 1e-8 per weight, averaged
    assert abs(spec - exact) <= 2e-7 * max(1.0, abs(exact)), (spec, exact)


@pytest.mark.parametrize("s", [0.1, -0.1])
def test_modified_matches_exact_diagonalisation(s):
    L, N = 12, 6
    exact = ed.psi_exact(L, N, s)
    runs = [oracle.run(L, N, 1024, seed, s, 0.1, 1000, modified=True)["psi"] for seed in range(8)]
    m, se = np.mean(runs), np.std(runs, ddof=1) / np.sqrt(len(runs))
    assert abs(m - exact) <= 5 * se + 0.01 * abs(exact), (m, se, exact)


def test_modified_agrees_with_plain():
    s = 0.3
    a = [oracle.run(10, 5, 512, seed, s, 0.1, 800, modified=True)["psi"] for seed in range(6)]
    b = [oracle.run(10, 5, 512, seed, s, 0.1, 800)["psi"] for seed in range(6)]
    se = math.sqrt(np.var(a, ddof=1) / 6 + np.var(b, ddof=1) / 6)
    assert abs(np.mean(a) - np.mean(b)) <= 5 * se + 2e-3


def test_modified_single_particle_closed_form():
    s = 0.4
    runs = [oracle.run(10, 1, 1000, seed, s, 0.1, 500, modified=True)["psi"] for seed in range(6)]
    m, se = np.mean(runs), np.std(runs, ddof=1) / np.sqrt(len(runs))
    assert abs(m - 2 * (math.exp(-s) - 1)) <= 5 * se + 2e-3


@pytest.mark.parametrize("n", [1, 9, 300])
def test_iid_ancestors_brute_force(n):
    rng = np.random.default_rng(n)
    w = rng.integers(0, 2**40, size=n, dtype=np.uint64)
    w[rng.random(n) < 0.3] = 0
    if w.sum() == 0:
        w[0] = 1
    beta, seed = 4, 31
    anc = oracle.ancestors_iid(w, beta, seed)
    S = [0]
    for v in w:
        S.append(S[-1] + int(v))
    T = S[-1]
    for j in range(n):
        r = oracle.philox([j, beta, 0, 4], seed)
        u = (int(r[1]) << 32) | int(r[0])
        alpha = (u * T) >> 64
        k = next(k for k in range(n) if S[k] <= alpha < S[k + 1])
        assert anc[j] == k
    assert np.all(w[anc] > 0)


def test_iid_copy_counts_are_multinomial():
    n = 2000
    w = np.full(n, 2**30, dtype=np.uint64)
    w[:n // 2] *= 3   # first half three times as likely
    counts = np.zeros(n)
    R = 50
    for beta in range(1, R + 1):
        counts += np.bincount(oracle.ancestors_iid(w, beta, 7), minlength=n)
    heavy, light = counts[:n // 2].sum() / R, counts[n // 2:].sum() / R
    assert abs(heavy - 0.75 * n) <= 5 * math.sqrt(n * 0.75 * 0.25 / R)
    assert abs(heavy + light - n) < 1e-9


def test_eq_selection_has_smaller_variance_than_iid():
    # Sec. 4.4: at the same N_c, equally spaced points ([eq]) give a smaller variance of
    # k-hat than independent ones ([iid]), which delete clones that [eq] keeps; with 40
    # runs each, equal variances would give a ratio above 1.9 with probability < 2.5 %
    L, N, s = 12, 6, 0.1
    eq = [oracle.run(L, N, 128, seed, s, 0.1, 500)["k_hat"] for seed in range(40)]
    iid = [oracle.run(L, N, 128, seed, s, 0.1, 500, iid=True)["k_hat"] for seed in range(40)]
    assert np.var(iid, ddof=1) > 2.5 * np.var(eq, ddof=1)
