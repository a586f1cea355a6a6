"""Pins of the cloning oracle (oracle/cloning_oracle.c) against what the paper and
the mathematics fix, never against itself.

Dynamics (Sec. 3.1 rates, Sec. 4 BKL):
  * the law of (C_dt, hops in [0, dt]) from a fixed start equals the exact
    transient expm(dt (z A - diag r)) of the counting generator (ED module);
  * P(no hop) = exp(-r(C_0) dt); particle number is conserved; K = sum dK;
  * mean activity in the steady state is 2 N (L-N) / (L-1).
Initial condition: a uniform N-subset (chi-square over all C(L, N) states).
Selection (Sec. 4.1, eq. alpha-Ups): brute force with exact rationals, the copy
  count bounds floor/ceil(N_c w_k / T), monotone ancestors, identity at equal
  weights, zero weights never chosen.
Estimator (eq. psihat): exact 0 at s = 0; the single-particle closed form
  2(e^-s - 1); exact psi from ED at L = 12; the O(1/N_c) bias of eq. (fit-finite-nc).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import ed


def mask_of(row):
    m = 0
    for i, v in enumerate(row):
        if v:
            m |= 1 << i
    return m


# ---------------------------------------------------------------- initial state

@pytest.mark.parametrize("L,N", [(6, 3), (7, 2)])
def test_init_is_uniform_subset(L, N):
    n = 60000
    sites = oracle.init_sites(L, N, n, seed=11)
    assert np.all(sites.sum(axis=1) == N)
    states = ed.basis(L, N)
    idx = {int(m): k for k, m in enumerate(states)}
    counts = np.zeros(len(states))
    for row in sites:
        counts[idx[mask_of(row)]] += 1
    exp = n / len(states)
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    dof = len(states) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


@pytest.mark.parametrize("N", [0, 5])
def test_init_empty_and_full(N):
    sites = oracle.init_sites(5, N, 10, seed=1)
    assert np.all(sites.sum(axis=1) == N)


# ---------------------------------------------------------------- dynamics

@pytest.mark.parametrize("L,N,x0,dt", [(6, 3, 0b000111, 0.7), (5, 2, 0b00101, 0.4)])
def test_transient_law_matches_matrix_exponential(L, N, x0, dt):
    n = 200000
    start = np.array([(x0 >> i) & 1 for i in range(L)], dtype=np.uint8)
    sites = np.tile(start, (n, 1))
    out, K, dK = oracle.evolve_sites(L, sites, dt, beta=3, seed=2024)
    assert np.all(out.sum(axis=1) == N)
    assert np.array_equal(K, dK)
    states = ed.basis(L, N)
    idx = {int(m): k for k, m in enumerate(states)}
    ends = np.array([idx[mask_of(r)] for r in out])
    # final-state law (z = 1)
    p_exact, _ = ed.transient_generating_function(L, N, x0, dt, 1.0)
    p_emp = np.bincount(ends, minlength=len(states)) / n
    sd = np.sqrt(p_exact * (1 - p_exact) / n)
    assert np.all(np.abs(p_emp - p_exact) <= 5 * sd + 1e-12)
    # hop-count generating function at z != 1, summed over end states
    for z in (0.5, 1.7):
        g_exact = float(ed.transient_generating_function(L, N, x0, dt, z)[0].sum())
        samples = z ** dK.astype(np.float64)
        assert abs(samples.mean() - g_exact) <= 5 * samples.std() / np.sqrt(n)
    # no hop at all: exp(-r(x0) dt)
    r0 = len(ed.hops(L, x0))
    q = math.exp(-r0 * dt)
    assert abs((dK == 0).mean() - q) <= 5 * math.sqrt(q * (1 - q) / n)


def test_steady_state_mean_activity():
    L, N, n, dt = 20, 10, 20000, 0.5
    sites = oracle.init_sites(L, N, n, seed=3)
    _, _, dK = oracle.evolve_sites(L, sites, dt, beta=1, seed=3)
    mean = dK.mean() / dt
    exact = 2.0 * N * (L - N) / (L - 1)
    assert abs(mean - exact) <= 5 * dK.std() / dt / math.sqrt(n)


def test_no_particles_no_hops():
    for N in (0, 7):
        sites = oracle.init_sites(7, N, 16, seed=1)
        out, K, dK = oracle.evolve_sites(7, sites, 5.0, beta=1, seed=1)
        assert np.all(dK == 0) and np.array_equal(out, sites)


# ---------------------------------------------------------------- selection

def brute_force_ancestors(w, U):
    """eq. (alpha-Ups) with exact rationals: alpha_j = (j + d) T / N_c, 0-based j,
    d = (U + 1/2) / 2^32; ancestor = 0-based k with S_k <= alpha_j < S_{k+1}."""
    n = len(w)
    T = sum(int(v) for v in w)
    d = Fraction(2 * U + 1, 2**33)
    S = [0]
    for v in w:
        S.append(S[-1] + int(v))
    out = []
    for j in range(n):
        a = (j + d) * T / n
        k = next(k for k in range(n) if S[k] <= a < S[k + 1])
        out.append(k)
    return np.array(out)


@pytest.mark.parametrize("n,zero_frac", [(1, 0.0), (7, 0.0), (50, 0.3), (257, 0.5)])
def test_ancestors_brute_force(n, zero_frac):
    rng = np.random.default_rng(n)
    for trial in range(4):
        w = rng.integers(0, 2**40, size=n, dtype=np.uint64)
        w[rng.random(n) < zero_frac] = 0
        if w.sum() == 0:
            w[0] = 1
        beta, seed = 5 + trial, 77
        anc = oracle.ancestors(w, beta, seed)
        U = oracle.resample_word(beta, seed)
        assert np.array_equal(anc, brute_force_ancestors(w, U))
        T = int(w.sum(dtype=np.uint64))
        copies = np.bincount(anc, minlength=n)
        assert copies.sum() == n
        assert np.all(np.diff(anc) >= 0)
        assert np.all(copies[w == 0] == 0)
        for k in range(n):
            lo = (n * int(w[k])) // T
            hi = -((-n * int(w[k])) // T)
            assert lo <= copies[k] <= hi


def test_equal_weights_identity():
    w = np.full(1000, 2**40, dtype=np.uint64)
    for beta in range(1, 6):
        assert np.array_equal(oracle.ancestors(w, beta, 9), np.arange(1000))


def test_weight_quantisation():
    n = 16384
    F = oracle.weight_scale(n)
    assert F == 61 - 14
    rng = np.random.default_rng(1)
    dK = rng.poisson(3.0, size=n).astype(np.int32)
    for s in (0.3, -0.3, 0.0, 1e-5):
        w, rc = oracle.weights(s, dK)
        assert rc == 0
        ref = dK.min() if s >= 0 else dK.max()
        assert np.all(w[dK == ref] == 2**F)
        k = np.abs(dK.astype(np.int64) - ref)
        target = np.ldexp(np.exp(-abs(s) * k), F)
        assert np.all(np.abs(w.astype(np.float64) - target) <= 0.5 + target * 2.0**-52)
        assert int(w.sum(dtype=np.uint64)) <= 2**61
    # worst case: all weights maximal at N_c = 2^20 still fits
    assert (2**20) * 2 ** oracle.weight_scale(2**20) == 2**61
    # out-of-range activity is reported, never silently clamped
    bad = np.array([0, 5000], dtype=np.int32)
    _, rc = oracle.weights(0.1, bad)
    assert rc == -3


# ---------------------------------------------------------------- estimator

def test_psi_term_definition():
    rng = np.random.default_rng(4)
    dK = rng.poisson(2.0, size=3000).astype(np.int32)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    counts = np.bincount(dK)
    for s in (0.2, -0.2, 1e-6, -3e-5, 2.5):
        ms = mpmath.mpf(s)
        total = mpmath.fsum(int(c) * mpmath.exp(-ms * k) for k, c in enumerate(counts) if c)
        exact = float(mpmath.log(total / dK.size))
        assert oracle.psi_term(s, dK) == pytest.approx(exact, rel=1e-14, abs=1e-300)


def test_s_zero_is_exact_and_identity():
    pop = oracle.Population(20, 10, 500, seed=8)
    for _ in range(20):
        pop.evolve(0.1)
        term, rc = pop.resample(0.0)
        assert term == 0.0 and rc == 0
        assert np.array_equal(pop.anc, np.arange(500))
    psi, khat = pop.estimates()
    assert psi == 0.0 and khat > 0


@pytest.mark.parametrize("s", [0.3, -0.4])
def test_single_particle_closed_form(s):
    # one particle: escape rate is always 2, so the estimate must converge to
    # 2(e^-s - 1) whatever the selection does
    runs = [oracle.run(10, 1, 1000, seed, s, 0.1, 500)["psi"] for seed in range(6)]
    m, se = np.mean(runs), np.std(runs, ddof=1) / np.sqrt(len(runs))
    assert abs(m - 2 * (math.exp(-s) - 1)) <= 5 * se + 2e-3


@pytest.mark.parametrize("s", [0.1, -0.1])
def test_matches_exact_diagonalisation(s):
    L, N = 12, 6
    exact = ed.psi_exact(L, N, s)
    runs = [oracle.run(L, N, 1024, seed, s, 0.1, 1000)["psi"] for seed in range(8)]
    m, se = np.mean(runs), np.std(runs, ddof=1) / np.sqrt(len(runs))
    # statistical error, plus O(1/N_c) and O(1/t_obs) systematic allowances
    assert abs(m - exact) <= 5 * se + 0.01 * abs(exact), (m, se, exact)


def test_bias_scales_as_one_over_nc():
    # eq. (fit-finite-nc): systematic error ~ A / N_c.  Small clone numbers at a
    # strong bias make the bias large enough to measure against exact psi.
    L, N, s = 8, 4, 1.0
    exact = ed.psi_exact(L, N, s)
    ncs = [4, 8, 16, 32]
    bias = []
    for nc in ncs:
        runs = [oracle.run(L, N, nc, seed, s, 0.1, 4000)["psi"] for seed in range(24)]
        bias.append(np.mean(runs) - exact)
    bias = np.array(bias)
    assert np.all(bias < 0) or np.all(bias > 0)
    slope = np.polyfit(np.log(ncs), np.log(np.abs(bias)), 1)[0]
    assert -1.5 < slope < -0.6, (bias, slope)


def test_particle_hole_symmetry_statistical():
    s = 0.2
    a = [oracle.run(9, 3, 512, seed, s, 0.1, 1000)["psi"] for seed in range(6)]
    b = [oracle.run(9, 6, 512, seed, s, 0.1, 1000)["psi"] for seed in range(6)]
    se = math.sqrt(np.var(a, ddof=1) / 6 + np.var(b, ddof=1) / 6)
    assert abs(np.mean(a) - np.mean(b)) <= 5 * se + 1e-3


@pytest.mark.parametrize("s", [0.0, 0.15])
def test_khat_matches_exact_activity(s):
    # eq. (khat) with the carried cumulative K (Sec. 4.2) estimates k(s) =
    # -psi'(s)/L (eq. def-calK); the exact derivative comes from ED
    L, N = 12, 6
    h = 1e-5
    k_exact = -(ed.psi_exact(L, N, s + h) - ed.psi_exact(L, N, s - h)) / (2 * h) / L
    runs = [oracle.run(L, N, 1024, seed, s, 0.1, 1000)["k_hat"] for seed in range(8)]
    m, se = np.mean(runs), np.std(runs, ddof=1) / np.sqrt(len(runs))
    assert abs(m - k_exact) <= 5 * se + 0.01 * k_exact, (m, se, k_exact)
