"""Pins of the oracle's Fourier density mode (eq. fourdens) against closed forms:
for independent uniform N-subsets of the ring, E|delta rho_n|^2 for n != 0 mod L is
(N/L) (L - N) / (L - 1) (the sum of e^{-2 pi i n X_j/L} over a uniform N-subset has
second moment N (L - N) / (L - 1)); n = 0 gives N^2 / L exactly; a single cluster
of N adjacent particles gives sin^2(pi n N / L) / (L sin^2(pi n / L))."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("L,N,n", [(20, 10, 1), (50, 25, 1), (50, 10, 3), (128, 64, 1)])
def test_uniform_subsets(L, N, n):
    sites = oracle.init_sites(L, N, 40000, seed=5)
    got = oracle.density_mode(sites, n)
    exact = N * (L - N) / ((L - 1) * L)
    # per-clone values are O(1) with spread ~ their mean
    assert abs(got - exact) <= 5 * 1.2 * exact / math.sqrt(40000)


def test_zero_mode_and_cluster():
    L, N = 30, 12
    sites = oracle.init_sites(L, N, 100, seed=1)
    assert oracle.density_mode(sites, 0) == pytest.approx(N * N / L, rel=1e-6)
    cluster = np.zeros((1, L), dtype=np.uint8)
    cluster[0, 7:7 + N] = 1
    for n in (1, 2, 5):
        exact = math.sin(math.pi * n * N / L) ** 2 / (L * math.sin(math.pi * n / L) ** 2)
        assert oracle.density_mode(cluster, n) == pytest.approx(exact, rel=1e-5, abs=1e-6)
