"""Pins of the exact-diagonalisation oracle against closed forms and invariants.

* N = 1 (or one hole): the walker always has two neighbours, every hop is one
  unit of K, so the tilted generator is exp(-s) x (ring adjacency) - 2, whose top
  eigenvalue is 2 exp(-s) - 2 (Sec. 3.1 rates).
* psi(0) = 0 (Z(0, t) = 1, Sec. 2.1).
* -psi'(0) is the mean activity (eq. psi-mean); on a finite ring with N fixed it
  is 2 N (L-N) / (L-1) (the paper prints the grand-canonical 2 L rho (1-rho)).
* particle-hole symmetry psi(L, N) = psi(L, L-N).
* power iteration agrees with the dense symmetric eigensolver.
"""
import math

import numpy as np
import pytest

from oracle import ed


@pytest.mark.parametrize("L", [3, 5, 8, 11])
@pytest.mark.parametrize("s", [-0.7, -0.05, 0.0, 0.2, 1.3])
def test_single_particle_closed_form(L, s):
    assert ed.psi_exact(L, 1, s) == pytest.approx(2 * math.exp(-s) - 2, abs=1e-12)
    assert ed.psi_exact(L, L - 1, s) == pytest.approx(2 * math.exp(-s) - 2, abs=1e-12)


@pytest.mark.parametrize("L,N", [(6, 3), (9, 4), (12, 6)])
def test_psi_zero_at_s_zero(L, N):
    assert abs(ed.psi_exact(L, N, 0.0)) < 1e-12


@pytest.mark.parametrize("L,N", [(6, 2), (8, 4), (10, 5), (12, 6), (12, 3)])
def test_mean_activity_at_s_zero(L, N):
    h = 1e-5
    d = (ed.psi_exact(L, N, h) - ed.psi_exact(L, N, -h)) / (2 * h)
    assert -d == pytest.approx(2.0 * N * (L - N) / (L - 1), rel=1e-7)


@pytest.mark.parametrize("L,N,s", [(8, 3, 0.4), (10, 4, -0.3), (12, 5, 0.08)])
def test_particle_hole_symmetry(L, N, s):
    assert ed.psi_exact(L, N, s) == pytest.approx(ed.psi_exact(L, L - N, s), abs=1e-12)


@pytest.mark.parametrize("L,N,s", [(8, 4, 0.3), (10, 5, -0.2), (7, 3, 1.0)])
def test_power_iteration_agrees(L, N, s):
    assert ed.psi_power(L, N, s) == pytest.approx(ed.psi_exact(L, N, s), abs=1e-9)


def test_psi_convex_and_decreasing_through_zero():
    ss = np.linspace(-0.5, 0.5, 11)
    ps = np.array([ed.psi_exact(10, 5, s) for s in ss])
    assert np.all(np.diff(ps, 2) > 0)       # convex (eq. psi-var: psi'' >= 0)
    assert np.all(np.diff(ps) < 0)          # -psi' = activity > 0


def test_transient_is_a_probability():
    vals, states = ed.transient_generating_function(6, 3, 0b000111, 0.8, 1.0)
    assert np.all(vals >= -1e-15)
    assert vals.sum() == pytest.approx(1.0, abs=1e-12)
