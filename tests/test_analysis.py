"""Crossover functions from an exact psi(lambda) grid (ED): K_L(0) is the exact mean
activity per site 2 N (L-N) / ((L-1) L) (eq. psi-mean), chi_L >= 0 (eq. psi-var,
convexity), K_L decreases with lambda, phi_L(0) = 0."""
import numpy as np
import pytest

from oracle import ed
from paper_1711_05095_gb300 import analysis


def test_crossover_from_exact_psi():
    L, N = 10, 5
    lam = np.linspace(-6.0, 6.0, 25)
    psi = np.array([ed.psi_exact(L, N, l / L**2) for l in lam])
    out = analysis.crossover(lam, psi, L)
    i0 = int(np.argmin(np.abs(out["lam"])))
    assert out["K"][i0] == pytest.approx(2.0 * N * (L - N) / ((L - 1) * L), rel=1e-3)
    assert np.all(out["chi"][2:-2] > 0)
    assert np.all(np.diff(out["K"]) < 0)
    assert abs(out["phi"][i0]) < 1e-12


def test_crossover_rejects_bad_input():
    with pytest.raises(ValueError):
        analysis.crossover([0.0, 1.0], [0.0, 1.0], 10)
