"""Pins of the finite-size extrapolation k(x) = k_inf (1 + A / x) of arXiv:1711.05095
(eq. fit-finite-tmax, x = t_obs, Sec. 5.1; eq. fit-finite-nc, x = N_c, Sec. 5.2):

* against the values the paper prints (tests/golden/finite_size_fits.txt): the printed
  "difference in k_inf" rows fix how that difference is taken (the paper prints no
  k values at the tabulated x, so the fit itself cannot be pinned to the tables);
* an algebra check of the fit (not a pin to the paper): points made from a printed
  (k_inf, A) give them back;
* against exact diagonalisation: extrapolating the oracle's psi over N_c removes most
  of its O(1/N_c) bias.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import ed
from paper_1711_05095_gb300 import analysis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "finite_size_fits.txt")


def golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t, L, method, A, k_exc, k_inc, diff, x1, x2, x3 = line.split()
            rows.append(dict(table=t, L=int(L), method=method, A=float(A), k_exc=float(k_exc),
                             k_inc=float(k_inc), diff=diff, x=(float(x1), float(x2), float(x3))))
    return rows


ROWS = golden_rows()


def test_golden_file_holds_both_tables():
    assert len(ROWS) == 10
    assert sum(r["table"] == "tmax" for r in ROWS) == 6 and sum(r["table"] == "nc" for r in ROWS) == 4


@pytest.mark.parametrize("row", ROWS, ids=lambda r: "%s-L%d-%s" % (r["table"], r["L"], r["method"]))
def test_two_point_fit_algebra(row):
    # an algebra check of fit_finite, not a pin to the paper's tables (whose k values at
    # each x are not printed): points made from a printed (k_inf, A) give them back
    x1, x2, _ = row["x"]
    k = [row["k_exc"] * (1.0 + row["A"] / x) for x in (x1, x2)]
    k_inf, A = analysis.fit_finite([x1, x2], k)
    assert abs(k_inf - row["k_exc"]) < 1e-12
    assert abs(A - row["A"]) < 1e-9 * max(1.0, row["A"])
    # the fitted k at the two points differs from k_inf by A/x in relative terms
    assert np.allclose(np.array(k) / k_inf - 1.0, [A / x1, A / x2], rtol=1e-9)


@pytest.mark.parametrize("row", ROWS, ids=lambda r: "%s-L%d-%s" % (r["table"], r["L"], r["method"]))
def test_printed_difference_is_relative_to_the_two_point_value(row):
    # reading: difference = |k_inf(incl.) - k_inf(exc.)| / k_inf(exc.), in percent,
    # printed to one decimal
    d = 100.0 * abs(row["k_inc"] - row["k_exc"]) / row["k_exc"]
    if row["diff"].startswith("<"):
        assert d < float(row["diff"][1:])
    else:
        assert abs(d - float(row["diff"])) <= 0.05 + 1e-9, (d, row["diff"])


def test_fit_rejects_bad_input():
    with pytest.raises(ValueError):
        analysis.fit_finite([1.0], [0.5])
    with pytest.raises(ValueError):
        analysis.fit_finite([1.0, 0.0], [0.5, 0.4])
    with pytest.raises(ValueError):
        analysis.fit_finite([1.0, 2.0], [0.5])


def test_extrapolation_in_nc_removes_the_cloning_bias():
    # strong bias and few clones (L = 8, N = 4, s = 1): the oracle's psi is biased by
    # A / N_c; the fit over N_c = 16, 32, 64 lands far closer to exact psi than the
    # largest population does (seeded runs, so the figures are fixed)
    L, N, s = 8, 4, 1.0
    exact = ed.psi_exact(L, N, s)
    ncs = [16, 32, 64]
    means, ses = [], []
    for nc in ncs:
        runs = [oracle.run(L, N, nc, seed, s, 0.1, 4000)["psi"] for seed in range(24)]
        means.append(np.mean(runs))
        ses.append(np.std(runs, ddof=1) / np.sqrt(len(runs)))
    raw = abs(means[-1] - exact)
    assert raw > 5 * ses[-1]                      # the bias is resolved at N_c = 64
    psi_inf, A = analysis.fit_finite(ncs, means)
    assert abs(psi_inf - exact) < 0.25 * raw, (psi_inf, exact, raw)
    assert A > 0    # psi < 0 and biased low: |psi(N_c)| = |psi_inf| (1 + A / N_c), A > 0
