"""Host-side analysis of cloning estimates (arXiv:1711.05095): the crossover functions
of an s-sweep (Sec. 3.4) and the finite-t_obs / finite-N_c extrapolations (Sec. 5).

From psi(s) estimated on a grid of lambda = s L^2 (eq. def-lambda):
  phi_L(lambda) = L psi(lambda / L^2)                      (rescaled free energy)
  K_L(lambda)   = -psi'(s) / L                             (eq. def-calK)
  chi_L(lambda) = psi''(s) / L,  X_L = -dK_L/dlambda       (eq. def-chi)
Derivatives are second-order finite differences on the (possibly uneven) grid.
The direct activity estimator k_hat (eq. khat) estimates K_L without differencing.
"""
import numpy as np


def crossover(lam, psi, L):
    lam = np.asarray(lam, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    if lam.ndim != 1 or lam.shape != psi.shape or lam.size < 3:
        raise ValueError("need matching 1-d arrays of at least 3 points")
    order = np.argsort(lam)
    lam, psi = lam[order], psi[order]
    s = lam / L**2
    dpsi = np.gradient(psi, s, edge_order=2)
    d2psi = np.gradient(dpsi, s, edge_order=2)
    K = -dpsi / L
    return dict(lam=lam, phi=L * psi, K=K, chi=d2psi / L, X=-np.gradient(K, lam, edge_order=2))


def fit_finite(x, k):
    """Extrapolation of an estimate k measured at several finite values x of the run
    length (x = t_obs, eq. fit-finite-tmax, Sec. 5.1) or of the population size
    (x = N_c, eq. fit-finite-nc, Sec. 5.2): k(x) = k_inf (1 + A / x) + O(x^-2).
    Least squares in the linear form k = a + b / x with a = k_inf and b = k_inf A, so
    two points give the exact two-point fit the paper tabulates.  Returns (k_inf, A).
    """
    x = np.asarray(x, dtype=np.float64)
    k = np.asarray(k, dtype=np.float64)
    if x.ndim != 1 or x.shape != k.shape or x.size < 2 or np.any(x <= 0):
        raise ValueError("need matching 1-d arrays of at least 2 points with x > 0")
    M = np.stack([np.ones_like(x), 1.0 / x], axis=1)
    (a, b), *_ = np.linalg.lstsq(M, k, rcond=None)
    return float(a), float(b / a)
