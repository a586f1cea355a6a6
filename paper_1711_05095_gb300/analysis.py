"""Host-side crossover functions of an s-sweep (arXiv:1711.05095, Sec. 3.4).

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
