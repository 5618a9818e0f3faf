"""Oracle: principal component scores and reconstruction, FP64.

Test infrastructure only: the library never imports this module.

Definitions followed
--------------------
* PACE, Eq. (2.7): A_il = lambda_l Phi_il' Sigma_Yi^{-1} Y_i^C with
  Sigma_Yi = sum_l lambda_l Phi_il Phi_il' + sigma^2 I (N_i x N_i),
  Phi_il = phi_l at subject i's observation points, Y_i^C = Y_i - mu(t_ij).
  Written out literally: one N_i x N_i solve per subject.
* Scores by integration (Section 2.1, dense data): A_il = integral of
  (Y_i(t) - mu(t)) phi_l(t) dt, as the Riemann sum over the observed nodes with
  the cell volume dV = prod_k 1/M_k.
* Reconstruction (Section 2.1): X_i(t) = mu(t) + sum_l A_il phi_l(t).
* MISE of a reconstruction (Section 4, Simulation I): (1/n) sum_i of the integral
  over Omega of (Xhat_i(t) - X_i(t))^2, the integral as the Riemann sum over all
  grid nodes with dV = prod_k 1/M_k.

Readings
--------
* Functions known on the grid (mu, phi) are evaluated at an observation through
  the bin that holds it (the binning of Section 3.2).
"""
from __future__ import annotations

import numpy as np

from .smoother import bin_of


def pace_scores_sparse(offs, t, y, m, mu, phi, lam, sigma2):
    """Eq. (2.7) for scattered data; phi is (P, L), lam (L,)."""
    offs = np.asarray(offs).astype(np.int64)
    b = bin_of(t, m)
    L = phi.shape[1]
    n = len(offs) - 1
    out = np.zeros((n, L))
    for i in range(n):
        sl = slice(offs[i], offs[i + 1])
        Phi = phi[b[sl], :]
        yc = np.asarray(y[sl], dtype=np.float64) - mu[b[sl]]
        S = (Phi * lam) @ Phi.T + sigma2 * np.eye(Phi.shape[0])
        if Phi.shape[0] == 0:
            continue
        x = np.linalg.solve(S, yc)
        out[i] = lam * (Phi.T @ x)
    return out


def pace_scores_dense(y, mask, mu, phi, lam, sigma2):
    """Eq. (2.7) for gridded data: the observed nodes of each subject."""
    y = np.asarray(y, dtype=np.float64)
    mk = np.asarray(mask).astype(bool)
    n, L = y.shape[0], phi.shape[1]
    out = np.zeros((n, L))
    for i in range(n):
        obs = np.nonzero(mk[i])[0]
        if obs.size == 0:
            continue
        Phi = phi[obs, :]
        S = (Phi * lam) @ Phi.T + sigma2 * np.eye(obs.size)
        out[i] = lam * (Phi.T @ np.linalg.solve(S, y[i, obs] - mu[obs]))
    return out


def integral_scores(y, mask, mu, phi, m):
    """Riemann sums of (Y_i - mu) phi_l over each subject's observed nodes."""
    y = np.asarray(y, dtype=np.float64)
    mk = np.asarray(mask).astype(bool)
    dv = 1.0 / float(np.prod(m))
    r = np.where(mk, y - mu[None, :], 0.0)
    return (r @ phi) * dv


def reconstruct(mu, phi, scores):
    """X_i = mu + sum_l A_il phi_l at the grid nodes (n x P)."""
    return mu[None, :] + np.asarray(scores) @ np.asarray(phi).T


def mise(xhat, x, m):
    """Mean over subjects of the Riemann sum of (xhat - x)^2 (n x P arrays)."""
    d = np.asarray(xhat, dtype=np.float64) - np.asarray(x, dtype=np.float64)
    dv = 1.0 / float(np.prod(m))
    return float(np.mean(np.sum(d * d, axis=1)) * dv)
