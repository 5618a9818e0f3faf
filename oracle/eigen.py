"""Oracle: matrixisation, eigendecomposition and random projection, FP64.

Test infrastructure only: the library never imports this module.

* Matrixisation, Section 3.1: Gamma_hat on the grid is reshaped to the P x P
  matrix Sigma (row = s flattened in C order, column = t).  The Riemann sums
  of the eigen-equations Eq. (3.1) give lambda = lambda_tilde * dV and
  phi = psi / sqrt(dV), dV = prod_k 1/M_k, so that sum phi^2 dV = 1.  For an
  irregular domain Omega the grid is the bounding box and Gamma is set to zero
  when s or t lies outside Omega.
* Random projection, Section 3.4: eigenpairs of a small projected matrix
  Q' Sigma Q stand in for those of Sigma.  The oracle follows the range-finder
  form of Halko, Martinsson and Tropp (the reference the paper builds on):
  Y = Sigma Omega, ``q`` rounds of re-orthonormalised power iteration,
  Q = orth(Y), B = Q' Sigma Q, B = U diag(theta) U', Psi = Q U.

Readings
* Omega (domain) = the bins where at least one observation fell.
* Sigma is symmetrised as (G + G')/2, and entries that are NaN (EMPTY points)
  are set to zero, as are rows and columns outside Omega.
* Sign: each eigenvector is flipped so that its entry of largest magnitude is
  positive.
* FVE_k = sum_{j<=k} lambda_j / (trace(Sigma) dV): the trace is available to
  both the full and the projected method.
"""
from __future__ import annotations

import numpy as np


def cell_volume(m):
    return 1.0 / float(np.prod(m))


def matrixize(G, domain):
    """Sigma = sym(G) with NaNs and out-of-domain rows/columns set to zero."""
    S = np.where(np.isnan(G), 0.0, np.asarray(G, dtype=np.float64))
    S = 0.5 * (S + S.T)
    dm = np.asarray(domain).astype(bool)
    S[~dm, :] = 0.0
    S[:, ~dm] = 0.0
    return S


def fix_signs(vecs):
    """Flip columns so that each column's entry of largest magnitude is positive."""
    vecs = np.array(vecs, dtype=np.float64, copy=True)
    for j in range(vecs.shape[1]):
        i = int(np.argmax(np.abs(vecs[:, j])))
        if vecs[i, j] < 0:
            vecs[:, j] = -vecs[:, j]
    return vecs


def rescale(theta, psi, m):
    """lambda = theta dV, phi = psi / sqrt(dV) (Riemann sums of Eq. 3.1)."""
    dv = cell_volume(m)
    return theta * dv, psi / np.sqrt(dv)


def eig_full(G, m, domain, k):
    """Leading k eigenpairs of the matrixised Gamma_hat by a dense symmetric solver."""
    S = matrixize(G, domain)
    theta, psi = np.linalg.eigh(S)
    order = np.argsort(theta)[::-1][:k]
    lam, phi = rescale(theta[order], fix_signs(psi[:, order]), m)
    fve = np.cumsum(lam) / (np.trace(S) * cell_volume(m))
    return lam, phi, fve


def orth(Y):
    """Orthonormal basis of range(Y) (Householder QR)."""
    Q, _ = np.linalg.qr(Y)
    return Q


def rproj_eig(G, m, domain, omega, k, power_iters):
    """Random-projection eigenpairs (range finder + Rayleigh-Ritz), FP64."""
    S = matrixize(G, domain)
    Y = S @ omega
    for _ in range(power_iters):
        Q = orth(Y)
        Y = S @ Q
    Q = orth(Y)
    B = Q.T @ S @ Q
    B = 0.5 * (B + B.T)
    theta, U = np.linalg.eigh(B)
    order = np.argsort(theta)[::-1][:k]
    psi = Q @ U[:, order]
    lam, phi = rescale(theta[order], fix_signs(psi), m)
    fve = np.cumsum(lam) / (np.trace(S) * cell_volume(m))
    return lam, phi, fve


def subspace_angle(A, B):
    """Largest principal angle (radians) between the column spans of A and B."""
    Qa = orth(A)
    Qb = orth(B)
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(np.clip(np.min(s), -1.0, 1.0)))
