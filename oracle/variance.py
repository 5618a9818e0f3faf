"""Oracle: the noise variance of Eq. (2.5)-(2.6), FP64.

Test infrastructure only: the library never imports this module.

Definitions followed
--------------------
* Eq. (2.5): b0(t) is the local linear fit at t of the squared observations
  Y_ij^2 with the weights 1/N_i of the mean smoother (Eq. 2.3) and bandwidth
  h_sigma; binned, it is the mean smoother applied to the bins
  (cnt, W = sum 1/N_i, V2 = sum Y^2/N_i).  b0(t) estimates E[Y(t)^2] =
  Gamma(t, t) + sigma^2 + mu(t)^2.
* sigma2_hat(t) = b0(t) - Gamma_hat(t, t) - mu_hat(t)^2.
* Eq. (2.6): sigma2_hat = integral over Omega of sigma2_hat(t), taken here as
  the mean over the grid nodes of Omega (the Riemann sum divided by |Omega|).

Readings where the paper is silent or at odds with itself
--------------------------------------------------------
* Sign of mu_hat^2: the paper prints + mu_hat mu_hat; since E[Y^2] = Gamma +
  sigma^2 + mu^2, the mean term is subtracted.
* Eq. (2.6) integrates over Omega without dividing by |Omega|; for a constant
  sigma^2 that is only right when |Omega| = 1, so the integral is divided by
  |Omega| (the number of domain nodes times the cell volume).
* Nodes where b0 is EMPTY (no observation in the window) are left out of the
  average; they are NaN in sigma2_hat(t).
"""
from __future__ import annotations

import math

import numpy as np

from .smoother import STATUS_EMPTY, smooth_mean


def sigma2_curve(m, h, cnt, W, V2, mu, gamma_diag):
    """sigma2_hat(t) at every node and the status of the b0 fit."""
    b0, st = smooth_mean(m, h, cnt, W, V2)
    mu = np.asarray(mu, dtype=np.float64)
    out = b0 - np.asarray(gamma_diag, dtype=np.float64) - mu * mu
    out = np.where(st == STATUS_EMPTY, math.nan, out)
    return out, st


def sigma2_scalar(sig_t, domain):
    """Eq. (2.6): the mean of sigma2_hat(t) over the domain nodes with a value."""
    dm = np.asarray(domain).astype(bool) & np.isfinite(sig_t)
    if not dm.any():
        return math.nan
    return float(np.mean(np.asarray(sig_t)[dm]))
