"""Oracle: cross-validated bandwidth score of the covariance smoother, FP64.

Test infrastructure only: the library never imports this module.

Section 3.3 selects bandwidths by cross-validation of the fitted smoother.
The reading used here is K-fold, subject-level: subjects are split into folds;
for fold f the covariance surface is fitted on the bins of all other folds,
Gamma^(-f), and scored on the held-out raw products of fold f at their bin
centres.  Because the fitted surface is evaluated at bin centres, the
held-out error per bin follows from three sums of the fold's pairs,
  sum_{pairs in bin} w_i (R_ij R_il - G)^2 = Q_f - 2 G V_f + G^2 W_f,
with W_f = sum w_i, V_f = sum w_i R R and Q_f = sum w_i (R R)^2.

Readings
* Bins whose fit is EMPTY are left out of the score; if they hold more than
  1% of the held-out weight the bandwidth scores +inf.
* The score is normalised by the held-out weight that was scored.
* Residuals use the mean fitted on all subjects.
"""
from __future__ import annotations

import math

import numpy as np

from . import smoother as sm


def cv_score(m, h, C, W, V, Q):
    """CV(h) from per-fold bins C, W, V, Q of shape (F, P, P)."""
    F = C.shape[0]
    Ct, Wt, Vt = C.sum(axis=0), W.sum(axis=0), V.sum(axis=0)
    err = 0.0
    w_in = 0.0
    w_out = 0.0
    for f in range(F):
        G, st = sm.smooth_cov_grid(m, h, Ct - C[f], Wt - W[f], Vt - V[f])
        inc = st != sm.STATUS_EMPTY
        g = np.where(inc, G, 0.0)
        e = Q[f] - 2.0 * g * V[f] + g * g * W[f]
        err += float(np.sum(e[inc]))
        w_in += float(np.sum(W[f][inc]))
        w_out += float(np.sum(W[f][~inc]))
    if w_out > 0.01 * (w_in + w_out) or w_in <= 0.0:
        return math.inf
    return err / w_in


def cv_grid(m, hs, C, W, V, Q):
    """CV score for each isotropic bandwidth in ``hs``; returns (scores, argmin)."""
    d = len(m)
    scores = np.array([cv_score(m, [h] * d, C, W, V, Q) for h in hs])
    return scores, int(np.argmin(scores))
