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


def cv_score(m, h, C, W, V, Q, smooth=None):
    """CV(h) from per-fold bins C, W, V, Q of shape (F, P, P).

    ``smooth(m, h, C, W, V) -> (G, status)`` fits the surface on the training
    bins: smoother.smooth_cov_grid by default, or any function computing the
    same estimator (grid.smooth_cov for larger grids)."""
    smooth = sm.smooth_cov_grid if smooth is None else smooth
    F = C.shape[0]
    Ct, Wt, Vt = C.sum(axis=0), W.sum(axis=0), V.sum(axis=0)
    err = 0.0
    w_in = 0.0
    w_out = 0.0
    for f in range(F):
        G, st = smooth(m, h, Ct - C[f], Wt - W[f], Vt - V[f])
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


# ----------------------------------------------------------------------------
# cross-validation of the mean smoother (Eq. 2.3)
# ----------------------------------------------------------------------------
# The same subject-level K-fold reading: for fold f the mean is fitted on the
# mean bins of the other folds and scored on fold f's observations at their bin
# centres with the weights 1/N_i of Eq. (2.3).  Because the fit is evaluated at
# bin centres, the held-out error of a bin follows from three sums of the
# fold's observations in it,
#   sum_{obs in bin} (1/N_i) (Y_ij - mu)^2 = V2_f - 2 mu V_f + mu^2 W_f,
# with W_f = sum 1/N_i, V_f = sum Y/N_i, V2_f = sum Y^2/N_i.  Bins whose fit is
# EMPTY are left out (+inf when they hold more than 1% of the held-out weight);
# the score is normalised by the held-out weight that was scored.

def mean_fold_bins(offs, t, y, m, fold, nfold):
    """Per-fold mean bins (cnt, W, V, V2), each (F, P), of scattered data."""
    offs = np.asarray(offs, dtype=np.int64)
    fold = np.asarray(fold)
    P = sm.grid_size(m)
    out = [np.zeros((nfold, P), dtype=np.int64)] + [np.zeros((nfold, P)) for _ in range(3)]
    for f in range(nfold):
        subj = np.nonzero(fold == f)[0]
        if subj.size == 0:
            continue
        idx = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in subj])
        sub_offs = np.concatenate([[0], np.cumsum(offs[subj + 1] - offs[subj])])
        c, W, V, V2 = sm.bin_mean_sparse(sub_offs, np.asarray(t)[idx], np.asarray(y)[idx], m)
        for a, b in zip(out, (c, W, V, V2)):
            a[f] = b
    return tuple(out)


def mean_cv_score(m, h, cnt, W, V, V2):
    """CV(h) of the mean smoother from per-fold mean bins of shape (F, P)."""
    F = cnt.shape[0]
    ct, wt, vt = cnt.sum(axis=0), W.sum(axis=0), V.sum(axis=0)
    err = w_in = w_out = 0.0
    for f in range(F):
        mu, st = sm.smooth_mean(m, h, ct - cnt[f], wt - W[f], vt - V[f])
        inc = st != sm.STATUS_EMPTY
        g = np.where(inc, mu, 0.0)
        e = V2[f] - 2.0 * g * V[f] + g * g * W[f]
        err += float(np.sum(e[inc]))
        w_in += float(np.sum(W[f][inc]))
        w_out += float(np.sum(W[f][~inc]))
    if w_out > 0.01 * (w_in + w_out) or w_in <= 0.0:
        return math.inf
    return err / w_in


def mean_cv_bruteforce(offs, t, y, m, h, fold, nfold):
    """The same score summed observation by observation: for each held-out
    observation, (1/N_i) (Y_ij - mu_hat^(-f)(centre of its bin))^2."""
    offs = np.asarray(offs, dtype=np.int64)
    cnt, W, V, V2 = mean_fold_bins(offs, t, y, m, fold, nfold)
    ct, wt, vt = cnt.sum(axis=0), W.sum(axis=0), V.sum(axis=0)
    b = sm.bin_of(t, m)
    err = w_in = w_out = 0.0
    for f in range(nfold):
        mu, st = sm.smooth_mean(m, h, ct - cnt[f], wt - W[f], vt - V[f])
        for i in np.nonzero(np.asarray(fold) == f)[0]:
            lo, hi = int(offs[i]), int(offs[i + 1])
            if hi == lo:
                continue
            wi = 1.0 / (hi - lo)
            for j in range(lo, hi):
                if st[b[j]] == sm.STATUS_EMPTY:
                    w_out += wi
                else:
                    err += wi * (float(y[j]) - mu[b[j]]) ** 2
                    w_in += wi
    if w_out > 0.01 * (w_in + w_out) or w_in <= 0.0:
        return math.inf
    return err / w_in
