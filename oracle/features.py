"""Oracle: the 32-number dataset summary fed to the bandwidth network (FP64).

Test infrastructure only.  The summary describes what drives the optimal
bandwidth of the smoothers of Eq. (2.3)-(2.4): sample size and sampling
density (n, N_i, bin occupancy), noise level against signal level, and the
roughness of the binned mean and covariance.

  0  d                               16  log 1st-difference roughness of mb, axis 1
  1  log n                             17  zero
  2  log mean N_i                      18  log roughness of g along s_1 (vs var g)
  3  std N_i / mean N_i                19  log roughness of g along the (s_1, t_1) diagonal
  4  log min N_i                       20  log (1 + mean pair count per covariance bin)
  5  log max N_i                       21  fraction of covariance bins with a pair
  6  log (1 + mean count per bin)      22-24 log bin width 1/M_k (0 beyond d)
  7  var(count) / mean(count)^2        25-31 zero
  8  skewness of count
  9  fraction of empty bins
 10  log mean within-bin variance sb = V2/W - (V/W)^2 over non-empty bins
 11  log variance of the binned mean mb = V/W over non-empty bins
 12-14 log 2nd-difference roughness of mb per axis (mean squared 2nd difference
       over consecutive non-empty triples, minus feature 11); 0 beyond d
 15  log 1st-difference roughness of mb along axis 0 (as 12, 1st differences)

Covariance raw means g = V/W on bins with W > 0 (the diagonal of gridded data
is excluded by the binning).  Roughness along a direction is the mean squared
difference of g over neighbour pairs that are both non-empty, divided by the
variance of g, logged.  The small constant 1e-12 keeps every log finite.
"""
from __future__ import annotations

import math

import numpy as np

NFEAT = 32
EPS = 1e-12


def _grid_view(a, m):
    return np.asarray(a, dtype=np.float64).reshape(tuple(m))


def _roughness(vals, ok, axis, order):
    """Mean squared finite difference of given order along axis over all-ok windows."""
    n = vals.shape[axis]
    if n <= order:
        return None
    sl = lambda k: tuple(slice(k, n - order + k) if ax == axis else slice(None)  # noqa: E731
                         for ax in range(vals.ndim))
    if order == 1:
        diff = vals[sl(1)] - vals[sl(0)]
        good = ok[sl(1)] & ok[sl(0)]
    else:
        diff = vals[sl(2)] - 2.0 * vals[sl(1)] + vals[sl(0)]
        good = ok[sl(2)] & ok[sl(1)] & ok[sl(0)]
    if not good.any():
        return None
    return float(np.mean(diff[good] ** 2))


def features(d, m, Ni, cnt, W, V, V2, C, Wc, Vc):
    """The 32-feature summary of one dataset.

    Ni: per-subject observation counts (n); cnt, W, V, V2: mean bins (P);
    C, Wc, Vc: pooled covariance bins (P x P).
    """
    f = np.zeros(NFEAT)
    Ni = np.asarray(Ni, dtype=np.float64)
    f[0] = d
    f[1] = math.log(len(Ni))
    f[2] = math.log(max(Ni.mean(), EPS))
    f[3] = Ni.std() / max(Ni.mean(), EPS)
    f[4] = math.log(max(Ni.min(), 1.0))
    f[5] = math.log(max(Ni.max(), 1.0))
    c = np.asarray(cnt, dtype=np.float64)
    mc = c.mean()
    f[6] = math.log1p(mc)
    f[7] = c.var() / mc ** 2 if mc > 0 else 0.0
    sd = c.std()
    f[8] = float(np.mean((c - mc) ** 3)) / sd ** 3 if sd > 0 else 0.0
    f[9] = float(np.mean(c == 0))
    W = np.asarray(W, dtype=np.float64)
    ne = W > 0
    mb = np.where(ne, np.asarray(V) / np.where(ne, W, 1.0), 0.0)
    sb = np.where(ne, np.asarray(V2) / np.where(ne, W, 1.0) - mb ** 2, 0.0)
    f[10] = math.log(max(float(np.mean(np.maximum(sb[ne], 0.0))), 0.0) + EPS) if ne.any() else 0.0
    varmb = float(np.var(mb[ne])) if ne.any() else 0.0
    f[11] = math.log(varmb + EPS)
    mbg, neg = _grid_view(mb, m), _grid_view(ne, m).astype(bool)
    for k in range(3):
        if k < d:
            r2 = _roughness(mbg, neg, k, 2)
            f[12 + k] = math.log((r2 if r2 is not None else 0.0) + EPS) - f[11]
    for k in range(2):
        if k < d:
            r1 = _roughness(mbg, neg, k, 1)
            f[15 + k] = math.log((r1 if r1 is not None else 0.0) + EPS) - f[11]
    Wc = np.asarray(Wc, dtype=np.float64)
    okc = Wc > 0
    g = np.where(okc, np.asarray(Vc, dtype=np.float64) / np.where(okc, Wc, 1.0), 0.0)
    varg = float(np.var(g[okc])) if okc.any() else 0.0
    lvg = math.log(varg + EPS)
    P = g.shape[0]
    s0 = int(np.prod(m[1:]))  # flat step of axis 0
    if P > s0:
        a, b = g[s0:, :], g[:-s0, :]
        good = okc[s0:, :] & okc[:-s0, :]
        r = float(np.mean((a - b)[good] ** 2)) if good.any() else 0.0
        f[18] = math.log(r + EPS) - lvg
        a, b = g[s0:, s0:], g[:-s0, :-s0]
        good = okc[s0:, s0:] & okc[:-s0, :-s0]
        r = float(np.mean((a - b)[good] ** 2)) if good.any() else 0.0
        f[19] = math.log(r + EPS) - lvg
    Cc = np.asarray(C, dtype=np.float64)
    f[20] = math.log1p(float(Cc.mean()))
    f[21] = float(np.mean(Cc > 0))
    for k in range(3):
        if k < d:
            f[22 + k] = math.log(1.0 / m[k])
    return f
