"""Oracle: the covariance smoother of Eq. (2.4) on the whole grid, stacked, FP64.

Test infrastructure only: the library never imports this module.

smoother.smooth_cov_grid evaluates Eq. (2.4) (binned, Section 3.2) at every
output pair with a Python loop over points, which limits it to grids of a
few hundred nodes.  This module computes the same quantities for grids of up
to 64 x 64 nodes (16.8M output pairs):

* every kernel moment S[alpha] (|alpha| <= 2) and T[alpha] (|alpha| <= 1) of
  smoother.cov_moments_grid, each as its own 2d successive 1-D sums (the
  product kernel); a 1-D sum along one axis is the product with the M x M
  band matrix B[x, j] = K((j - x)/(h M)) ((j - x)/(h M))^power (the weights of
  smoother.tap_weights), applied with a matrix product instead of a loop over
  the offsets;
* the number of non-empty bin pairs in each window (smoother.nonempty_grid) as
  the same products with the 0/1 band of the window;
* the normal equations at each output pair assembled from those moments as in
  smoother.normal_matrix, and the solve and status rules of
  smoother.solve_point applied over a stack of points (block.solve_points).

Nothing is shared between moments and no sum is reordered beyond the matrix
product's own order of a 1-D sum.
"""
from __future__ import annotations

import numpy as np

from .block import solve_points
from .smoother import grid_size, moment_indices, tap_weights


def band_matrix(mk, hk, power, box=False):
    """B[x, j]: weight of bin j in the 1-D sum at output x (zero outside |u| < 1)."""
    ks, wts = tap_weights(mk, hk, power)
    if box:
        wts = np.ones_like(wts)
    B = np.zeros((mk, mk))
    for k, wk in zip(ks, wts):
        x = np.arange(max(0, -k), min(mk, mk - k))
        B[x, x + k] = wk
    return B


def conv_axis_mm(arr, axis, mk, hk, power, box=False):
    """out[.., x, ..] = sum_j B[x, j] arr[.., j, ..] along ``axis`` (same as
    smoother.conv_axis, with the sum over offsets done as a matrix product)."""
    B = band_matrix(mk, hk, power, box)
    a = np.moveaxis(arr, axis, -1)
    out = a @ B.T
    return np.ascontiguousarray(np.moveaxis(out, -1, axis))


def moments(m, h, W, V):
    """S[alpha], T[alpha] of smoother.cov_moments_grid (P x P each)."""
    d = len(m)
    shape = tuple(m) + tuple(m)
    Wg = np.asarray(W, float).reshape(shape)
    Vg = np.asarray(V, float).reshape(shape)
    axes_m = list(m) + list(m)
    axes_h = list(h) + list(h)
    P = grid_size(m)
    S, T = {}, {}
    for alpha in moment_indices(2 * d, 2):
        a = Wg
        for ax in range(2 * d):
            a = conv_axis_mm(a, ax, axes_m[ax], axes_h[ax], alpha[ax])
        S[alpha] = a.reshape(P, P)
    for alpha in moment_indices(2 * d, 1):
        a = Vg
        for ax in range(2 * d):
            a = conv_axis_mm(a, ax, axes_m[ax], axes_h[ax], alpha[ax])
        T[alpha] = a.reshape(P, P)
    return S, T


def nonempty(m, h, C):
    """Non-empty bin pairs in each output pair's window (smoother.nonempty_grid)."""
    d = len(m)
    shape = tuple(m) + tuple(m)
    a = (np.asarray(C).reshape(shape) > 0).astype(np.float64)
    axes_m = list(m) + list(m)
    axes_h = list(h) + list(h)
    for ax in range(2 * d):
        a = conv_axis_mm(a, ax, axes_m[ax], axes_h[ax], 0, box=True)
    P = grid_size(m)
    return np.rint(a).astype(np.int64).reshape(P, P)


def fit_pairs(S, T, ne, d, p, q, mu=None, chunk=1 << 20):
    """Gamma_hat and status at the output pairs (p[k], q[k]) from the moments S, T
    and window counts ne of a grid (smoother.normal_matrix + solve_point rules)."""
    D = 2 * d + 1
    unit = []
    for j in range(D):
        e = [0] * (2 * d)
        if j > 0:
            e[j - 1] = 1
        unit.append(tuple(e))
    p = np.asarray(p)
    q = np.asarray(q)
    val = np.empty(p.size)
    st = np.empty(p.size, dtype=np.uint8)
    for lo in range(0, p.size, chunk):
        pp = p[lo:lo + chunk]
        qq = q[lo:lo + chunk]
        A = np.empty((pp.size, D, D))
        r = np.empty((pp.size, D))
        for i in range(D):
            r[:, i] = T[unit[i]][pp, qq]
            for j in range(D):
                alpha = tuple(a + b for a, b in zip(unit[i], unit[j]))
                A[:, i, j] = S[alpha][pp, qq]
        v, s = solve_points(A, r, ne[pp, qq])
        if mu is not None:
            keep = s != 2
            v[keep] -= mu[pp[keep]] * mu[qq[keep]]
        val[lo:lo + chunk] = v
        st[lo:lo + chunk] = s
    return val, st


def smooth_cov(m, h, C, W, V, mu=None, rows=None, chunk=1 << 20):
    """Gamma_hat and status (smoother.smooth_cov_grid) at every output pair, or at
    the output rows ``rows`` only (all t for each s in rows)."""
    P = grid_size(m)
    S, T = moments(m, h, W, V)
    ne = nonempty(m, h, C)
    rows = np.arange(P) if rows is None else np.asarray(rows)
    p = np.repeat(rows, P)
    q = np.tile(np.arange(P), rows.size)
    val, st = fit_pairs(S, T, ne, len(m), p, q, mu, chunk)
    return val.reshape(rows.size, P), st.reshape(rows.size, P)


def bin_cov_sparse_pairs(offs, t, r, m, fold=None, nfold=0):
    """smoother.bin_cov_sparse with the ordered pairs j != l of every subject listed
    as index arrays and summed per bin by np.bincount (same sums, any order).

    Returns C (int64), W, V, Q of shape (F, P, P), F = max(nfold, 1)."""
    from .smoother import bin_of
    P = grid_size(m)
    F = max(nfold, 1)
    offs = np.asarray(offs, dtype=np.int64)
    Ni = np.diff(offs)
    b = bin_of(t, m)
    r = np.asarray(r, dtype=np.float64)
    subj = np.repeat(np.arange(Ni.size), Ni)
    # for every observation j, the observations l of its subject
    js, ls = [], []
    for N in np.unique(Ni):
        if N < 2:
            continue
        sel = np.nonzero(Ni == N)[0]
        jj, ll = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        keep = jj != ll
        jj, ll = jj[keep], ll[keep]
        base = offs[sel][:, None]
        js.append((base + jj[None, :]).ravel())
        ls.append((base + ll[None, :]).ravel())
    if not js:
        z = np.zeros((F, P, P))
        return z.astype(np.int64), z, z.copy(), z.copy()
    j = np.concatenate(js)
    l = np.concatenate(ls)
    N = Ni[subj[j]].astype(np.float64)
    w = 1.0 / (N * (N - 1.0))
    f = np.asarray(fold)[subj[j]] if nfold > 0 else np.zeros(j.size, dtype=np.int64)
    idx = (f.astype(np.int64) * P + b[j]) * P + b[l]
    prod = r[j] * r[l]
    n = F * P * P
    C = np.bincount(idx, minlength=n).astype(np.int64).reshape(F, P, P)
    W = np.bincount(idx, weights=w, minlength=n).reshape(F, P, P)
    V = np.bincount(idx, weights=w * prod, minlength=n).reshape(F, P, P)
    Q = np.bincount(idx, weights=w * prod * prod, minlength=n).reshape(F, P, P)
    return C, W, V, Q
