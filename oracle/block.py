"""Oracle: the covariance smoother of Eq. (2.4) on blocks of output pairs, FP64.

Test infrastructure only: the library never imports this module.

The binned estimator of smoother.py needs the P x P covariance bins, which a
32 x 32 x 32 grid (P^2 = 1.07e9 pairs) does not allow.  This module evaluates
the same estimator at chosen output pairs only: a set S of s-nodes against a
box T of t-nodes (a row when S is one node and T the whole grid, a tile when
both are small boxes).

Definitions (gridded data, Section 3.2 binning, Eq. 2.4 weights)
----------------------------------------------------------------
For output nodes x and bins p, the kernel matrix of exponent alpha is

    K_alpha[x, p] = prod_k K(u_k) u_k^alpha_k,   u_k = (p_k - x_k) / (h_k M_k),

(K the Epanechnikov kernel, u = (c_p - x)/h in bin units, as smoother._window).
The normal equations of Eq. (2.4) at the output pair (s, t) sum over bin pairs
(p, q) with the design z = [1, u_s, u_t]; written with kernel matrices,

    A_ij(s, t) = sum_{p, q} K_alpha(i,j)[s, p] W[p, q] K_beta(i,j)[t, q]
    r_i(s, t)  = sum_{p, q} K_alpha(i)[s, p]   V[p, q] K_beta(i)[t, q]

where alpha and beta are the s- and t-exponents of z_i z_j (or z_i), and
C, W, V are the covariance bins of smoother.bin_cov_dense:

    W[p, q] = sum_i w_i M_ip M_iq,  V[p, q] = sum_i w_i R_ip R_iq  (p != q; 0 on p == q)

with w_i = 1/(N_i (N_i - 1)).  The sum over p is taken first, as the matrix
products (K_alpha (w M)^T) M and (K_alpha (w R)^T) R minus the p == q terms
(the zeroed diagonal); the sum over q then runs as 1-D sums along each t axis
(smoother.conv_axis) over a box that holds every window of T.  The solve and
the status rules are those of smoother.solve_point, applied point by point
through solve_points (the same rules over a stack of systems).
"""
from __future__ import annotations

import numpy as np

from .smoother import (PIVOT_RTOL, STATUS_EMPTY, STATUS_FALLBACK, STATUS_OK, conv_axis,
                       epanechnikov, grid_size, moment_indices, pair_weights)


def solve_points(A, r, nonempty):
    """solve_point over a stack: A (N, D, D), r (N, D), nonempty (N,).

    Same rules: EMPTY when A_00 <= 0 (NaN); FALLBACK (r_0/A_00) when nonempty < D,
    when a Cholesky pivot (natural order) is not positive, or when a pivot is at
    most PIVOT_RTOL times its diagonal entry; otherwise OK with beta_0 of the solve.
    """
    A = np.asarray(A, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    N, D, _ = A.shape
    val = np.full(N, np.nan)
    st = np.full(N, STATUS_EMPTY, dtype=np.uint8)
    a00 = A[:, 0, 0]
    live = a00 > 0.0
    val[live] = r[live, 0] / a00[live]
    st[live] = STATUS_FALLBACK
    cand = live & (np.asarray(nonempty) >= D)
    # Cholesky A = L L^T column by column, tracking the pivots
    L = np.zeros_like(A)
    good = cand.copy()
    for j in range(D):
        piv = A[:, j, j] - np.sum(L[:, j, :j] ** 2, axis=1)
        ok = good & (piv > 0.0) & (piv > PIVOT_RTOL * A[:, j, j])
        good = ok
        ljj = np.sqrt(np.where(ok, piv, 1.0))
        L[:, j, j] = ljj
        for i in range(j + 1, D):
            L[:, i, j] = (A[:, i, j] - np.sum(L[:, i, :j] * L[:, j, :j], axis=1)) / ljj
    if good.any():
        beta = np.linalg.solve(A[good], r[good][:, :, None])[:, :, 0]
        val[good] = beta[:, 0]
        st[good] = STATUS_OK
    return val, st


def _coords(flat, m):
    """(len, d) per-axis integer coordinates of flat C-order node indices."""
    flat = np.asarray(flat, dtype=np.int64)
    out = np.empty((flat.size, len(m)), dtype=np.int64)
    rem = flat.copy()
    for k in range(len(m) - 1, -1, -1):
        out[:, k] = rem % m[k]
        rem //= m[k]
    return out


def taps(mk, hk):
    """Largest integer offset k with |k|/(h M) < 1 on an axis of M bins."""
    k = 0
    while (k + 1) / (hk * mk) < 1.0:
        k += 1
    return k


def window_union(nodes, m, h):
    """Sorted flat indices of every bin inside the kernel window of some node."""
    cs = _coords(nodes, m)
    tk = [taps(mk, hk) for mk, hk in zip(m, h)]
    keep = np.zeros(tuple(m), dtype=bool)
    for c in cs:
        keep[tuple(slice(max(0, c[k] - tk[k]), min(m[k], c[k] + tk[k] + 1))
                   for k in range(len(m)))] = True
    return np.nonzero(keep.ravel())[0]


def kernel_matrix(nodes, bins, m, h, alpha):
    """K_alpha[x, p] for output nodes x and bins p (flat indices)."""
    cx = _coords(nodes, m).astype(np.float64)
    cp = _coords(bins, m).astype(np.float64)
    K = np.ones((cx.shape[0], cp.shape[0]))
    for k in range(len(m)):
        u = (cp[None, :, k] - cx[:, None, k]) / (h[k] * m[k])
        K *= epanechnikov(u) * u ** alpha[k]
    return K


def _box(lo, hi, m, h):
    """Box of the t-nodes [lo, hi) expanded by the kernel half-width, clipped."""
    blo, bhi = [], []
    for k in range(len(m)):
        tk = taps(m[k], h[k])
        blo.append(max(0, lo[k] - tk))
        bhi.append(min(m[k], hi[k] + tk))
    return blo, bhi


def _box_nodes(lo, hi, m):
    axes = [np.arange(a, b) for a, b in zip(lo, hi)]
    g = np.meshgrid(*axes, indexing="ij")
    flat = np.zeros(g[0].size, dtype=np.int64)
    for k in range(len(m)):
        flat = flat * m[k] + g[k].ravel()
    return flat


def smooth_cov_block(y, mask, mu, m, h, S, t_lo, t_hi):
    """Gamma_hat (residual mode) and status at the pairs S x box[t_lo, t_hi).

    y, mask: n x P gridded data (mask None = fully observed); mu: the mean fit at
    the nodes; S: flat s-node indices; t_lo/t_hi: per-axis node range of T.
    Returns (|S|, |T|) arrays in C order of the T box.
    """
    m = tuple(int(v) for v in m)
    h = np.asarray(h, dtype=np.float64)
    d = len(m)
    D = 2 * d + 1
    y = np.asarray(y, dtype=np.float64)
    mk = np.ones(y.shape, dtype=bool) if mask is None else np.asarray(mask).astype(bool)
    mf = mk.astype(np.float64)
    wi = pair_weights(mk.sum(axis=1))
    R = np.where(mk, y - np.asarray(mu, dtype=np.float64)[None, :], 0.0)
    S = np.asarray(S, dtype=np.int64)
    A_nodes = window_union(S, m, h)
    blo, bhi = _box(t_lo, t_hi, m, h)
    B_nodes = _box_nodes(blo, bhi, m)
    bshape = tuple(b - a for a, b in zip(blo, bhi))
    # position of every A bin inside the box (or -1) for the zeroed diagonal
    pos_in_box = -np.ones(len(A_nodes), dtype=np.int64)
    lookup = {int(q): j for j, q in enumerate(B_nodes)}
    for a, p in enumerate(A_nodes):
        pos_in_box[a] = lookup.get(int(p), -1)
    shared = pos_in_box >= 0
    diagC = mf[:, A_nodes].sum(axis=0)                       # C[p, p] before zeroing
    diagW = (mf[:, A_nodes] * wi[:, None]).sum(axis=0)
    diagV = ((R[:, A_nodes] ** 2) * wi[:, None]).sum(axis=0)

    full_box = len(B_nodes) == grid_size(m)

    def columns(X, nodes, whole=False):
        return X if whole else X[:, nodes]

    def s_side(alpha, leftA, rightB, diag):
        """sum_p K_alpha[s, p] X[p, q] over p in A, p != q, for q in the box."""
        K = kernel_matrix(S, A_nodes, m, h, alpha)
        out = (K @ leftA.T) @ rightB
        out[:, pos_in_box[shared]] -= K[:, shared] * diag[shared][None, :]
        return out

    def t_side(X, beta):
        """sum_q K_beta[t, q] X[s, q] for t in T, via 1-D sums along each t axis."""
        a = X.reshape((X.shape[0],) + bshape)
        for k in range(d):
            # conv_axis takes u = (q - t)/(h M) with the grid's own M on that axis
            a = conv_axis(a, k + 1, m[k], h[k], beta[k])
        sl = tuple([slice(None)] + [slice(t_lo[k] - blo[k], t_hi[k] - blo[k]) for k in range(d)])
        return a[sl].reshape(X.shape[0], -1)

    unit = []
    for j in range(D):
        e = [0] * (2 * d)
        if j > 0:
            e[j - 1] = 1
        unit.append(e)
    need_S = {}
    for i in range(D):
        for j in range(D):
            e = [a + b for a, b in zip(unit[i], unit[j])]
            need_S[(i, j)] = (tuple(e[:d]), tuple(e[d:]))
    mfA, RA = mf[:, A_nodes], R[:, A_nodes]
    wmA, wRA = mfA * wi[:, None], RA * wi[:, None]
    mfB, RB = columns(mf, B_nodes, full_box), columns(R, B_nodes, full_box)
    Ws = {al: s_side(al, wmA, mfB, diagW) for al in moment_indices(d, 2)}
    Vs = {al: s_side(al, wRA, RB, diagV) for al in moment_indices(d, 1)}
    nT = int(np.prod([b - a for a, b in zip(t_lo, t_hi)]))
    nS = len(S)
    Amat = np.empty((nS, nT, D, D))
    rvec = np.empty((nS, nT, D))
    cache = {}
    for (i, j), (al, be) in need_S.items():
        key = ("S", al, be)
        if key not in cache:
            cache[key] = t_side(Ws[al], be)
        Amat[:, :, i, j] = cache[key]
    for i in range(D):
        al, be = tuple(unit[i][:d]), tuple(unit[i][d:])
        rvec[:, :, i] = t_side(Vs[al], be)
    # non-empty bin pairs: sum over the window of 1[C > 0]
    Cblk = mfA.T @ mfB
    Cblk[np.nonzero(shared)[0], pos_in_box[shared]] -= diagC[shared]
    Cpos = (np.rint(Cblk) > 0).astype(np.float64)
    Ks0 = (kernel_matrix(S, A_nodes, m, h, (0,) * d) > 0).astype(np.float64)
    N1 = Ks0 @ Cpos
    a = N1.reshape((nS,) + bshape)
    for k in range(d):
        tk = taps(m[k], h[k])
        out = np.zeros_like(a)
        n = a.shape[k + 1]
        for off in range(-tk, tk + 1):
            lo, hi = max(0, -off), min(n, n - off)
            if lo >= hi:
                continue
            dst = [slice(None)] * a.ndim
            src = [slice(None)] * a.ndim
            dst[k + 1] = slice(lo, hi)
            src[k + 1] = slice(lo + off, hi + off)
            out[tuple(dst)] += a[tuple(src)]
        a = out
    sl = tuple([slice(None)] + [slice(t_lo[k] - blo[k], t_hi[k] - blo[k]) for k in range(d)])
    nonempty = np.rint(a[sl]).reshape(nS, nT).astype(np.int64)
    val, st = solve_points(Amat.reshape(-1, D, D), rvec.reshape(-1, D), nonempty.ravel())
    return val.reshape(nS, nT), st.reshape(nS, nT)


def smooth_cov_rows(y, mask, mu, m, h, rows):
    """Gamma_hat[rows, :] over the whole grid (residual mode) and status."""
    return smooth_cov_block(y, mask, mu, m, h, rows, [0] * len(m), list(m))
