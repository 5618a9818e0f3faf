"""Oracle: binning and the local linear smoothers of Section 2.1, in FP64.

Test infrastructure only (see the package docstring): the library never
imports this module.

Definitions followed
--------------------
* Mean smoother, Eq. (2.3): beta = argmin sum_i (1/N_i) sum_j K_h(t - t_ij)
  [Y_ij - b0 - sum_k b_k (t_k - t_ij,k)]^2, mu_hat(t) = b0.
* Covariance smoother, Eq. (2.4): the same in 2d dimensions over ordered pairs
  j != l of one subject, weights 1/(N_i(N_i-1)), responses Y_ij Y_il (raw
  mode, Gamma_hat = b0 - mu_hat(s) mu_hat(t)) or residual products
  R_ij R_il with R = Y - mu_hat (residual mode, Gamma_hat = b0).
* Product kernel K_h(u) = prod_k K(u_k / h_k) / h_k with the Epanechnikov
  K(u) = 3/4 (1 - u^2) on |u| < 1 (Section 2.1 and assumption A.2).
* Binning, Section 3.2: observations are moved to the centre of the bin of a
  regular grid that contains them; the local linear fit then runs over the
  bins, each bin carrying its summed weight W_b and summed weighted response
  V_b.  Bins are [k/M, (k+1)/M) per axis (the last one closed), centres
  (k + 1/2)/M.

Readings where the paper is silent
----------------------------------
* Simple (nearest-bin) binning, the last bin closed at t = 1.
* Slope variables are u = (c_b - x)/h; the paper writes (x - c_b) unscaled.
  The intercept b0 is the same for both.
* Status per output point: EMPTY when no weight falls in the window (value
  NaN); FALLBACK when fewer than D = (number of unknowns) non-empty bins fall
  in the window, or when a Cholesky pivot of the normal matrix in natural
  variable order falls to PIVOT_RTOL times its diagonal entry or below (value
  T0/S0, the local constant fit); OK otherwise.
* Diagonal exclusion j != l is at observation level: for gridded data the bin
  pair p == q holds only j == l pairs and is zeroed; for scattered data pairs
  of distinct observations that share a bin are kept.
"""
from __future__ import annotations

import math

import numpy as np

STATUS_OK = 0
STATUS_FALLBACK = 1
STATUS_EMPTY = 2

PIVOT_RTOL = 1e-9


# ----------------------------------------------------------------------------
# grid helpers
# ----------------------------------------------------------------------------

def grid_size(m):
    return int(np.prod(m))


def centres(m):
    """Bin centres (k + 1/2)/M_k, flattened in C order: (P, d)."""
    axes = [(np.arange(mk) + 0.5) / mk for mk in m]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in mesh], axis=1)


def bin_of(t, m):
    """Flat C-order bin index of each location in ``t`` (N x d): simple binning."""
    t = np.atleast_2d(np.asarray(t, dtype=np.float64))
    flat = np.zeros(t.shape[0], dtype=np.int64)
    for k, mk in enumerate(m):
        idx = np.floor(t[:, k] * mk).astype(np.int64)
        idx = np.clip(idx, 0, mk - 1)
        flat = flat * mk + idx
    return flat


def epanechnikov(u):
    """K(u) = 3/4 (1 - u^2) for |u| < 1, else 0 (zero on the boundary |u| = 1)."""
    u = np.asarray(u, dtype=np.float64)
    return np.where(np.abs(u) < 1.0, 0.75 * (1.0 - u * u), 0.0)


# ----------------------------------------------------------------------------
# binning (Section 3.2) of the mean and covariance estimators' sums
# ----------------------------------------------------------------------------

def bin_mean_dense(y, mask, m):
    """Mean bins of gridded data with the 1/N_i weights of Eq. (2.3).

    Returns cnt (int64, number of observations per bin), W = sum_i mask/N_i,
    V = sum_i mask Y/N_i and V2 = sum_i mask Y^2/N_i (the last one feeds the
    variance smoother of Eq. 2.5).  Subjects with no observation are skipped.
    """
    y = np.asarray(y, dtype=np.float64)
    mk = np.asarray(mask).astype(bool)
    Ni = mk.sum(axis=1)
    wi = np.where(Ni > 0, 1.0 / np.maximum(Ni, 1), 0.0)
    cnt = mk.sum(axis=0).astype(np.int64)
    W = np.zeros(y.shape[1])
    V = np.zeros(y.shape[1])
    V2 = np.zeros(y.shape[1])
    for i in range(y.shape[0]):
        obs = mk[i]
        W[obs] += wi[i]
        V[obs] += wi[i] * y[i, obs]
        V2[obs] += wi[i] * y[i, obs] ** 2
    return cnt, W, V, V2


def bin_mean_sparse(offs, t, y, m):
    """Mean bins of scattered data (one loop per subject), weights 1/N_i."""
    P = grid_size(m)
    cnt = np.zeros(P, dtype=np.int64)
    W = np.zeros(P)
    V = np.zeros(P)
    V2 = np.zeros(P)
    b = bin_of(t, m)
    for i in range(len(offs) - 1):
        lo, hi = int(offs[i]), int(offs[i + 1])
        Ni = hi - lo
        if Ni == 0:
            continue
        for j in range(lo, hi):
            cnt[b[j]] += 1
            W[b[j]] += 1.0 / Ni
            V[b[j]] += y[j] / Ni
            V2[b[j]] += y[j] ** 2 / Ni
    return cnt, W, V, V2


def pair_weights(Ni):
    """w_i = 1/(N_i (N_i - 1)) of Eq. (2.4); zero for subjects with N_i < 2."""
    Ni = np.asarray(Ni, dtype=np.float64)
    return np.where(Ni >= 2, 1.0 / np.maximum(Ni * (Ni - 1.0), 1.0), 0.0)


def residuals_dense(y, mask, mu):
    """R_ip = Y_ip - mu_hat(c_p) where observed, 0 elsewhere."""
    mk = np.asarray(mask).astype(bool)
    return np.where(mk, np.asarray(y, dtype=np.float64) - mu[None, :], 0.0)


def bin_cov_dense(r, mask):
    """Covariance bins of gridded data, Eq. (2.4) binned (Section 3.2).

    For each ordered pair of nodes p != q:
      C_pq = #{i : both observed}                      (exact integers)
      W_pq = sum_i w_i M_ip M_iq,  V_pq = sum_i w_i r_ip r_iq M_ip M_iq
    with w_i = 1/(N_i(N_i-1)).  The p == q entries hold only j == l pairs and
    are zero.  ``r`` holds the responses (residuals, or raw Y for raw mode).
    """
    mk = np.asarray(mask).astype(bool)
    mf = mk.astype(np.float64)
    Ni = mk.sum(axis=1)
    wi = pair_weights(Ni)
    rr = np.where(mk, np.asarray(r, dtype=np.float64), 0.0)
    # 0/1 products summed in float64 are exact integers below 2^53
    C = np.rint(mf.T @ mf).astype(np.int64)
    W = (mf * wi[:, None]).T @ mf
    V = (rr * wi[:, None]).T @ rr
    np.fill_diagonal(C, 0)
    np.fill_diagonal(W, 0.0)
    np.fill_diagonal(V, 0.0)
    return C, W, V


def bin_cov_sparse(offs, t, r, m, fold=None, nfold=0):
    """Covariance bins of scattered data: explicit loop over ordered pairs j != l.

    Returns arrays of shape (F, P, P), F = max(nfold, 1):
      C (int64 pair counts), W = sum w_i, V = sum w_i r_ij r_il,
      Q = sum w_i (r_ij r_il)^2 (the held-out sum of squares for CV).
    Subject i contributes to fold ``fold[i]`` (all to fold 0 when nfold = 0).
    """
    P = grid_size(m)
    F = max(nfold, 1)
    C = np.zeros((F, P, P), dtype=np.int64)
    W = np.zeros((F, P, P))
    V = np.zeros((F, P, P))
    Q = np.zeros((F, P, P))
    b = bin_of(t, m)
    for i in range(len(offs) - 1):
        lo, hi = int(offs[i]), int(offs[i + 1])
        Ni = hi - lo
        if Ni < 2:
            continue
        wi = 1.0 / (Ni * (Ni - 1.0))
        f = int(fold[i]) if nfold > 0 else 0
        for j in range(lo, hi):
            for l in range(lo, hi):
                if j == l:
                    continue
                p, q = b[j], b[l]
                prod = r[j] * r[l]
                C[f, p, q] += 1
                W[f, p, q] += wi
                V[f, p, q] += wi * prod
                Q[f, p, q] += wi * prod * prod
    return C, W, V, Q


def residuals_sparse(t, y, mu, m):
    """R_ij = Y_ij - mu_hat(c_bin(t_ij)) for scattered data."""
    return np.asarray(y, dtype=np.float64) - mu[bin_of(t, m)]


# ----------------------------------------------------------------------------
# per-point local linear solve
# ----------------------------------------------------------------------------

def solve_point(A, r, n_nonempty):
    """Intercept of the local linear normal equations A beta = r, with status.

    EMPTY    A_00 = 0 (no weight in the window): NaN.
    FALLBACK fewer non-empty bins than unknowns, or a Cholesky pivot (natural
             order) at most PIVOT_RTOL times its diagonal: local constant T0/S0.
    OK       beta_0 of the full solve.
    """
    D = A.shape[0]
    if not (A[0, 0] > 0.0):
        return math.nan, STATUS_EMPTY
    lc = r[0] / A[0, 0]
    if n_nonempty < D:
        return lc, STATUS_FALLBACK
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        return lc, STATUS_FALLBACK
    piv = np.diag(L) ** 2
    if np.any(piv <= PIVOT_RTOL * np.diag(A)):
        return lc, STATUS_FALLBACK
    beta = np.linalg.solve(A, r)
    return float(beta[0]), STATUS_OK


def unravel(p, m):
    """Per-axis bin coordinates of flat C-order index p."""
    out = []
    for mk in reversed(m):
        out.append(p % mk)
        p //= mk
    return out[::-1]


def _window(j, m, h):
    """Per-axis bin indices i with K(u) > 0, u = (c_i - c_j)/h = (i - j)/(h M).

    The output point is the centre of bin j (per-axis integer coordinates).
    """
    idx, us = [], []
    for k, mk in enumerate(m):
        i = np.arange(mk)
        u = (i - j[k]) / (h[k] * mk)
        keep = np.abs(u) < 1.0
        idx.append(i[keep])
        us.append(u[keep])
    return idx, us


def _window_design(j, m, h):
    """Flat bin indices of the window around centre j, kernel weights, design rows z.

    z = [1, u_1, ..., u_d] with u = (c - x)/h.  The 1/h_k factors of K_h are
    dropped: they scale every equation alike and leave beta_0 unchanged.
    """
    idx, us = _window(j, m, h)
    if any(len(a) == 0 for a in idx):
        return np.zeros(0, dtype=np.int64), np.zeros(0), np.zeros((0, 1 + len(m)))
    grids = np.meshgrid(*idx, indexing="ij")
    ugrids = np.meshgrid(*us, indexing="ij")
    flat = np.zeros(grids[0].size, dtype=np.int64)
    for k, mk in enumerate(m):
        flat = flat * mk + grids[k].ravel()
    uu = np.stack([g.ravel() for g in ugrids], axis=1)
    kern = np.prod(epanechnikov(uu), axis=1)
    z = np.concatenate([np.ones((uu.shape[0], 1)), uu], axis=1)
    return flat, kern, z


def smooth_mean_point(p, m, h, cnt, W, V):
    """mu_hat at the centre of bin p by Eq. (2.3) over the bins:
    A = sum K W z z', r = sum K V z."""
    flat, kern, z = _window_design(unravel(p, m), m, np.asarray(h, float))
    if flat.size == 0:
        return math.nan, STATUS_EMPTY
    kw = kern * W[flat]
    A = (z * kw[:, None]).T @ z
    r = z.T @ (kern * V[flat])
    nonempty = int(np.count_nonzero(cnt[flat] > 0))
    return solve_point(A, r, nonempty)


def smooth_mean(m, h, cnt, W, V):
    """mu_hat and status at every bin centre of the grid ``m``."""
    P = grid_size(m)
    mu = np.empty(P)
    st = np.empty(P, dtype=np.uint8)
    for p in range(P):
        mu[p], st[p] = smooth_mean_point(p, m, h, cnt, W, V)
    return mu, st


def cov_moments_point(p, q, m, h, C, W, V):
    """Normal equations of Eq. (2.4) binned, at output pair (c_p, c_q).

    Sums run over bin pairs (p', q') in the product window:
      A = sum K(s) K(t) W z z',  r = sum K(s) K(t) V z,
      z = [1, u_s, u_t] (2d + 1 entries).
    Returns (A, r, number of non-empty bin pairs).
    """
    h = np.asarray(h, float)
    fs, ks, zs = _window_design(unravel(p, m), m, h)
    ft, kt, zt = _window_design(unravel(q, m), m, h)
    d = len(m)
    D = 2 * d + 1
    if fs.size == 0 or ft.size == 0:
        return np.zeros((D, D)), np.zeros(D), 0
    Wb = W[np.ix_(fs, ft)]
    Vb = V[np.ix_(fs, ft)]
    Cb = C[np.ix_(fs, ft)]
    Kst = ks[:, None] * kt[None, :]
    # design rows for every (p', q') pair of the window
    z = np.concatenate([
        np.ones((fs.size, ft.size, 1)),
        np.broadcast_to(zs[:, None, 1:], (fs.size, ft.size, d)),
        np.broadcast_to(zt[None, :, 1:], (fs.size, ft.size, d)),
    ], axis=2).reshape(-1, D)
    kw = (Kst * Wb).ravel()
    kv = (Kst * Vb).ravel()
    A = (z * kw[:, None]).T @ z
    r = z.T @ kv
    return A, r, int(np.count_nonzero(Cb > 0))


def smooth_cov_points(pairs, m, h, C, W, V, mu=None):
    """Gamma_hat at output bin-centre pairs ``pairs`` ((K, 2) flat indices).

    Residual mode (mu=None): Gamma_hat = b0.  Raw mode (responses Y Y, mu
    given): Gamma_hat = b0 - mu_hat(s) mu_hat(t), Eq. (2.4).
    """
    out = np.empty(len(pairs))
    st = np.empty(len(pairs), dtype=np.uint8)
    for k, (p, q) in enumerate(pairs):
        A, r, ne = cov_moments_point(int(p), int(q), m, h, C, W, V)
        if A[0, 0] > 0:
            out[k], st[k] = solve_point(A, r, ne)
        else:
            out[k], st[k] = math.nan, STATUS_EMPTY
        if mu is not None and st[k] != STATUS_EMPTY:
            out[k] -= mu[p] * mu[q]
    return out, st


# ----------------------------------------------------------------------------
# whole-grid moments by separable sums (pinned to the window sums above)
# ----------------------------------------------------------------------------

def tap_weights(mk, hk, power):
    """1-D weights K(u) u^power for bin offsets k, u = k/(h M), |u| < 1."""
    ks = np.arange(-mk + 1, mk)
    u = ks / (hk * mk)
    keep = np.abs(u) < 1.0
    ks, u = ks[keep], u[keep]
    return ks, epanechnikov(u) * u ** power


def conv_axis(arr, axis, mk, hk, power):
    """out[.., j, ..] = sum_k K(u_k) u_k^power arr[.., j + k, ..], zero outside."""
    ks, wts = tap_weights(mk, hk, power)
    out = np.zeros_like(arr)
    n = arr.shape[axis]
    for k, wk in zip(ks, wts):
        lo, hi = max(0, -k), min(n, n - k)
        if lo >= hi:
            continue
        dst = [slice(None)] * arr.ndim
        src = [slice(None)] * arr.ndim
        dst[axis] = slice(lo, hi)
        src[axis] = slice(lo + k, hi + k)
        out[tuple(dst)] += wk * arr[tuple(src)]
    return out


def moment_indices(naxes, maxdeg):
    """Multi-indices alpha over ``naxes`` axes with |alpha| <= maxdeg."""
    out = [()]
    for _ in range(naxes):
        out = [a + (e,) for a in out for e in range(maxdeg + 1)]
    return [a for a in out if sum(a) <= maxdeg]


def cov_moments_grid(m, h, W, V):
    """All kernel moments of Eq. (2.4) binned, at every output pair, FP64.

    S[alpha] = sum K W prod u^alpha (|alpha| <= 2), T[alpha] = sum K V prod u^alpha
    (|alpha| <= 1) over the 2d axes (s_1..s_d, t_1..t_d).  Each moment is the
    product-kernel sum evaluated as 2d successive 1-D sums (the kernel is a
    product over coordinates); no intermediate is shared between moments.
    """
    d = len(m)
    shape = tuple(m) + tuple(m)
    Wg = np.asarray(W, float).reshape(shape)
    Vg = np.asarray(V, float).reshape(shape)
    axes_m = list(m) + list(m)
    axes_h = list(h) + list(h)
    S, T = {}, {}
    for alpha in moment_indices(2 * d, 2):
        a = Wg
        for ax in range(2 * d):
            a = conv_axis(a, ax, axes_m[ax], axes_h[ax], alpha[ax])
        S[alpha] = a.reshape(grid_size(m), grid_size(m))
    for alpha in moment_indices(2 * d, 1):
        a = Vg
        for ax in range(2 * d):
            a = conv_axis(a, ax, axes_m[ax], axes_h[ax], alpha[ax])
        T[alpha] = a.reshape(grid_size(m), grid_size(m))
    return S, T


def nonempty_grid(m, h, C):
    """Number of non-empty bin pairs in each output point's window (2d-dim box sum)."""
    d = len(m)
    shape = tuple(m) + tuple(m)
    a = (np.asarray(C).reshape(shape) > 0).astype(np.float64)
    for ax in range(2 * d):
        mk, hk = (list(m) + list(m))[ax], (list(h) + list(h))[ax]
        ks, _ = tap_weights(mk, hk, 0)
        out = np.zeros_like(a)
        n = a.shape[ax]
        for k in ks:
            lo, hi = max(0, -k), min(n, n - k)
            if lo >= hi:
                continue
            dst = [slice(None)] * a.ndim
            src = [slice(None)] * a.ndim
            dst[ax] = slice(lo, hi)
            src[ax] = slice(lo + k, hi + k)
            out[tuple(dst)] += a[tuple(src)]
        a = out
    return np.rint(a).astype(np.int64).reshape(grid_size(m), grid_size(m))


def normal_matrix(S, T, d, p, q):
    """Assemble A (2d+1 square) and r at output pair (p, q) from moment arrays."""
    D = 2 * d + 1
    A = np.empty((D, D))
    r = np.empty(D)
    unit = []
    for j in range(D):
        e = [0] * (2 * d)
        if j > 0:
            e[j - 1] = 1
        unit.append(e)
    for i in range(D):
        r[i] = T[tuple(unit[i])][p, q]
        for j in range(D):
            alpha = tuple(a + b for a, b in zip(unit[i], unit[j]))
            A[i, j] = S[alpha][p, q]
    return A, r


def smooth_cov_grid(m, h, C, W, V, mu=None):
    """Gamma_hat (P x P) and status at every output pair, via cov_moments_grid."""
    d = len(m)
    P = grid_size(m)
    S, T = cov_moments_grid(m, h, W, V)
    ne = nonempty_grid(m, h, C)
    G = np.empty((P, P))
    st = np.empty((P, P), dtype=np.uint8)
    for p in range(P):
        for q in range(P):
            A, r = normal_matrix(S, T, d, p, q)
            G[p, q], st[p, q] = solve_point(A, r, ne[p, q])
            if mu is not None and st[p, q] != STATUS_EMPTY:
                G[p, q] -= mu[p] * mu[q]
    return G, st


# ----------------------------------------------------------------------------
# the dense pipeline up to Gamma_hat (Section 2.1 estimators, binned)
# ----------------------------------------------------------------------------

def dense_gamma(y, mask, m, h_mu, h_cov, mode="residual"):
    """mu_hat, Gamma_hat and statuses for gridded data (full grid, FP64)."""
    cnt, W, V, _ = bin_mean_dense(y, mask, m)
    mu, st_mu = smooth_mean(m, h_mu, cnt, W, V)
    mu0 = np.where(np.isnan(mu), 0.0, mu)
    if mode == "residual":
        r = residuals_dense(y, mask, mu0)
        C, Wc, Vc = bin_cov_dense(r, mask)
        G, st = smooth_cov_grid(m, h_cov, C, Wc, Vc)
    else:
        C, Wc, Vc = bin_cov_dense(y, mask)
        G, st = smooth_cov_grid(m, h_cov, C, Wc, Vc, mu=mu0)
    return dict(mu=mu, mu_status=st_mu, cnt=cnt, C=C, W=Wc, V=Vc, gamma=G, status=st)
