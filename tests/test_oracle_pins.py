"""Pins of the FP64 oracle to facts outside itself (CPU only).

Every check compares the oracle with something it does not contain: closed
forms, exact rational arithmetic, the unbinned estimator of Eq. (2.3)/(2.4)
solved by a generic least-squares routine over raw observations, invariants
(exact reproduction of affine surfaces by local linear fits, symmetry of
Gamma_hat), integer brute force, and a dense symmetric eigensolver.  The
planted-mistake tests at the end show that a plausible error in the oracle
fails at least one pin.
"""
from fractions import Fraction

import numpy as np
import pytest

import fpca_synth as fs
from oracle import cv as ocv
from oracle import eigen as oe
from oracle import smoother as sm


def epan_frac(u):
    return Fraction(3, 4) * (1 - u * u) if abs(u) < 1 else Fraction(0)


# ----------------------------------------------------------------------------
# binning counts: closed forms and integer brute force (bit-exact)
# ----------------------------------------------------------------------------

def test_counts_full_grid_closed_form():
    n, P = 7, 12
    mask = np.ones((n, P), dtype=np.uint8)
    C, W, V = sm.bin_cov_dense(np.zeros((n, P)), mask)
    expect = np.full((P, P), n, dtype=np.int64)
    np.fill_diagonal(expect, 0)
    assert np.array_equal(C, expect)
    # W_pq = n / (P (P - 1)) off the diagonal for fully observed subjects
    wexp = np.full((P, P), n / (P * (P - 1.0)))
    np.fill_diagonal(wexp, 0.0)
    assert np.allclose(W, wexp, rtol=1e-15, atol=0)


def test_counts_mask_integer_bruteforce():
    rng = np.random.default_rng(3)
    n, P = 9, 10
    mask = (rng.random((n, P)) < 0.6).astype(np.uint8)
    C, _, _ = sm.bin_cov_dense(np.zeros((n, P)), mask)
    brute = np.zeros((P, P), dtype=np.int64)
    for i in range(n):
        obs = [p for p in range(P) if mask[i, p]]
        for a in obs:
            for b in obs:
                if a != b:
                    brute[a, b] += 1
    assert np.array_equal(C, brute)


def test_sparse_counts_histogram_identity():
    """C_pq = sum_i (n_ip n_iq - [p == q] n_ip) with n_ip the per-subject bin counts."""
    D = fs.make_sparse(2, (4, 5), 30, [1.0, 0.5], nmin=1, nmax=9, seed=11, nfold=3)
    r = np.ones_like(D.y)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, D.nfold)
    P = D.P
    expect = np.zeros((3, P, P), dtype=np.int64)
    b = sm.bin_of(D.t, D.m)
    for i in range(D.n):
        cnt = np.bincount(b[D.offs[i]:D.offs[i + 1]], minlength=P).astype(np.int64)
        expect[D.fold[i]] += np.outer(cnt, cnt) - np.diag(cnt)
    assert np.array_equal(C, expect)
    # with unit responses V = W and Q = W
    assert np.allclose(V, W) and np.allclose(Q, W)


def test_mean_bins_sparse_vs_dense_layout():
    """Scattered points placed on bin centres bin exactly like gridded data."""
    rng = np.random.default_rng(5)
    m = (3, 4)
    n, P = 6, 12
    mask = (rng.random((n, P)) < 0.7).astype(np.uint8)
    mask[:, 0] = 1
    y = rng.standard_normal((n, P))
    c = sm.centres(m)
    offs = [0]
    ts, ys = [], []
    for i in range(n):
        for p in range(P):
            if mask[i, p]:
                ts.append(c[p])
                ys.append(y[i, p])
        offs.append(len(ys))
    a = sm.bin_mean_dense(y, mask, m)
    b = sm.bin_mean_sparse(np.array(offs), np.array(ts), np.array(ys), m)
    assert np.array_equal(a[0], b[0])
    for u, v in zip(a[1:], b[1:]):
        assert np.allclose(u, v, rtol=1e-14, atol=1e-15)


def test_bin_of_edges():
    m = (4,)
    t = np.array([[0.0], [0.25], [0.2499999], [0.999999], [1.0]])
    assert list(sm.bin_of(t, m)) == [0, 1, 0, 3, 3]


# ----------------------------------------------------------------------------
# the local linear operator
# ----------------------------------------------------------------------------

def test_d1_textbook_exact_rational():
    """d = 1: beta_0 = sum K (S2 - S1 u) V / (S0 S2 - S1^2), in exact rationals."""
    m = (8,)
    h = 0.4  # h M = 3.2: taps -3..3
    rng = np.random.default_rng(1)
    Wb = rng.integers(1, 5, size=8).astype(float)
    Vb = rng.integers(-9, 10, size=8).astype(float)
    cnt = np.ones(8, dtype=np.int64)
    mu, st = sm.smooth_mean(m, [h], cnt, Wb, Vb)
    hm = Fraction(16, 5)
    for j in range(8):
        S0 = S1 = S2 = T0 = T1 = Fraction(0)
        for i in range(8):
            u = Fraction(i - j) / hm
            k = epan_frac(u)
            w = Fraction(Wb[i]).limit_denominator()
            v = Fraction(Vb[i]).limit_denominator()
            S0 += k * w
            S1 += k * w * u
            S2 += k * w * u * u
            T0 += k * v
            T1 += k * v * u
        exact = (S2 * T0 - S1 * T1) / (S0 * S2 - S1 * S1)
        assert st[j] == sm.STATUS_OK
        assert abs(mu[j] - float(exact)) <= 1e-13 * max(1.0, abs(float(exact)))


def _random_positive_bins(rng, P, fill=0.8):
    W = rng.random(P) * (rng.random(P) < fill)
    return W


def test_mean_affine_reproduction_2d():
    rng = np.random.default_rng(2)
    m = (9, 7)
    c = sm.centres(m)
    W = _random_positive_bins(rng, c.shape[0])
    a, b = 0.7, np.array([-1.3, 2.1])
    V = W * (a + c @ b)
    cnt = (W > 0).astype(np.int64)
    mu, st = sm.smooth_mean(m, [0.35, 0.45], cnt, W, V)
    ok = st == sm.STATUS_OK
    assert ok.sum() > 0.8 * ok.size
    assert np.max(np.abs(mu[ok] - (a + c[ok] @ b))) < 1e-12


def test_cov_affine_reproduction_and_symmetry_2d():
    rng = np.random.default_rng(4)
    m = (5, 6)
    P = 30
    c = sm.centres(m)
    A = rng.random((P, P)) * (rng.random((P, P)) < 0.7)
    W = A + A.T
    np.fill_diagonal(W, 0.0)
    C = (W > 0).astype(np.int64)
    a, bs, bt = 0.3, np.array([1.1, -0.4]), np.array([-0.7, 0.9])
    Vaff = W * (a + (c @ bs)[:, None] + (c @ bt)[None, :])
    G, st = sm.smooth_cov_grid(m, [0.5, 0.45], C, W, Vaff)
    ok = st == sm.STATUS_OK
    truth = a + (c @ bs)[:, None] + (c @ bt)[None, :]
    assert ok.mean() > 0.9
    assert np.max(np.abs(G[ok] - truth[ok])) < 1e-11
    # symmetry with symmetric responses
    B = rng.standard_normal((P, P))
    Vs = W * (B + B.T)
    G2, st2 = sm.smooth_cov_grid(m, [0.5, 0.45], C, W, Vs)
    assert np.array_equal(st2, st2.T)
    ok2 = st2 != sm.STATUS_EMPTY
    assert np.max(np.abs(G2 - G2.T)[ok2]) < 1e-12


def test_separable_moments_equal_window_sums():
    rng = np.random.default_rng(6)
    m = (5, 4)
    P = 20
    W = rng.random((P, P))
    V = rng.standard_normal((P, P))
    C = np.ones((P, P), dtype=np.int64)
    h = [0.55, 0.6]
    G, st = sm.smooth_cov_grid(m, h, C, W, V)
    pairs = np.array([(p, q) for p in range(P) for q in range(P)])
    g2, st2 = sm.smooth_cov_points(pairs, m, h, C, W, V)
    assert np.array_equal(st.ravel(), st2)
    assert np.allclose(G.ravel(), g2, rtol=1e-11, atol=1e-12)


def _unbinned_lstsq(X, y, w):
    """Weighted least squares by a generic solver: minimise sum w (y - X b)^2."""
    sw = np.sqrt(w)
    b, *_ = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)
    return b[0]


def test_binned_equals_unbinned_mean_and_cov():
    """Points on bin centres: the binned fit equals Eq. (2.3)/(2.4) fitted on raw data."""
    rng = np.random.default_rng(8)
    m = (4, 4)
    h = [0.55, 0.55]
    n = 5
    P = 16
    c = sm.centres(m)
    mask = (rng.random((n, P)) < 0.8).astype(np.uint8)
    y = rng.standard_normal((n, P))
    cnt, W, V, _ = sm.bin_mean_dense(y, mask, m)
    mu, st = sm.smooth_mean(m, h, cnt, W, V)
    # raw-data mean fit at each centre, Eq. (2.3)
    for j in range(P):
        rows, ys, ws = [], [], []
        for i in range(n):
            Ni = mask[i].sum()
            for p in range(P):
                if not mask[i, p]:
                    continue
                u = (c[p] - c[j]) / np.array(h)
                k = np.prod(np.where(np.abs(u) < 1, 0.75 * (1 - u * u), 0.0))
                if k > 0:
                    rows.append([1.0, *(c[j] - c[p])])
                    ys.append(y[i, p])
                    ws.append(k / Ni)
        if st[j] == sm.STATUS_OK:
            assert abs(mu[j] - _unbinned_lstsq(np.array(rows), np.array(ys), np.array(ws))) < 1e-11
    # raw-pair covariance fit, Eq. (2.4), residual responses
    r = sm.residuals_dense(y, mask, mu)
    C, Wc, Vc = sm.bin_cov_dense(r, mask)
    G, stc = sm.smooth_cov_grid(m, h, C, Wc, Vc)
    checked = 0
    for (a, b) in [(0, 5), (3, 12), (6, 6), (15, 0), (9, 10)]:
        rows, ys, ws = [], [], []
        for i in range(n):
            obs = [p for p in range(P) if mask[i, p]]
            Ni = len(obs)
            if Ni < 2:
                continue
            for p in obs:
                for q in obs:
                    if p == q:
                        continue
                    us = (c[p] - c[a]) / np.array(h)
                    ut = (c[q] - c[b]) / np.array(h)
                    k = np.prod(np.where(np.abs(us) < 1, 0.75 * (1 - us * us), 0.0)) * \
                        np.prod(np.where(np.abs(ut) < 1, 0.75 * (1 - ut * ut), 0.0))
                    if k > 0:
                        rows.append([1.0, *(c[a] - c[p]), *(c[b] - c[q])])
                        ys.append(r[i, p] * r[i, q])
                        ws.append(k / (Ni * (Ni - 1.0)))
        if stc[a, b] == sm.STATUS_OK:
            ref = _unbinned_lstsq(np.array(rows), np.array(ys), np.array(ws))
            assert abs(G[a, b] - ref) < 1e-11
            checked += 1
    assert checked >= 4


def test_raw_mode_matches_definition():
    """Raw mode: Gamma_hat = b0(Y Y) - mu(s) mu(t) (Eq. 2.4 as printed)."""
    D = fs.make_dense(2, (5, 5), 20, [2.0, 1.0], sigma=0.3, seed=9)
    h = [0.5, 0.5]
    out = sm.dense_gamma(D.y, D.mask, D.m, h, h, mode="raw")
    C, W, V = sm.bin_cov_dense(D.y, D.mask)
    G0, st0 = sm.smooth_cov_grid(D.m, h, C, W, V)
    mu = out["mu"]
    ok = st0 == sm.STATUS_OK
    assert np.allclose(out["gamma"][ok], (G0 - np.outer(mu, mu))[ok], rtol=1e-12, atol=1e-12)


def test_status_rules():
    m = (6,)
    W = np.zeros(6)
    V = np.zeros(6)
    cnt = np.zeros(6, dtype=np.int64)
    W[0], V[0], cnt[0] = 2.0, 4.0, 1
    # h M = 1.2: taps -1..1; bin 0 alone in the window of bins 0 and 1
    mu, st = sm.smooth_mean(m, [0.2], cnt, W, V)
    assert st[0] == sm.STATUS_FALLBACK and mu[0] == 2.0
    assert st[1] == sm.STATUS_FALLBACK and mu[1] == 2.0
    assert st[3] == sm.STATUS_EMPTY and np.isnan(mu[3])


# ----------------------------------------------------------------------------
# eigen step
# ----------------------------------------------------------------------------

def test_rproj_exact_on_rank_r():
    rng = np.random.default_rng(12)
    m = (10, 10)
    P = 100
    U, _ = np.linalg.qr(rng.standard_normal((P, 5)))
    theta = np.array([9.0, 5.0, 3.0, 2.0, 1.0])
    G = (U * theta) @ U.T
    dom = np.ones(P, dtype=bool)
    lam_f, phi_f, fve_f = oe.eig_full(G, m, dom, 5)
    om = fs.gaussian_test_matrix(P, 8, 1)
    lam_r, phi_r, fve_r = oe.rproj_eig(G, m, dom, om, 5, 0)
    assert np.allclose(lam_f, theta / P, rtol=1e-12)
    assert np.allclose(lam_r, lam_f, rtol=1e-10)
    assert np.allclose(phi_r, phi_f, atol=1e-9)
    assert np.allclose(fve_r, fve_f, rtol=1e-12) and abs(fve_f[-1] - 1.0) < 1e-12


def test_rescaling_orthonormal_riemann():
    """phi = psi/sqrt(dV): the Riemann sum of phi_k phi_l over the grid is the identity."""
    D = fs.dense_2d_full()
    G = D.true_gamma()
    lam, phi, _ = oe.eig_full(G, D.m, np.ones(D.P, bool), 4)
    dv = 1.0 / D.P
    assert np.allclose(phi.T @ phi * dv, np.eye(4), atol=1e-12)
    assert np.allclose(lam, D.lam, rtol=1e-12)
    assert oe.subspace_angle(phi, D.true_phi()) < 1e-10


@pytest.mark.slow
def test_eigen_recovery_from_synthetic_data():
    """Large n, small noise: lambda_hat and phi_hat approach the truth (Thm 2.4 rates)."""
    D = fs.make_dense(2, (16, 16), 3000, [8.0, 4.0, 2.0, 1.0], sigma=0.1, seed=21)
    # h M = 1.12: taps -1..1.  The local linear bias of a frequency-1 product
    # over the four axes shrinks lambda by about 1 - 4 (2 pi)^2 m2 / 2 ~ 0.91,
    # m2 = sum K u^2 h^2 / sum K ~ 1.1e-3 here; sampling error ~ sqrt(2/n) ~ 3%.
    h = [0.07, 0.07]
    out = sm.dense_gamma(D.y, D.mask, D.m, h, h)
    lam, phi, _ = oe.eig_full(out["gamma"], D.m, out["cnt"] > 0, 4)
    assert np.all(np.abs(lam / D.lam - 1) < 0.15)
    assert np.all(np.abs((lam / lam[0]) / (D.lam / D.lam[0]) - 1) < 0.1)
    assert oe.subspace_angle(phi, D.true_phi()) < 0.05
    for k in range(4):
        assert oe.subspace_angle(phi[:, :k + 1], D.true_phi()[:, :k + 1]) < 0.1


# ----------------------------------------------------------------------------
# cross-validation
# ----------------------------------------------------------------------------

def test_cv_from_bins_equals_bruteforce():
    D = fs.make_sparse(1, (6,), 24, [1.0, 0.5], nmin=2, nmax=6, sigma=0.3, mean="1d", seed=17, nfold=3)
    m = D.m
    r = D.y - 0.1  # any fixed residual definition
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, m, D.fold, D.nfold)
    h = 0.45
    score = ocv.cv_score(m, [h], C, W, V, Q)
    c = sm.centres(m)
    b = sm.bin_of(D.t, m)
    num = 0.0
    den = 0.0
    for f in range(3):
        # unbinned fit of training pairs, moved to bin centres, by lstsq
        rows_all = []
        for i in range(D.n):
            if D.fold[i] == f:
                continue
            lo, hi = D.offs[i], D.offs[i + 1]
            Ni = hi - lo
            if Ni < 2:
                continue
            for j in range(lo, hi):
                for l in range(lo, hi):
                    if j != l:
                        rows_all.append((c[b[j]][0], c[b[l]][0], r[j] * r[l], 1.0 / (Ni * (Ni - 1.0))))
        rows_all = np.array(rows_all)

        def fit(xs, xt):
            us = (rows_all[:, 0] - xs) / h
            ut = (rows_all[:, 1] - xt) / h
            k = np.where(np.abs(us) < 1, 0.75 * (1 - us * us), 0) * \
                np.where(np.abs(ut) < 1, 0.75 * (1 - ut * ut), 0)
            sel = k > 0
            X = np.stack([np.ones(sel.sum()), xs - rows_all[sel, 0], xt - rows_all[sel, 1]], 1)
            return _unbinned_lstsq(X, rows_all[sel, 2], k[sel] * rows_all[sel, 3])

        for i in range(D.n):
            if D.fold[i] != f:
                continue
            lo, hi = D.offs[i], D.offs[i + 1]
            Ni = hi - lo
            if Ni < 2:
                continue
            for j in range(lo, hi):
                for l in range(lo, hi):
                    if j != l:
                        g = fit(c[b[j]][0], c[b[l]][0])
                        w = 1.0 / (Ni * (Ni - 1.0))
                        num += w * (r[j] * r[l] - g) ** 2
                        den += w
    assert np.isfinite(score)
    assert abs(score - num / den) < 1e-10 * max(1.0, abs(score))


# ----------------------------------------------------------------------------
# planted mistakes: each must fail a pin above
# ----------------------------------------------------------------------------

def _affine_cov_error(monkeypatch=None):
    rng = np.random.default_rng(4)
    m = (5, 6)
    P = 30
    c = sm.centres(m)
    A = rng.random((P, P)) * (rng.random((P, P)) < 0.7)
    W = A + A.T
    np.fill_diagonal(W, 0.0)
    C = (W > 0).astype(np.int64)
    truth = 0.3 + (c @ np.array([1.1, -0.4]))[:, None] + (c @ np.array([-0.7, 0.9]))[None, :]
    pairs = np.array([(p, q) for p in range(P) for q in range(P)])
    G, st = sm.smooth_cov_points(pairs, m, [0.5, 0.45], C, W, W * truth)
    ok = st == sm.STATUS_OK
    return np.max(np.abs(G[ok] - truth.ravel()[ok]))


def test_planted_dropped_cross_term_fails_affine(monkeypatch):
    assert _affine_cov_error() < 1e-11
    orig = sm.cov_moments_point

    def dropped(p, q, m, h, C, W, V):
        A, r, ne = orig(p, q, m, h, C, W, V)
        A = A.copy()
        d = len(m)
        A[1:1 + d, 1 + d:] = 0.0  # forget the s-t cross moments
        A[1 + d:, 1:1 + d] = 0.0
        return A, r, ne

    monkeypatch.setattr(sm, "cov_moments_point", dropped)
    assert _affine_cov_error() > 1e-6


def test_planted_wrong_kernel_fails_textbook(monkeypatch):
    monkeypatch.setattr(sm, "epanechnikov",
                        lambda u: np.where(np.abs(u) < 1, 0.75 * (1 - np.abs(u)), 0.0))
    with pytest.raises(AssertionError):
        test_d1_textbook_exact_rational()


def test_planted_wrong_weights_fail_unbinned(monkeypatch):
    monkeypatch.setattr(sm, "pair_weights", lambda Ni: 1.0 / np.maximum(np.asarray(Ni, float) ** 2, 1))
    with pytest.raises(AssertionError):
        test_binned_equals_unbinned_mean_and_cov()


def test_planted_missing_rescale_fails_riemann(monkeypatch):
    monkeypatch.setattr(oe, "rescale", lambda theta, psi, m: (theta, psi))
    with pytest.raises(AssertionError):
        test_rescaling_orthonormal_riemann()
