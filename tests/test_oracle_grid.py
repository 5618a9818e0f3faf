"""Pins of oracle/grid.py (the stacked whole-grid covariance smoother) to the
per-point definitions of oracle/smoother.py, on the CPU.

grid.smooth_cov must give the statuses of smoother.smooth_cov_grid exactly and its
values to rounding; its band-matrix sums must equal the offset-loop sums of
smoother.conv_axis; the CV score through it must equal the one through the
per-point smoother.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import cv as ocv
from oracle import grid as og
from oracle import smoother as sm


@pytest.mark.parametrize("mk,hk,power", [(7, 0.3, 0), (16, 0.15, 1), (16, 0.4, 2), (5, 1.5, 2),
                                         (12, 0.05, 0)])
def test_band_matrix_sum_equals_offset_sum(mk, hk, power):
    rng = np.random.default_rng(mk * 10 + power)
    a = rng.standard_normal((3, mk, 4))
    ref = sm.conv_axis(a, 1, mk, hk, power)
    got = og.conv_axis_mm(a, 1, mk, hk, power)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_band_matrix_box_counts_the_window():
    # box weights: the window length of every output (a closed form)
    mk, hk = 9, 0.3
    T = max(k for k in range(mk) if k / (hk * mk) < 1.0)
    got = og.conv_axis_mm(np.ones((1, mk)), 1, mk, hk, 0, box=True)[0]
    ref = [min(T, mk - 1 - x) - max(-T, -x) + 1 for x in range(mk)]
    assert np.array_equal(got, ref)


def _bins(m, seed, dropout=0.25):
    D = fs.make_dense(len(m), m, 40, [2.0, 1.0], sigma=0.3, seed=seed, dropout=dropout,
                      domain="disk" if len(m) == 2 else "full",
                      mean="sincos" if len(m) == 2 else "1d")
    cnt, Wm, Vm, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, (0.2,) * len(m), cnt, Wm, Vm)
    mu = np.where(np.isnan(mu), 0.0, mu)
    return sm.bin_cov_dense(sm.residuals_dense(D.y, D.mask, mu), D.mask)


@pytest.mark.parametrize("m,h", [((10, 12), (0.25, 0.2)), ((9, 8), (0.5, 0.12)), ((30,), (0.1,)),
                                 ((6, 7), (0.08, 0.08))])
def test_stacked_grid_equals_per_point_smoother(m, h):
    C, W, V = _bins(m, seed=sum(m))
    G0, s0 = sm.smooth_cov_grid(m, h, C, W, V)
    G1, s1 = og.smooth_cov(m, h, C, W, V)
    assert np.array_equal(s0, s1)
    assert np.array_equal(np.isnan(G0), np.isnan(G1))
    fin = ~np.isnan(G0)
    assert np.allclose(G1[fin], G0[fin], rtol=1e-11, atol=1e-12 * np.abs(G0[fin]).max())
    # selected rows only
    rows = np.array([0, 5, len(G0) - 1])
    Gr, sr = og.smooth_cov(m, h, C, W, V, rows=rows, chunk=37)
    assert np.array_equal(sr, s0[rows])
    assert np.allclose(Gr[fin[rows]], G0[rows][fin[rows]], rtol=1e-11, atol=1e-12)


def test_stacked_grid_raw_mode_subtracts_the_mean_product():
    m, h = (8, 9), (0.3, 0.3)
    C, W, V = _bins(m, seed=4)
    mu = np.linspace(-1.0, 2.0, 72)
    G0, s0 = sm.smooth_cov_grid(m, h, C, W, V, mu=mu)
    G1, s1 = og.smooth_cov(m, h, C, W, V, mu=mu)
    assert np.array_equal(s0, s1)
    fin = ~np.isnan(G0)
    assert np.allclose(G1[fin], G0[fin], rtol=1e-11, atol=1e-12)


def test_cv_through_the_stacked_grid_equals_per_point():
    D = fs.make_sparse(2, (7, 6), 150, [2.0, 1.0], nmin=3, nmax=10, sigma=0.4, seed=3, nfold=4)
    mu = np.linspace(-0.2, 0.3, D.P)
    r = sm.residuals_sparse(D.t, D.y, mu, D.m)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, 4)
    for h in (0.2, 0.35):
        a = ocv.cv_score(D.m, [h, h], C, W, V, Q)
        b = ocv.cv_score(D.m, [h, h], C, W, V, Q, smooth=og.smooth_cov)
        assert (np.isinf(a) and np.isinf(b)) or abs(a - b) <= 1e-11 * abs(a)


def test_vectorised_sparse_binning_equals_pair_loop():
    D = fs.make_sparse(2, (6, 5), 120, [2.0, 1.0], nmin=1, nmax=9, sigma=0.4, seed=8, nfold=3)
    r = sm.residuals_sparse(D.t, D.y, np.linspace(-0.3, 0.2, D.P), D.m)
    ref = sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, 3)
    got = og.bin_cov_sparse_pairs(D.offs, D.t, r, D.m, D.fold, 3)
    assert np.array_equal(got[0], ref[0])
    for a, b in zip(got[1:], ref[1:]):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-15)
    # no folds
    ref = sm.bin_cov_sparse(D.offs, D.t, r, D.m)
    got = og.bin_cov_sparse_pairs(D.offs, D.t, r, D.m)
    assert np.array_equal(got[0], ref[0])
    assert np.allclose(got[2], ref[2], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d,m", [(1, (40,)), (2, (9, 7))])
def test_mean_cv_bin_formula_equals_held_out_observations(d, m):
    """CV of the mean smoother from per-fold bins equals the held-out error summed
    observation by observation (brute force), for several bandwidths."""
    D = fs.make_sparse(d, m, 80, [2.0, 1.0], nmin=2, nmax=9, sigma=0.4, seed=21 + d, nfold=4,
                       mean="1d" if d == 1 else "sincos")
    cnt, W, V, V2 = ocv.mean_fold_bins(D.offs, D.t, D.y, m, D.fold, 4)
    for h in (0.12, 0.3, 0.6):
        a = ocv.mean_cv_score(m, [h] * d, cnt, W, V, V2)
        b = ocv.mean_cv_bruteforce(D.offs, D.t, D.y, m, [h] * d, D.fold, 4)
        assert (np.isinf(a) and np.isinf(b)) or abs(a - b) <= 1e-11 * abs(b)
    # the fold bins add up to the bins of all subjects
    c0, W0, V0, V20 = sm.bin_mean_sparse(D.offs, D.t, D.y, m)
    assert np.array_equal(cnt.sum(0), c0)
    assert np.allclose(W.sum(0), W0, rtol=1e-13) and np.allclose(V2.sum(0), V20, rtol=1e-12)


def test_mean_cv_planted_mistake_is_caught():
    """A mean fitted WITH the held-out fold (no cross-validation) scores lower than
    the held-out score: the bin formula must not be leaking the fold."""
    m = (30,)
    D = fs.make_sparse(1, m, 60, [2.0], nmin=3, nmax=8, sigma=0.6, seed=5, nfold=3, mean="1d")
    cnt, W, V, V2 = ocv.mean_fold_bins(D.offs, D.t, D.y, m, D.fold, 3)
    h = [0.08]
    honest = ocv.mean_cv_score(m, h, cnt, W, V, V2)
    leak = 0.0
    wsum = 0.0
    mu, st = sm.smooth_mean(m, h, cnt.sum(0), W.sum(0), V.sum(0))
    for f in range(3):
        inc = st != sm.STATUS_EMPTY
        g = np.where(inc, mu, 0.0)
        leak += float(np.sum((V2[f] - 2 * g * V[f] + g * g * W[f])[inc]))
        wsum += float(np.sum(W[f][inc]))
    assert leak / wsum < honest
