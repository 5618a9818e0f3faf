"""Pins of the oracle's 32-number dataset summary (`oracle/features.py`).

Every feature is checked against a value worked out by hand from its
definition on small inputs whose statistics have closed forms: subject and bin
counts with known moments, bins built from explicit observations, binned means
that are linear or quadratic along an axis (finite differences known exactly),
and covariance surfaces that vary along one direction only.  A wrong axis
step, a dropped emptiness rule or a sign error in a moment changes one of
these values.
"""
import math

import numpy as np
import pytest

from oracle import features as of

EPS = of.EPS


def _flat_bins(mb):
    """Mean bins with W = 1, V = mb, V2 = mb^2 (no within-bin spread)."""
    mb = np.asarray(mb, dtype=np.float64).ravel()
    P = mb.size
    return np.ones(P), np.ones(P), mb.copy(), mb ** 2


def _cov_bins(g):
    g = np.asarray(g, dtype=np.float64)
    return np.ones_like(g), np.ones_like(g), g.copy()


def test_subject_and_bin_counts():
    m = (4,)
    Ni = np.array([2.0, 4.0, 6.0])
    cnt = np.array([0.0, 0.0, 3.0, 1.0])
    W = np.array([0.0, 0.0, 1.0, 1.0])
    V = np.array([0.0, 0.0, 2.0, 5.0])
    V2 = V ** 2
    C, Wc, Vc = np.zeros((4, 4)), np.zeros((4, 4)), np.zeros((4, 4))
    f = of.features(1, m, Ni, cnt, W, V, V2, C, Wc, Vc)
    assert f[0] == 1
    assert f[1] == pytest.approx(math.log(3))
    assert f[2] == pytest.approx(math.log(4))
    assert f[3] == pytest.approx(math.sqrt(8.0 / 3.0) / 4.0)   # population std / mean
    assert f[4] == pytest.approx(math.log(2))
    assert f[5] == pytest.approx(math.log(6))
    # counts 0, 0, 3, 1: mean 1, variance 1.5, third central moment 1.5, half empty
    assert f[6] == pytest.approx(math.log(2))
    assert f[7] == pytest.approx(1.5)
    assert f[8] == pytest.approx(1.5 / 1.5 ** 1.5)
    assert f[9] == pytest.approx(0.5)
    # no covariance pairs at all
    assert f[20] == pytest.approx(0.0)
    assert f[21] == pytest.approx(0.0)
    assert f[22] == pytest.approx(math.log(1.0 / 4.0))
    assert np.all(f[23:] == 0.0) and f[17] == 0.0


def test_within_bin_variance_and_variance_of_bin_means():
    # bin 0: observations 1 and 3 (mean 2, spread 1); bin 1: one observation 5;
    # bin 2: empty
    m = (3,)
    W = np.array([2.0, 1.0, 0.0])
    V = np.array([4.0, 5.0, 0.0])
    V2 = np.array([10.0, 25.0, 0.0])
    cnt = np.array([2.0, 1.0, 0.0])
    Z = np.zeros((3, 3))
    f = of.features(1, m, np.array([1.0, 2.0]), cnt, W, V, V2, Z, Z, Z)
    assert f[10] == pytest.approx(math.log(0.5 + EPS))      # mean of (1, 0)
    assert f[11] == pytest.approx(math.log(2.25 + EPS))     # var of (2, 5)


@pytest.mark.parametrize("b", [0.5, -2.0])
def test_roughness_of_a_linear_mean_with_a_gap(b):
    # mb_j = 1 + b j on six bins, bin 2 empty: first differences exist only on
    # the pairs (0, 1), (3, 4), (4, 5), all equal to b; no second difference
    # window avoids the gap except (3, 4, 5), where it is 0
    m = (6,)
    j = np.arange(6.0)
    mb = 1.0 + b * j
    cnt, W, V, V2 = _flat_bins(mb)
    W[2] = cnt[2] = V[2] = V2[2] = 0.0
    Z = np.zeros((6, 6))
    f = of.features(1, m, np.array([3.0]), cnt, W, V, V2, Z, Z, Z)
    varmb = np.var(mb[[0, 1, 3, 4, 5]])
    assert f[11] == pytest.approx(math.log(varmb + EPS))
    assert f[15] == pytest.approx(math.log(b * b + EPS) - f[11])
    assert f[12] == pytest.approx(math.log(EPS) - f[11])
    assert f[13] == 0.0 and f[14] == 0.0 and f[16] == 0.0   # beyond d = 1


def test_roughness_of_a_quadratic_mean():
    m = (7,)
    j = np.arange(7.0)
    c = 0.3
    mb = c * j ** 2
    cnt, W, V, V2 = _flat_bins(mb)
    Z = np.zeros((7, 7))
    f = of.features(1, m, np.array([3.0]), cnt, W, V, V2, Z, Z, Z)
    # second differences are 2c everywhere; first differences c (2j + 1)
    assert f[12] == pytest.approx(math.log(4 * c * c + EPS) - f[11])
    r1 = np.mean((c * (2 * j[:-1] + 1)) ** 2)
    assert f[15] == pytest.approx(math.log(r1 + EPS) - f[11])


def test_roughness_per_axis_on_a_2d_grid():
    # mb(j0, j1) = alpha j0 + beta j1: first differences alpha along axis 0 and
    # beta along axis 1, second differences zero
    m = (4, 5)
    alpha, beta = 0.7, -0.2
    j0, j1 = np.meshgrid(np.arange(4.0), np.arange(5.0), indexing="ij")
    mb = alpha * j0 + beta * j1
    cnt, W, V, V2 = _flat_bins(mb)
    Z = np.zeros((20, 20))
    f = of.features(2, m, np.array([3.0]), cnt, W, V, V2, Z, Z, Z)
    assert f[15] == pytest.approx(math.log(alpha ** 2 + EPS) - f[11])
    assert f[16] == pytest.approx(math.log(beta ** 2 + EPS) - f[11])
    assert f[12] == pytest.approx(math.log(EPS) - f[11])
    assert f[13] == pytest.approx(math.log(EPS) - f[11])
    assert f[14] == 0.0 and f[17] == 0.0
    assert f[22] == pytest.approx(math.log(0.25)) and f[23] == pytest.approx(math.log(0.2))
    assert f[24] == 0.0 and np.all(f[25:] == 0.0)


def test_covariance_roughness_along_s1_and_the_diagonal_1d():
    # g(s, t) = a s + b t on a 1-D grid: steps of a along s, a + b along the
    # diagonal; g(s, t) = phi(s - t) is constant along the diagonal
    M = 6
    s, t = np.meshgrid(np.arange(M, dtype=float), np.arange(M, dtype=float), indexing="ij")
    a, b = 0.4, 1.1
    g = a * s + b * t
    C, Wc, Vc = _cov_bins(g)
    cnt, W, V, V2 = _flat_bins(np.zeros(M))
    f = of.features(1, (M,), np.array([2.0]), cnt, W, V, V2, C, Wc, Vc)
    lvg = math.log(np.var(g) + EPS)
    assert f[18] == pytest.approx(math.log(a * a + EPS) - lvg)
    assert f[19] == pytest.approx(math.log((a + b) ** 2 + EPS) - lvg)
    g2 = np.cos(s - t)
    C, Wc, Vc = _cov_bins(g2)
    f = of.features(1, (M,), np.array([2.0]), cnt, W, V, V2, C, Wc, Vc)
    assert f[19] == pytest.approx(math.log(EPS) - math.log(np.var(g2) + EPS))
    assert f[20] == pytest.approx(math.log(2.0))    # one pair per bin
    assert f[21] == pytest.approx(1.0)


def test_covariance_roughness_uses_the_first_axis_step_2d():
    # on a 3 x 4 grid, g depends only on the second coordinate of s: it is
    # constant along s_1, so that roughness is zero; a flat step of 1 (the
    # second axis) would see the variation instead
    m = (3, 4)
    P = 12
    s_idx = np.arange(P)
    s2 = s_idx % 4
    g = np.repeat((0.5 * s2 ** 2)[:, None], P, axis=1) + np.arange(P)[None, :] * 0.0
    C, Wc, Vc = _cov_bins(g)
    cnt, W, V, V2 = _flat_bins(np.zeros(P))
    f = of.features(2, m, np.array([2.0]), cnt, W, V, V2, C, Wc, Vc)
    lvg = math.log(np.var(g) + EPS)
    assert f[18] == pytest.approx(math.log(EPS) - lvg)
    # and a surface varying along s_1 by a per step is seen with a^2
    s1 = s_idx // 4
    g1 = np.repeat((0.3 * s1)[:, None], P, axis=1)
    C, Wc, Vc = _cov_bins(g1)
    f = of.features(2, m, np.array([2.0]), cnt, W, V, V2, C, Wc, Vc)
    assert f[18] == pytest.approx(math.log(0.09 + EPS) - math.log(np.var(g1) + EPS))


def test_empty_covariance_bins_are_skipped():
    # a step between two non-empty bins is counted only when both ends have pairs
    M = 4
    g = np.zeros((M, M))
    g[1, :] = 3.0
    Wc = np.ones((M, M))
    Wc[1, 0] = 0.0             # the (0,0)-(1,0) and (1,0)-(2,0) steps drop out
    Vc = g * Wc
    C = Wc.copy()
    cnt, W, V, V2 = _flat_bins(np.zeros(M))
    f = of.features(1, (M,), np.array([2.0]), cnt, W, V, V2, C, Wc, Vc)
    ok = Wc > 0
    gv = np.where(ok, g, 0.0)
    steps = [(gv[i + 1, j] - gv[i, j]) ** 2 for i in range(M - 1) for j in range(M)
             if ok[i + 1, j] and ok[i, j]]
    lvg = math.log(np.var(gv[ok]) + EPS)
    assert len(steps) == 3 * M - 2
    assert f[18] == pytest.approx(math.log(np.mean(steps) + EPS) - lvg)
    assert f[21] == pytest.approx((M * M - 1) / (M * M))
