"""Pins of the block/row form of the covariance smoother (oracle/block.py).

The block form evaluates the binned estimator of Eq. (2.4) from the data at
chosen output pairs.  It is pinned to the whole-grid form of oracle/smoother.py
(itself pinned to affine reproduction, brute-force unbinned fits and symmetry in
test_oracle_pins.py) on grids small enough to hold all P x P bins, masked and
fully observed, d = 2 and 3; and the stacked solve is pinned to the per-point one.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import block as ob
from oracle import smoother as sm


def test_solve_points_matches_solve_point():
    rng = np.random.default_rng(5)
    D = 7
    As, rs, ns = [], [], []
    for k in range(200):
        X = rng.standard_normal((D + 3, D))
        A = X.T @ X
        kind = k % 5
        if kind == 1:
            A[:, 3] = A[:, 2]          # exactly singular
            A[3, :] = A[2, :]
        elif kind == 2:
            A[0, 0] = 0.0              # empty window
        elif kind == 3:
            A[4, 4] = A[4, 4] * 1e-12 + 1e-14   # tiny pivot
        As.append(A)
        rs.append(rng.standard_normal(D))
        ns.append(3 if kind == 4 else 50)
    val, st = ob.solve_points(np.array(As), np.array(rs), np.array(ns))
    for A, r, n, v, s in zip(As, rs, ns, val, st):
        v0, s0 = sm.solve_point(A, r, n)
        assert s == s0
        if np.isnan(v0):
            assert np.isnan(v)
        else:
            assert abs(v - v0) <= 1e-9 * max(1.0, abs(v0))


def _grid_reference(D, h):
    cnt, W, V, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h, cnt, W, V)
    mu0 = np.where(np.isnan(mu), 0.0, mu)
    r = sm.residuals_dense(D.y, D.mask, mu0)
    C, Wc, Vc = sm.bin_cov_dense(r, D.mask)
    G, st = sm.smooth_cov_grid(D.m, h, C, Wc, Vc)
    return mu0, G, st


def _box_flat(lo, hi, m):
    axes = [np.arange(a, b) for a, b in zip(lo, hi)]
    g = np.meshgrid(*axes, indexing="ij")
    flat = np.zeros(g[0].size, dtype=np.int64)
    for k in range(len(m)):
        flat = flat * m[k] + g[k].ravel()
    return flat


@pytest.mark.parametrize("case", ["d2_masked", "d3_full", "d3_masked_narrow"])
def test_block_matches_whole_grid(case):
    if case == "d2_masked":
        D = fs.make_dense(2, (7, 6), 30, [2.0, 1.0], sigma=0.4, seed=11, dropout=0.3)
        h = np.array([0.35, 0.5])
        boxes = [((0, 0), (3, 2), (2, 1), (7, 6)), ((4, 3), (7, 6), (0, 0), (3, 4))]
    elif case == "d3_full":
        D = fs.make_dense(3, (5, 4, 4), 20, [2.0, 1.0], sigma=0.3, mean="exp", seed=12)
        h = np.array([0.5, 0.6, 0.6])
        boxes = [((0, 0, 0), (2, 2, 4), (1, 0, 0), (4, 4, 3)), ((3, 1, 2), (5, 4, 4), (0, 0, 0), (5, 4, 4))]
    else:
        D = fs.make_dense(3, (4, 4, 5), 15, [2.0, 1.0], sigma=0.3, mean="exp", seed=13, dropout=0.4)
        h = np.array([0.3, 0.3, 0.18])      # one-node windows on the last axis: FALLBACK occurs
        boxes = [((0, 0, 0), (4, 4, 5), (0, 0, 0), (4, 4, 5))]
    m = D.m
    mu0, G, st = _grid_reference(D, h)
    seen = set()
    for slo, shi, tlo, thi in boxes:
        S = _box_flat(slo, shi, m)
        T = _box_flat(tlo, thi, m)
        val, stb = ob.smooth_cov_block(D.y, D.mask, mu0, m, h, S, tlo, thi)
        ref, rst = G[np.ix_(S, T)], st[np.ix_(S, T)]
        assert np.array_equal(stb, rst)
        ok = rst != sm.STATUS_EMPTY
        assert np.allclose(val[ok], ref[ok], rtol=1e-10, atol=1e-12 * np.abs(ref[ok]).max())
        assert np.all(np.isnan(val[~ok]))
        seen |= set(np.unique(rst).tolist())
    if case == "d3_masked_narrow":
        assert sm.STATUS_FALLBACK in seen


def test_rows_symmetric_d3():
    D = fs.make_dense(3, (6, 5, 4), 25, [2.0, 1.0, 0.5], sigma=0.3, mean="exp", seed=14)
    h = np.array([0.4, 0.45, 0.6])
    cnt, W, V, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h, cnt, W, V)
    rows = np.array([0, 37, 119])
    G, st = ob.smooth_cov_rows(D.y, None, mu, D.m, h, rows)
    Gt, _ = ob.smooth_cov_rows(D.y, None, mu, D.m, h, np.arange(D.P))
    assert np.allclose(G, Gt[rows], rtol=1e-12, atol=0)
    assert np.allclose(Gt, Gt.T, rtol=1e-10, atol=1e-13 * np.abs(Gt).max())
    assert np.all(st == sm.STATUS_OK)
