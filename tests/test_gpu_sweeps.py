"""The two t-side sweeps of the FP32 d = 2 covariance smoother against the oracle.

fpca_smooth_cov_project (FPCA_F32 / FPCA_F32C) evaluates the t-side of the moment
sums either with the scalar sweep (every grid and window) or with the packed-pair
sweep (t-planes 32 or 64 wide, the same half-width on both t axes, up to 39
taps), and by default times both once per grid and window and keeps the faster.
Each choice is compared element by element with the FP64 oracle
(oracle/grid.py, pinned to the per-point smoother) on grids that leave a ragged
last block of t1-rows, from 7 to 39 taps, in the t >= s half mode (symmetric
bins, mirrored), with the fused projection y = Gamma_hat Omega (every pair
fitted) and with the K-fold CV epilogue.

The K-fold CV grid also runs batched: every (bandwidth, fold) item's s-side
arrays first, then one persistent t-side launch over all items' tiles; its
scores are compared with the oracle and with the item-by-item path.

Tolerances: FP32 moments rel-L2 <= 1e-5 on points both sides fit with the full
local linear model; statuses equal outside the pivot band (assert_status_band);
CV score rel 1e-4 with the same argmin; y rel-L2 <= 1e-5.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import cv as ocv
from oracle import grid as og
from oracle import smoother as sm
from parity_helpers import assert_status_band, grid_pairs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_1510_04439_gb300 import binding
    return binding


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def same_taps_h(m, T):
    """Bandwidths with exactly T taps each side on every axis: T < h M <= T + 1."""
    return tuple((T + 0.5) / mk for mk in m)


def dense_bins(m, n, seed):
    D = fs.make_dense(2, m, n, [2.0, 1.0, 0.5], sigma=0.3, seed=seed, dropout=0.2, domain="disk")
    cnt, Wm, Vm, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, (0.2, 0.2), cnt, Wm, Vm)
    mu = np.where(np.isnan(mu), 0.0, mu)
    return sm.bin_cov_dense(sm.residuals_dense(D.y, D.mask, mu), D.mask)


@pytest.mark.parametrize("m,T", [((21, 32), 3), ((21, 32), 12), ((11, 64), 9), ((9, 64), 5),
                                 ((20, 64), 19)])
def test_sweeps_vs_oracle(B, m, T):
    ctx = B.Context(0)
    h = same_taps_h(m, T)
    C, W, V = dense_bins(m, 60, seed=m[0] * 100 + T)
    P = m[0] * m[1]
    rG, rst = og.smooth_cov(m, h, C, W, V)
    results = {}
    for kern in (1, 2, 0):
        ctx.set_sweep_kernel(kern)
        for prec in (B.F32, B.F32C):
            G = torch.empty(P, P, dtype=torch.float32, device=DEV)
            st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
            ctx.smooth_cov_project(m, dev(C, torch.int32), dev(W, torch.float32),
                                   dev(V, torch.float32), [h], prec, gamma=G, status=st)
            ctx.sync()
            g = G.cpu().numpy().astype(np.float64)
            s = st.cpu().numpy()
            assert_status_band(s, rst, grid_pairs(P), m, h, C, W, V, max_mismatch=P * P // 1000)
            ok = (rst == sm.STATUS_OK) & (s == sm.STATUS_OK)
            assert rel_l2(g[ok], rG[ok]) <= 1e-5, (kern, prec)
            fb = (rst == sm.STATUS_FALLBACK) & (s == sm.STATUS_FALLBACK)
            if fb.any():
                assert rel_l2(g[fb], rG[fb]) <= 1e-5
            assert np.array_equal(np.isnan(g), rst == sm.STATUS_EMPTY)
            results[(kern, prec)] = (g, s)
    # the two sweeps add the same terms in different groupings: equal statuses
    # outside the band, values within the FP32 tolerance of each other
    for prec in (B.F32, B.F32C):
        g1, s1 = results[(1, prec)]
        g2, s2 = results[(2, prec)]
        ok = (s1 == sm.STATUS_OK) & (s2 == sm.STATUS_OK)
        assert np.mean(s1 == s2) > 0.999
        assert rel_l2(g2[ok], g1[ok]) <= 1e-5


def pivot_ratios(m, h, W, V, ne):
    """Smallest Cholesky pivot ratio (Schur-complement diagonal over the original
    diagonal, natural order) of every output pair's (2d+1)^2 system, from the FP64
    moments; 0 where a pivot is not positive, NaN where the window is empty or has
    fewer than 2d+1 non-empty bins (those are not solved)."""
    d = len(m)
    D = 2 * d + 1
    S, _ = og.moments(m, h, W, V)
    unit = [tuple(int(j > 0 and k == j - 1) for k in range(2 * d)) for j in range(D)]
    P = S[(0,) * (2 * d)].shape[0]
    A = np.empty((P * P, D, D))
    for i in range(D):
        for j in range(D):
            A[:, i, j] = S[tuple(a + b for a, b in zip(unit[i], unit[j]))].ravel()
    diag = np.einsum("nii->ni", A).copy()
    ratio = np.full(P * P, np.inf)
    live = np.ones(P * P, dtype=bool)
    for k in range(D):
        piv = A[:, k, k]
        with np.errstate(divide="ignore", invalid="ignore"):
            rk = np.where(diag[:, k] > 0, piv / diag[:, k], 0.0)
        ratio = np.where(live, np.minimum(ratio, rk), ratio)
        live &= piv > 0
        safe = np.where(piv > 0, piv, 1.0)
        for i in range(k + 1, D):
            lik = A[:, i, k] / safe
            A[:, i, k + 1:] -= lik[:, None] * A[:, k, k + 1:]
    ratio[~live] = 0.0
    ratio[(diag[:, 0] <= 0) | (ne.ravel() < D)] = np.nan
    return ratio.reshape(P, P)


def test_escalated_points_vs_fp64(B):
    """The points whose FP32 elimination meets a pivot below 1e-2 of its diagonal are
    solved again in float-float (about 48 bits) rather than FP64.  Their inputs are
    the FP32 moments, rounded to about u = 2^-24 of their scale, so the fitted value
    moves by about u times the system's conditioning, which the smallest pivot ratio
    r bounds (kappa ~ 1/r); the float-float rounding (~2^-48 kappa) is 2^24 times
    smaller, so an FP64 solve of the same moments would give the same values to that
    order.  Checked against the FP64 oracle (FP64 moments, FP64 solve) on a disk grid
    with 20 % dropout, where the one-sided windows at the rim give small ratios: per
    band of r, the rel-L2 error on points both sides fit stays within
    64 u / r_low (r_low the band's lower edge), the points with r >= 1e-2 (FP32 solve
    only) within 64 u / 1e-2."""
    ctx = B.Context(0)
    m = (32, 32)
    h = same_taps_h(m, 4)
    C, W, V = dense_bins(m, 60, seed=77)
    P = m[0] * m[1]
    rG, rst = og.smooth_cov(m, h, C, W, V)
    ratio = pivot_ratios(m, h, W, V, og.nonempty(m, h, C))
    G = torch.empty(P, P, dtype=torch.float32, device=DEV)
    st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
    ctx.smooth_cov_project(m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32),
                           [h], B.F32C, gamma=G, status=st)
    ctx.sync()
    g = G.cpu().numpy().astype(np.float64)
    s = st.cpu().numpy()
    both = (rst == sm.STATUS_OK) & (s == sm.STATUS_OK)
    u = 2.0 ** -24
    report = {}
    for lo, hi in [(1e-2, np.inf), (1e-3, 1e-2), (1e-4, 1e-3), (1e-5, 1e-4)]:
        sel = both & (ratio >= lo) & (ratio < hi)
        if not sel.any():
            continue
        err = rel_l2(g[sel], rG[sel])
        worst = float(np.max(np.abs(g[sel] - rG[sel])) / np.max(np.abs(rG[sel])))
        report[lo] = (int(sel.sum()), err, worst)
        assert err <= 64 * u / lo, (lo, report)
    print("escalation bands (r_low: points, rel-L2, max |err| / max |Gamma|):", report)
    assert sum(v[0] for lo, v in report.items() if lo < 1e-2) >= 1000, report


@pytest.mark.parametrize("kern", [1, 2])
def test_sweeps_projection_epilogue(B, kern):
    """y = Gamma_hat Omega fused into the sweep (every pair fitted, no mirror)."""
    ctx = B.Context(0)
    ctx.set_sweep_kernel(kern)
    m, T, l = (13, 64), 7, 18
    h = same_taps_h(m, T)
    C, W, V = dense_bins(m, 50, seed=5)
    P = m[0] * m[1]
    om = fs.gaussian_test_matrix(P, l, 3).astype(np.float32)
    y = torch.empty(P, l, dtype=torch.float32, device=DEV)
    G = torch.empty(P, P, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_project(m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32),
                           [h], B.F32C, omega=dev(om), y=y, gamma=G)
    ctx.sync()
    rG, rst = og.smooth_cov(m, h, C, W, V)
    ref = np.where(np.isnan(rG), 0.0, rG) @ om.astype(np.float64)
    assert rel_l2(y.cpu().numpy().astype(np.float64), ref) <= 1e-5
    # y is the product of the surface the same call wrote
    g = np.nan_to_num(G.cpu().numpy().astype(np.float64))
    assert rel_l2(y.cpu().numpy().astype(np.float64), g @ om.astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("kern,batch", [(1, False), (2, False), (0, True)])
def test_sweeps_cv_epilogue(B, kern, batch):
    """K-fold CV scores through either sweep, item by item or as one batched
    launch over the whole (bandwidth, fold) grid, against the oracle's CV."""
    ctx = B.Context(0)
    ctx.set_sweep_kernel(kern)
    ctx.set_cv_batch(batch)
    m = (16, 32)
    D = fs.make_sparse(2, m, 3000, [2.0, 1.0], nmin=5, nmax=20, sigma=0.5, seed=12, nfold=5)
    mu = np.linspace(-0.2, 0.3, D.P)
    r = sm.residuals_sparse(D.t, D.y, mu, m)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, m, D.fold, 5)
    Ts = [2, 4, 8]
    hs = [same_taps_h(m, T) for T in Ts]
    cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32),
                           hs, B.F32C, q=dev(Q, torch.float32), nfold=5, cv=cv)
    ctx.sync()
    ref = np.array([ocv.cv_score(m, list(h), C, W, V, Q, smooth=og.smooth_cov) for h in hs])
    got = cv.cpu().numpy()
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=1e-4)
    assert np.argmin(np.where(fin, got, np.inf)) == np.argmin(np.where(fin, ref, np.inf))


def test_sweep_choice_is_remembered(B):
    """Automatic mode times both sweeps once per grid and window: the second call
    launches no timing runs."""
    ctx = B.Context(0)
    m, T = (16, 64), 9
    h = same_taps_h(m, T)
    C, W, V = dense_bins(m, 30, seed=9)
    P = m[0] * m[1]
    G = torch.empty(P, P, dtype=torch.float32, device=DEV)
    args = (m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32), [h], B.F32C)
    l0 = ctx.launches
    ctx.smooth_cov_project(*args, gamma=G)
    first = ctx.launches - l0
    ctx.sync()
    g1 = G.clone()
    l0 = ctx.launches
    ctx.smooth_cov_project(*args, gamma=G)
    second = ctx.launches - l0
    ctx.sync()
    assert first == second + 4      # two timing runs of each sweep, once
    assert torch.equal(G, g1)       # the remembered choice gives the same surface


@pytest.mark.parametrize("m,comp", [((16, 64), True), ((21, 32), False), ((12, 16), True)])
def test_cv_grid_batched_matches_items_and_oracle(B, m, comp):
    """One launch over the whole CV grid (bandwidths of different windows on each
    axis, so the items' tiles differ in shape) gives the item-by-item scores and
    the oracle's; the grid kernel runs once, the per-item sweeps not at all."""
    K = 4
    D = fs.make_sparse(2, m, 2500, [2.0, 1.0], nmin=6, nmax=18, sigma=0.5, seed=31, nfold=K)
    mu = np.linspace(-0.1, 0.2, D.P)
    r = sm.residuals_sparse(D.t, D.y, mu, m)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, m, D.fold, K)
    taps = [(2, 5), (4, 3), (3, 9), (6, 6)] if m[1] < 64 else [(2, 5), (3, 9)]
    hs = [((T1 + 0.5) / m[0], (T2 + 0.5) / m[1]) for T1, T2 in taps]
    prec = B.F32C if comp else B.F32
    args = (m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32), hs, prec)
    out = {}
    for batch in (True, False):
        ctx = B.Context(0)
        ctx.set_sweep_kernel(1)
        ctx.set_cv_batch(batch)
        cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
        ctx.profile(True)
        ctx.smooth_cov_project(*args, q=dev(Q, torch.float32), nfold=K, cv=cv)
        ctx.sync()
        out[batch] = (cv.cpu().numpy(), ctx.profile_read())
    (cb, pb), (ci, pi) = out[True], out[False]
    assert pb["cov_cv_grid"][1] == 1 and "cov_hpass_solve" not in pb
    assert "cov_cv_grid" not in pi and pi["cov_hpass_solve"][1] == len(hs) * K
    ref = np.array([ocv.cv_score(m, list(h), C, W, V, Q, smooth=og.smooth_cov) for h in hs])
    fin = np.isfinite(ref)
    for got in (cb, ci):
        assert np.array_equal(np.isfinite(got), fin)
        assert np.allclose(got[fin], ref[fin], rtol=1e-4)
    # the same sums per point: batched and item-by-item agree far inside the tolerance
    assert np.allclose(cb[fin], ci[fin], rtol=1e-6)


def test_cv_schedule_choice_is_remembered(B):
    """Automatic CV schedule: the first call runs the grid item by item, then times
    the batched and the item-by-item schedule; later calls run only the one kept,
    with the same scores."""
    K = 5
    m = (16, 32)
    D = fs.make_sparse(2, m, 1500, [2.0, 1.0], nmin=6, nmax=18, sigma=0.5, seed=7, nfold=K)
    mu = np.zeros(D.P)
    r = sm.residuals_sparse(D.t, D.y, mu, m)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, m, D.fold, K)
    hs = [((T + 0.5) / m[0], (T + 0.5) / m[1]) for T in (2, 3, 5)]
    ctx = B.Context(0)
    args = (m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32), hs, B.F32C)
    out = []
    for _ in range(3):
        cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
        l0 = ctx.launches
        ctx.smooth_cov_project(*args, q=dev(Q, torch.float32), nfold=K, cv=cv)
        ctx.sync()
        out.append((ctx.launches - l0, cv.cpu().numpy()))
    (n1, c1), (n2, c2), (n3, c3) = out
    assert n2 == n3 and n1 > 2 * n2          # three schedules' worth of launches, once
    # (the FP64 atomic sums of the CV terms may add in another order)
    assert np.allclose(c2, c1, rtol=1e-6) and np.allclose(c2, c3, rtol=1e-12)
