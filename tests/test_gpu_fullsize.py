"""Parity at the workloads' full sizes, against the FP64 oracle.

* 64 x 64 disk grid, n = 1000 (the benchmark's workload and launch
  configuration: BF16 tensor-core binning, compensated FP32 moments): the
  oracle's whole surface Gamma_hat (oracle/grid.py, 16.8M points) gives the
  random-projection eigenpairs with the same Omega and the noise variance of
  Eq. (2.5)-(2.6); the GPU's must agree within the BF16-binning tolerances.
* Sparse longitudinal workload, n = 20 000 subjects, 64 x 64 bins, 5 folds:
  the fits on the training bins of a fold at h = 0.03, 0.15, 0.3 (3 to 39
  taps each side) against the oracle's per-point fits at sampled output
  pairs, and the GPU's CV score against the score written out from the GPU's
  own fitted surfaces and the oracle's bins.

These take minutes of CPU time for the oracle (marked slow).
"""
import math

import numpy as np
import pytest

import fpca_synth as fs
from oracle import eigen as oe
from oracle import grid as og
from oracle import smoother as sm
from oracle import variance as ov
from parity_helpers import assert_status_band

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = "cuda:0"


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_dense_64x64_eigenpairs_and_noise_variance_vs_oracle():
    from paper_1510_04439_gb300 import binding as B
    from paper_1510_04439_gb300 import pipeline
    ctx = B.Context(0)
    D = fs.dense_2d_disk()
    h = (0.15, 0.15)
    k, l, q = 8, 18, 2
    om = fs.gaussian_test_matrix(D.P, l, fs.SEED_BASE)
    bufs = pipeline.alloc_dense(torch, torch.device(DEV), D.P, k, B.BF16, B.F32)
    pipeline.run_dense(ctx, D.m, dev(D.y, torch.float32), dev(D.mask), h, h, k, bufs,
                       bin_prec=B.BF16, smooth_prec=B.F32C, omega=dev(om, torch.float32),
                       power_iters=q)
    sig_t = torch.empty(D.P, dtype=torch.float64, device=DEV)
    s2 = torch.empty(1, dtype=torch.float64, device=DEV)
    ctx.sigma2(D.m, bufs.cnt, bufs.w, bufs.v2, h, bufs.mu, bufs.gamma.reshape(-1), D.P + 1,
               sig_t, None, s2, domain=bufs.cnt)
    ctx.sync()
    # the oracle on the same (FP32-rounded) observations
    y = D.y.astype(np.float32).astype(np.float64)
    cnt, Wm, Vm, V2m = sm.bin_mean_dense(y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h, cnt, Wm, Vm)
    mu0 = np.where(np.isnan(mu), 0.0, mu)
    C, W, V = sm.bin_cov_dense(sm.residuals_dense(y, D.mask, mu0), D.mask)
    S, T = og.moments(D.m, h, W, V)
    ne = og.nonempty(D.m, h, C)
    P = D.P
    G, st = og.fit_pairs(S, T, ne, 2, np.repeat(np.arange(P), P), np.tile(np.arange(P), P))
    G = G.reshape(P, P)
    del S, T
    dom = cnt > 0
    # eigenpairs: the same range finder with the same Omega on the oracle's surface
    lam, phi, fve = oe.rproj_eig(G, D.m, dom, om, k, q)
    glam = bufs.evals.cpu().numpy()
    gphi = bufs.evecs.cpu().numpy().T
    assert np.allclose(glam, lam, rtol=1e-2), (glam, lam)
    for j in range(k):   # lambda_j = 8 2^(1-j): every gap is half the eigenvalue
        assert oe.subspace_angle(gphi[:, j:j + 1], phi[:, j:j + 1]) <= 5e-2, j
    assert oe.subspace_angle(gphi, phi) <= 5e-2
    assert np.allclose(bufs.fve.cpu().numpy(), fve, rtol=1e-2)
    # noise variance: b0 of the squared observations minus the surface's diagonal
    rsig, _ = ov.sigma2_curve(D.m, h, cnt, Wm, V2m, mu, np.diag(G))
    rs2 = ov.sigma2_scalar(rsig, dom)
    gs2 = float(s2.item())
    assert math.isclose(gs2, rs2, rel_tol=2e-2), (gs2, rs2)
    # the estimate is far above the true 0.25 on both sides: the local linear
    # surface is biased low on its diagonal at h = 0.15 on this workload
    assert rs2 > 1.0


@pytest.mark.parametrize("hh,npts", [(0.03, 300), (0.15, 300), (0.3, 120)])
def test_sparse_64x64_fold_fits_and_cv_vs_oracle(hh, npts):
    from paper_1510_04439_gb300 import binding as B
    ctx = B.Context(0)
    D = fs.sparse_2d()
    m, P, F = D.m, D.P, D.nfold
    hmu = (0.1, 0.1)
    data = ctx.sparse(dev(D.offs), dev(D.t), dev(D.y))
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(2))
    ctx.bin_mean(data, m, cnt, w, v)
    mu = torch.empty(P, dtype=torch.float64, device=DEV)
    ctx.smooth_mean(m, cnt, w, v, hmu, mu)
    Cg = torch.empty(F, P, P, dtype=torch.int32, device=DEV)
    Wg, Vg, Qg = (torch.empty(F, P, P, dtype=torch.float32, device=DEV) for _ in range(3))
    ctx.bin_cov(data, m, mu, B.F32, Cg, Wg, Vg, q=Qg, fold=dev(D.fold), nfold=F)
    cvg = torch.empty(1, dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(m, Cg, Wg, Vg, [(hh, hh)], B.F32C, q=Qg, nfold=F, cv=cvg)
    ctx.sync()
    # the oracle's bins from the data
    rc, rw, rv, _ = sm.bin_mean_sparse(D.offs, D.t, D.y, m)
    rmu, _ = sm.smooth_mean(m, hmu, rc, rw, rv)
    assert np.allclose(mu.cpu().numpy(), rmu, rtol=1e-10, atol=1e-12)
    r = sm.residuals_sparse(D.t, D.y, rmu, m)
    C, W, V, Q = og.bin_cov_sparse_pairs(D.offs, D.t, r, m, D.fold, F)
    assert np.array_equal(Cg.cpu().numpy(), C), "pair counts must be bit-exact"
    rng = np.random.default_rng(int(hh * 1000))
    err = win = wout = 0.0
    for f in range(F):
        # the GPU's fit on the training bins of fold f (pooled minus fold f)
        Ct = (Cg.sum(0) - Cg[f]).to(torch.int32)   # torch sums int32 into int64
        Wt, Vt = (x.sum(0) - x[f] for x in (Wg, Vg))
        Gf = torch.empty(P, P, dtype=torch.float32, device=DEV)
        sf = torch.empty(P, P, dtype=torch.uint8, device=DEV)
        ctx.smooth_cov_project(m, Ct, Wt, Vt, [(hh, hh)], B.F32C, gamma=Gf, status=sf)
        ctx.sync()
        g = Gf.cpu().numpy().astype(np.float64)
        s = sf.cpu().numpy()
        # CV terms of fold f written out from the GPU surface and the oracle's bins
        inc = s != sm.STATUS_EMPTY
        gz = np.where(inc, g, 0.0)
        e = Q[f] - 2.0 * gz * V[f] + gz * gz * W[f]
        err += float(np.sum(e[inc]))
        win += float(np.sum(W[f][inc]))
        wout += float(np.sum(W[f][~inc]))
        if f >= 2:
            continue   # the oracle's per-point fits on folds 0 and 1
        Ctr, Wtr, Vtr = C.sum(0) - C[f], W.sum(0) - W[f], V.sum(0) - V[f]
        inside = np.nonzero(rc > 0)[0]
        pairs = np.stack([rng.choice(P, npts), rng.choice(P, npts)], 1)
        pairs[: npts // 2] = np.stack([rng.choice(inside, npts // 2),
                                       rng.choice(inside, npts // 2)], 1)
        pairs = np.concatenate([pairs, [[0, 0], [P - 1, P - 1], [0, P - 1], [P // 2, P // 2]]])
        ref, rst = sm.smooth_cov_points(pairs, m, (hh, hh), Ctr, Wtr, Vtr)
        gs = g[pairs[:, 0], pairs[:, 1]]
        ss = s[pairs[:, 0], pairs[:, 1]]
        # sparse windows (h = 0.03: 3 x 3 bins each side, ~16% of bin pairs hold a
        # pair) often give near-singular systems: every status mismatch must lie in
        # the pivot band FP32 moments cannot decide
        nbad = assert_status_band(ss, rst, pairs, m, (hh, hh), Ctr, Wtr, Vtr)
        assert nbad <= len(pairs) // 2
        ok = (rst == sm.STATUS_OK) & (ss == sm.STATUS_OK)
        assert ok.sum() > npts // 4
        assert rel_l2(gs[ok], ref[ok]) <= 1e-5
        fb = (rst == sm.STATUS_FALLBACK) & (ss == sm.STATUS_FALLBACK)
        if fb.any():
            assert rel_l2(gs[fb], ref[fb]) <= 1e-5
        assert np.array_equal(np.isnan(gs), rst == sm.STATUS_EMPTY)
    ref_cv = math.inf if (wout > 0.01 * (win + wout) or win <= 0.0) else err / win
    got = float(cvg.item())
    if math.isinf(ref_cv):
        assert math.isinf(got)
    else:
        assert math.isclose(got, ref_cv, rel_tol=1e-4), (got, ref_cv)
