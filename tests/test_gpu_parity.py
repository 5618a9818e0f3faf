"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated per result):
  counts                          bit-exact
  FP64 path (bins, mean, Gamma)   rel-L2 <= 1e-6 (observed ~1e-13)
  FP32 moments (+ FP32/FP64 solve) rel-L2 <= 1e-5 on OK points
  BF16 binning products            W elementwise rel <= 2^-8, V rel-L2 <= 5e-3,
                                   Gamma_hat rel-L2 <= 5e-3
  random projection (FP32 Sigma)   lambda rel <= 1e-4, subspace angle <= 1e-3 rad
  dense eigensolver (FP64)         lambda rel <= 1e-10, subspace angle <= 1e-8 rad
Statuses: FP64 paths must equal the oracle's everywhere.  An FP32 path may
differ only at points whose oracle pivot ratio lies in the band where FP32
moments cannot decide the status ([1e-10, 1e-3], BAND); every mismatch is
checked against that band (assert_status_band), and values are compared where
both sides fitted the full local linear model.
"""
import math

import numpy as np
import pytest

import fpca_synth as fs
from oracle import eigen as oe
from oracle import smoother as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    from paper_1510_04439_gb300 import binding as B
    return B.Context(0)


@pytest.fixture(scope="module")
def B():
    from paper_1510_04439_gb300 import binding
    return binding


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


from parity_helpers import BAND, assert_status_band, grid_pairs, oracle_ratio  # noqa: E402,F401


# ----------------------------------------------------------------------------
# mean bins and mean smoother
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("y32", [False, True])
def test_mean_bins_dense(ctx, y32):
    D = fs.dense_2d_disk(n=120, m=32)
    y = D.y.astype(np.float32) if y32 else D.y
    P = D.P
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v, v2 = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(3))
    ctx.bin_mean(ctx.dense(dev(y), dev(D.mask)), D.m, cnt, w, v, v2)
    ctx.sync()
    rc, rw, rv, rv2 = sm.bin_mean_dense(y.astype(np.float64), D.mask, D.m)
    assert np.array_equal(host(cnt), rc)
    for a, b in ((w, rw), (v, rv), (v2, rv2)):
        assert np.allclose(host(a), b, rtol=1e-13, atol=1e-13)


def test_mean_bins_sparse(ctx):
    D = fs.make_sparse(2, (16, 16), 300, [2.0, 1.0], nmin=1, nmax=12, seed=5, nfold=0)
    P = D.P
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v, v2 = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(3))
    ctx.bin_mean(ctx.sparse(dev(D.offs), dev(D.t), dev(D.y)), D.m, cnt, w, v, v2)
    ctx.sync()
    rc, rw, rv, rv2 = sm.bin_mean_sparse(D.offs, D.t, D.y, D.m)
    assert np.array_equal(host(cnt), rc)
    for a, b in ((w, rw), (v, rv), (v2, rv2)):
        assert np.allclose(host(a), b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,h", [((50,), (0.07,)), ((32, 32), (0.15, 0.1)), ((8, 8, 8), (0.3, 0.3, 0.3)),
                                 ((20, 20), (0.02, 0.02)), ((12, 10), (0.9, 1.5))])
def test_smooth_mean(ctx, m, h):
    rng = np.random.default_rng(len(m) * 100 + m[0])
    P = int(np.prod(m))
    cnt = rng.integers(0, 3, size=P).astype(np.int32)
    W = np.where(cnt > 0, rng.random(P) + 0.1, 0.0)
    V = W * rng.standard_normal(P)
    mu = torch.empty(P, dtype=torch.float64, device=DEV)
    st = torch.empty(P, dtype=torch.uint8, device=DEV)
    ctx.smooth_mean(m, dev(cnt), dev(W), dev(V), h, mu, st)
    ctx.sync()
    rmu, rst = sm.smooth_mean(m, h, cnt.astype(np.int64), W, V)
    assert np.array_equal(host(st), rst)
    ok = rst != sm.STATUS_EMPTY
    assert np.allclose(host(mu)[ok], rmu[ok], rtol=1e-10, atol=1e-11)
    assert np.all(np.isnan(host(mu)[~ok]))


# ----------------------------------------------------------------------------
# covariance bins
# ----------------------------------------------------------------------------

def test_cov_bins_dense_f64(ctx, B):
    D = fs.dense_2d_disk(n=37, m=16)
    P = D.P
    mu = sm.smooth_mean(D.m, (0.2, 0.2), *sm.bin_mean_dense(D.y, D.mask, D.m)[:3])[0]
    mu = np.where(np.isnan(mu), 0.0, mu)
    C = torch.empty(P, P, dtype=torch.int32, device=DEV)
    W = torch.empty(P, P, dtype=torch.float64, device=DEV)
    V = torch.empty(P, P, dtype=torch.float64, device=DEV)
    ctx.bin_cov(ctx.dense(dev(D.y), dev(D.mask)), D.m, dev(mu), B.F64, C, W, V)
    ctx.sync()
    rC, rW, rV = sm.bin_cov_dense(sm.residuals_dense(D.y, D.mask, mu), D.mask)
    assert np.array_equal(host(C), rC)
    assert np.allclose(host(W), rW, rtol=1e-12, atol=1e-16)
    assert np.allclose(host(V), rV, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m,n", [((8, 16), 3), ((16, 24), 70), ((32, 32), 129)])
def test_cov_bins_dense_bf16_tensor_core(ctx, B, m, n):
    D = fs.make_dense(2, m, n, [3.0, 1.0, 0.5], sigma=0.4, seed=n, domain="disk", dropout=0.15)
    P = D.P
    mu = np.zeros(P)
    C = torch.empty(P, P, dtype=torch.int32, device=DEV)
    W = torch.empty(P, P, dtype=torch.float32, device=DEV)
    V = torch.empty(P, P, dtype=torch.float32, device=DEV)
    ctx.bin_cov(ctx.dense(dev(D.y), dev(D.mask)), D.m, dev(mu), B.BF16, C, W, V)
    ctx.sync()
    rC, rW, rV = sm.bin_cov_dense(sm.residuals_dense(D.y, D.mask, mu), D.mask)
    assert np.array_equal(host(C), rC), "tensor-core pair counts must be exact"
    gw = host(W).astype(np.float64)
    pos = rW > 0
    assert np.all(gw[~pos] == 0.0)
    assert np.max(np.abs(gw[pos] / rW[pos] - 1.0)) <= 2.0 ** -8
    assert rel_l2(host(V).astype(np.float64), rV) <= 5e-3
    assert np.allclose(gw, gw.T, rtol=1e-6, atol=0)


def test_cov_bins_bf16_rejects_unaligned_grid(ctx, B):
    m = (10, 10)
    P = 100
    y = torch.zeros(4, P, dtype=torch.float64, device=DEV)
    C = torch.empty(P, P, dtype=torch.int32, device=DEV)
    W = torch.empty(P, P, dtype=torch.float32, device=DEV)
    with pytest.raises(B.FpcaError) as e:
        ctx.bin_cov(ctx.dense(y), m, torch.zeros(P, dtype=torch.float64, device=DEV), B.BF16, C, W, W)
    assert e.value.status == B.E_UNSUPPORTED


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cov_bins_sparse_folds(ctx, B, prec):
    D = fs.make_sparse(2, (8, 8), 200, [2.0, 1.0], nmin=1, nmax=9, seed=13, nfold=5)
    P = D.P
    mu = np.linspace(-0.5, 0.5, P)
    dt = torch.float64 if prec == "f64" else torch.float32
    C = torch.empty(5, P, P, dtype=torch.int32, device=DEV)
    W, V, Q = (torch.empty(5, P, P, dtype=dt, device=DEV) for _ in range(3))
    ctx.bin_cov(ctx.sparse(dev(D.offs), dev(D.t), dev(D.y)), D.m, dev(mu),
                B.F64 if prec == "f64" else B.F32, C, W, V, q=Q, fold=dev(D.fold), nfold=5)
    ctx.sync()
    r = sm.residuals_sparse(D.t, D.y, mu, D.m)
    rC, rW, rV, rQ = sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, 5)
    assert np.array_equal(host(C), rC)
    tol = 1e-12 if prec == "f64" else 2e-6
    for a, b in ((W, rW), (V, rV), (Q, rQ)):
        assert np.allclose(host(a).astype(np.float64), b, rtol=tol, atol=tol * np.abs(b).max())


# ----------------------------------------------------------------------------
# covariance smoother
# ----------------------------------------------------------------------------

def _oracle_cov_bins(D, h_mu):
    cnt, Wm, Vm, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h_mu, cnt, Wm, Vm)
    mu = np.where(np.isnan(mu), 0.0, mu)
    C, W, V = sm.bin_cov_dense(sm.residuals_dense(D.y, D.mask, mu), D.mask)
    return cnt, mu, C, W, V


def test_smooth_cov_f64_full_grid(ctx, B):
    D = fs.dense_2d_full()
    h = (0.15, 0.15)
    _, _, C, W, V = _oracle_cov_bins(D, h)
    P = D.P
    G = torch.empty(P, P, dtype=torch.float64, device=DEV)
    st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W), dev(V), [h], B.F64, gamma=G, status=st)
    ctx.sync()
    rG, rst = sm.smooth_cov_grid(D.m, h, C, W, V)
    assert np.array_equal(host(st), rst)
    assert rel_l2(host(G), rG) <= 1e-6
    assert np.max(np.abs(host(G) - rG)) <= 1e-9 * np.max(np.abs(rG))


@pytest.mark.parametrize("prec", ["f32", "f32c", "f64"])
def test_smooth_cov_d1(ctx, B, prec):
    D = fs.make_dense(1, (40,), 60, [2.0, 1.0], sigma=0.3, mean="1d", seed=3, dropout=0.3)
    h = (0.12,)
    _, _, C, W, V = _oracle_cov_bins(D, h)
    P = D.P
    dt = torch.float64 if prec == "f64" else torch.float32
    p = {"f32": B.F32, "f32c": B.F32C, "f64": B.F64}[prec]
    G = torch.empty(P, P, dtype=dt, device=DEV)
    st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W, dt), dev(V, dt), [h], p, gamma=G, status=st)
    ctx.sync()
    rG, rst = sm.smooth_cov_grid(D.m, h, C, W, V)
    ok = (rst == sm.STATUS_OK) & (host(st) == sm.STATUS_OK)
    if prec == "f64":
        assert np.array_equal(host(st), rst)
    else:
        assert_status_band(host(st), rst, grid_pairs(P), D.m, h, C, W, V, max_mismatch=P * P // 1000)
    tol = 1e-6 if prec == "f64" else 1e-5
    assert rel_l2(host(G).astype(np.float64)[ok], rG[ok]) <= tol


def test_smooth_cov_affine_and_symmetry_through_abi(ctx, B):
    rng = np.random.default_rng(21)
    m = (12, 16)
    P = 192
    c = sm.centres(m)
    A = rng.random((P, P)) * (rng.random((P, P)) < 0.6)
    W = A + A.T
    np.fill_diagonal(W, 0.0)
    C = (W > 0).astype(np.int32)
    # an affine surface that is not symmetric in (s, t) (bins flagged as such: every
    # pair fitted) and a symmetric one (t >= s fitted, the rest mirrored)
    truth_a = 0.4 + (c @ np.array([1.0, -2.0]))[:, None] + (c @ np.array([0.5, 0.3]))[None, :]
    truth_s = 0.4 + (c @ np.array([1.0, -2.0]))[:, None] + (c @ np.array([1.0, -2.0]))[None, :]
    h = (0.3, 0.35)
    for truth, symmetric in ((truth_a, False), (truth_s, True)):
        for prec, dt, tol in ((B.F64, torch.float64, 1e-10), (B.F32, torch.float32, 2e-4)):
            G = torch.empty(P, P, dtype=dt, device=DEV)
            st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
            ctx.smooth_cov_project(m, dev(C), dev(W, dt), dev(W * truth, dt), [h], prec, gamma=G,
                                   status=st, symmetric=symmetric)
            ctx.sync()
            ok = host(st) == sm.STATUS_OK
            assert ok.mean() > 0.9
            assert np.max(np.abs(host(G).astype(np.float64)[ok] - truth[ok])) <= tol * np.abs(truth).max()
    # symmetric responses give a symmetric surface
    Bm = rng.standard_normal((P, P))
    Vs = W * (Bm + Bm.T)
    G = torch.empty(P, P, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_project(m, dev(C), dev(W, torch.float32), dev(Vs, torch.float32), [h], B.F32, gamma=G)
    ctx.sync()
    g = host(G).astype(np.float64)
    fin = np.isfinite(g) & np.isfinite(g.T)
    assert np.max(np.abs(g - g.T)[fin]) <= 1e-5 * np.max(np.abs(g[fin]))


def test_smooth_cov_raw_mode_f64(ctx, B):
    D = fs.make_dense(2, (8, 8), 40, [2.0, 1.0], sigma=0.3, seed=33, dropout=0.2)
    h = (0.3, 0.3)
    out = sm.dense_gamma(D.y, D.mask, D.m, h, h, mode="raw")
    P = D.P
    C, W, V = sm.bin_cov_dense(D.y, D.mask)
    G = torch.empty(P, P, dtype=torch.float64, device=DEV)
    st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W), dev(V), [h], B.F64,
                           mu_raw=dev(np.where(np.isnan(out["mu"]), 0.0, out["mu"])), gamma=G, status=st)
    ctx.sync()
    assert np.array_equal(host(st), out["status"])
    ok = out["status"] != sm.STATUS_EMPTY
    assert rel_l2(host(G)[ok], out["gamma"][ok]) <= 1e-6


def test_smooth_cov_two_bandwidths_one_call(ctx, B):
    D = fs.dense_2d_full()
    _, _, C, W, V = _oracle_cov_bins(D, (0.15, 0.15))
    P = D.P
    hs = [(0.15, 0.15), (0.3, 0.2)]
    G = torch.empty(2, P, P, dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W), dev(V), hs, B.F64, gamma=G)
    G1 = torch.empty(P, P, dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W), dev(V), [hs[1]], B.F64, gamma=G1)
    ctx.sync()
    assert torch.equal(G[1], G1)
    pairs = np.array([(0, 0), (17, 200), (255, 3), (128, 129)])
    ref, _ = sm.smooth_cov_points(pairs, D.m, hs[1], C, W, V)
    got = host(G1)[pairs[:, 0], pairs[:, 1]]
    assert np.allclose(got, ref, rtol=1e-10)


def test_smooth_cov_rejects_bad_arguments(ctx, B):
    P = 16
    z = torch.zeros(P, P, dtype=torch.float64, device=DEV)
    c = torch.zeros(P, P, dtype=torch.int32, device=DEV)
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_cov_project((4, 4), c, z, z, [(0.0, 0.1)], B.F64, gamma=z)
    assert e.value.status == B.E_INVALID_ARG
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_cov_project((4, 4), c, z, z, [(0.1, 0.1)], B.F32, gamma=z)
    assert e.value.status == B.E_UNSUPPORTED


# ----------------------------------------------------------------------------
# eigen step
# ----------------------------------------------------------------------------

def test_eig_dense_and_rproj_vs_oracle(ctx, B):
    D = fs.make_dense(2, (16, 16), 200, [8.0, 4.0, 2.0, 1.0], sigma=0.3, seed=44)
    h = (0.15, 0.15)
    out = sm.dense_gamma(D.y, D.mask, D.m, h, h)
    G = out["gamma"]
    P, k, l = D.P, 4, 12
    dom = out["cnt"] > 0
    # dense FP64 eigensolver
    ev = torch.empty(k, dtype=torch.float64, device=DEV)
    vec = torch.empty(k, P, dtype=torch.float64, device=DEV)
    fve = torch.empty(k, dtype=torch.float64, device=DEV)
    ctx.rproj_eig(D.m, dev(G), k, ev, vec, fve, domain=dev(out["cnt"], torch.int32), full=True)
    ctx.sync()
    lam, phi, rfve = oe.eig_full(G, D.m, dom, k)
    assert np.allclose(host(ev), lam, rtol=1e-10)
    # sine of the largest principal angle (arccos cannot resolve below ~2e-8)
    Qg, _ = np.linalg.qr(host(vec).T)
    Qo, _ = np.linalg.qr(phi)
    assert np.linalg.norm(Qg - Qo @ (Qo.T @ Qg), 2) <= 1e-8
    for j in range(k):  # sign convention: the largest-magnitude entry is positive
        vj = host(vec)[j]
        assert vj[np.argmax(np.abs(vj))] > 0 or np.sum(np.abs(vj) > 0.999 * np.abs(vj).max()) > 1
        assert abs(abs(vj @ phi[:, j]) / D.P - 1.0) <= 1e-8
    assert np.allclose(host(fve), rfve, rtol=1e-10)
    # random projection on FP32 Sigma with the same Omega
    om = fs.gaussian_test_matrix(P, l, 7)
    ctx.rproj_eig(D.m, dev(G, torch.float32), k, ev, vec, fve, domain=dev(out["cnt"], torch.int32),
                  omega=dev(om, torch.float32), power_iters=2)
    ctx.sync()
    lam_r, phi_r, fve_r = oe.rproj_eig(G, D.m, dom, om, k, 2)
    assert np.allclose(host(ev), lam_r, rtol=1e-4)
    for j in range(k):
        assert oe.subspace_angle(host(vec)[j:j + 1].T, phi_r[:, j:j + 1]) <= 1e-3
    assert np.allclose(host(fve), fve_r, rtol=1e-4)


@pytest.mark.parametrize("m,l", [((23, 31), 6), ((23, 31), 12), ((23, 31), 18), ((17, 45), 24),
                                 ((17, 45), 40), ((40, 41), 64),
                                 ((22, 31), 6), ((22, 31), 18), ((34, 45), 24), ((24, 30), 12),
                                 ((80, 80), 18)])
def test_rproj_widths_and_ragged_grids(ctx, m, l):
    """Random projection at every width the projection kernel is built for (l <= 8, 20,
    24, 64), on grids whose node counts leave ragged row tiles and k ranges, with a
    ragged domain; the same Omega on both sides.  For 8 < l <= 20 and P a multiple of 8
    (24 x 30, 80 x 80) the rows of Sigma arrive by bulk copies; 80 x 80 has k ranges
    longer than one staged chunk of Omega and a half-filled last row tile."""
    P = m[0] * m[1]
    rng = np.random.default_rng(l + P)
    s = (np.arange(m[0]) + 0.5) / m[0]
    t = (np.arange(m[1]) + 0.5) / m[1]
    S, T = np.meshgrid(s, t, indexing="ij")
    lam0 = [8.0, 4.0, 2.0, 1.0, 0.5, 0.25]
    phis = [np.cos(np.pi * (j + 1) * S) * np.sin(np.pi * (j % 3 + 1) * T + 0.3 * j)
            for j in range(len(lam0))]
    F = np.stack([f.ravel() for f in phis], axis=1)
    G = F @ np.diag(lam0) @ F.T
    E = rng.standard_normal((P, P)) * 1e-3
    G = G + 0.5 * (E + E.T)
    cnt = ((S - 0.5) ** 2 + (T - 0.5) ** 2 <= 0.23).astype(np.int32).ravel()
    k = min(6, l - 1)   # the projection needs k < l
    om = fs.gaussian_test_matrix(P, l, 11)
    ev = torch.empty(k, dtype=torch.float64, device=DEV)
    vec = torch.empty(k, P, dtype=torch.float64, device=DEV)
    fve = torch.empty(k, dtype=torch.float64, device=DEV)
    ctx.rproj_eig(m, dev(G, torch.float32), k, ev, vec, fve, domain=dev(cnt, torch.int32),
                  omega=dev(om, torch.float32), power_iters=2)
    ctx.sync()
    lam_r, phi_r, fve_r = oe.rproj_eig(G.astype(np.float32).astype(np.float64), m, cnt > 0, om,
                                       k, 2)
    assert np.allclose(host(ev), lam_r, rtol=1e-4)
    for j in range(k):
        assert oe.subspace_angle(host(vec)[j:j + 1].T, phi_r[:, j:j + 1]) <= 1e-3
    assert np.allclose(host(fve), fve_r, rtol=1e-4)


# ----------------------------------------------------------------------------
# end to end
# ----------------------------------------------------------------------------

def test_pipeline_bf16_f32_small_end_to_end(ctx, B):
    from paper_1510_04439_gb300 import pipeline
    D = fs.make_dense(2, (16, 16), 300, [8.0, 4.0, 2.0, 1.0], sigma=0.5, seed=55, domain="disk",
                      dropout=0.1)
    h = (0.15, 0.15)
    k, l = 4, 14
    om = fs.gaussian_test_matrix(D.P, l, 9)
    bufs = pipeline.alloc_dense(torch, torch.device(DEV), D.P, k, B.BF16, B.F32)
    pipeline.run_dense(ctx, D.m, dev(D.y), dev(D.mask), h, h, k, bufs, bin_prec=B.BF16,
                       smooth_prec=B.F32, omega=dev(om, torch.float32), power_iters=2)
    ctx.sync()
    ref = sm.dense_gamma(D.y, D.mask, D.m, h, h)
    assert np.array_equal(host(bufs.ccnt), ref["C"])
    assert np.allclose(host(bufs.mu)[ref["cnt"] > 0], ref["mu"][ref["cnt"] > 0], rtol=1e-12, atol=1e-12)
    ok = (ref["status"] == sm.STATUS_OK) & (host(bufs.status) == sm.STATUS_OK)
    dom = ref["cnt"] > 0
    inside = ok & dom[:, None] & dom[None, :]
    assert rel_l2(host(bufs.gamma).astype(np.float64)[inside], ref["gamma"][inside]) <= 5e-3
    lam, phi, _ = oe.rproj_eig(ref["gamma"], D.m, dom, om, k, 2)
    assert np.allclose(host(bufs.evals), lam, rtol=1e-2)
    assert oe.subspace_angle(host(bufs.evecs).T, phi) <= 5e-2


@pytest.mark.slow
def test_pipeline_full_size_disk_64x64_n1000(ctx, B):
    """The benchmark's workload and launch configuration: exact counts, sampled
    Gamma_hat points against the oracle's window sums, eigen properties."""
    from paper_1510_04439_gb300 import pipeline
    D = fs.dense_2d_disk()
    h = (0.15, 0.15)
    k, l = 8, 18
    om = fs.gaussian_test_matrix(D.P, l, fs.SEED_BASE)
    bufs = pipeline.alloc_dense(torch, torch.device(DEV), D.P, k, B.BF16, B.F32)
    pipeline.run_dense(ctx, D.m, dev(D.y, torch.float32), dev(D.mask), h, h, k, bufs,
                       bin_prec=B.BF16, smooth_prec=B.F32C, omega=dev(om, torch.float32),
                       power_iters=2)
    ctx.sync()
    y32 = D.y.astype(np.float32).astype(np.float64)
    cnt, mu, C, W, V = _oracle_cov_bins(type(D)(**{**D.__dict__, "y": y32}), h)
    assert np.array_equal(host(bufs.ccnt), C), "pair counts must be bit-exact"
    gmu = host(bufs.mu)
    assert np.allclose(gmu[cnt > 0], mu[cnt > 0], rtol=1e-11, atol=1e-12)
    rng = np.random.default_rng(0)
    inside = np.nonzero(cnt > 0)[0]
    pairs = np.stack([rng.choice(inside, 300), rng.choice(inside, 300)], 1)
    pairs = np.concatenate([pairs, [[inside[0], inside[0]], [inside[-1], inside[0]],
                                    [inside[len(inside) // 2]] * 2]], 0)
    ref, rst = sm.smooth_cov_points(pairs, D.m, h, C, W, V)
    g = host(bufs.gamma).astype(np.float64)[pairs[:, 0], pairs[:, 1]]
    gst = host(bufs.status)[pairs[:, 0], pairs[:, 1]]
    assert_status_band(gst, rst, pairs, D.m, h, C, W, V, max_mismatch=3)
    ok = rst == sm.STATUS_OK
    assert rel_l2(g[ok], ref[ok]) <= 5e-3
    # eigen properties of the returned pairs on the GPU's own surface
    lam = host(bufs.evals)
    phi = host(bufs.evecs).T
    assert np.all(np.diff(lam) <= 0)
    dv = 1.0 / D.P
    assert np.allclose(phi.T @ phi * dv, np.eye(k), atol=1e-4)
    S = oe.matrixize(host(bufs.gamma).astype(np.float64), cnt > 0)
    resid = np.linalg.norm(S @ phi * dv - phi * lam[None, :], axis=0) / np.abs(lam)
    assert np.all(resid[:4] <= 1e-2)


# ----------------------------------------------------------------------------
# cross-validation and the fused projection
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cv_scores_vs_oracle(ctx, B, prec):
    from oracle import cv as ocv
    D = fs.make_sparse(2, (8, 8), 400, [2.0, 1.0], nmin=3, nmax=12, sigma=0.4, seed=77, nfold=5)
    P = D.P
    mu = np.linspace(-0.2, 0.3, P)
    r = sm.residuals_sparse(D.t, D.y, mu, D.m)
    C, W, V, Q = sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, 5)
    hs = [0.1, 0.2, 0.35]
    ref = np.array([ocv.cv_score(D.m, [h, h], C, W, V, Q) for h in hs])
    dt = torch.float64 if prec == "f64" else torch.float32
    cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W, dt), dev(V, dt), [(h, h) for h in hs],
                           B.F64 if prec == "f64" else B.F32, q=dev(Q, dt), nfold=5, cv=cv)
    ctx.sync()
    got = host(cv)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    tol = 1e-9 if prec == "f64" else 1e-4
    assert np.allclose(got[fin], ref[fin], rtol=tol)
    if fin.sum() >= 2:
        assert np.argmin(np.where(fin, got, np.inf)) == np.argmin(np.where(fin, ref, np.inf))


def test_fused_projection_matches_product(ctx, B):
    D = fs.dense_2d_full()
    h = (0.15, 0.15)
    _, _, C, W, V = _oracle_cov_bins(D, h)
    rG, rst = sm.smooth_cov_grid(D.m, h, C, W, V)
    P, l = D.P, 10
    om = fs.gaussian_test_matrix(P, l, 3)
    y = torch.empty(P, l, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W), dev(V), [h], B.F64,
                           omega=dev(om, torch.float32), y=y)
    ctx.sync()
    ref = np.where(np.isnan(rG), 0.0, rG) @ om.astype(np.float32).astype(np.float64)
    assert rel_l2(host(y).astype(np.float64), ref) <= 1e-6


@pytest.mark.parametrize("prec", ["f32", "f32c"])
@pytest.mark.parametrize("m,h", [((13, 16), (0.2, 0.25)), ((20, 24), (0.3, 0.12)), ((9, 8), (0.6, 0.45))])
def test_smooth_cov_f32_d2_ragged_tiles(ctx, B, prec, m, h):
    """FP32 t-side kernel: t-plane rows not a multiple of the tile height, wide and narrow windows."""
    D = fs.make_dense(2, m, 80, [2.0, 1.0, 0.5], sigma=0.3, seed=m[0] * 7 + m[1], dropout=0.2)
    _, _, C, W, V = _oracle_cov_bins(D, (0.3, 0.3))
    P = D.P
    p = B.F32 if prec == "f32" else B.F32C
    G = torch.empty(P, P, dtype=torch.float32, device=DEV)
    st = torch.empty(P, P, dtype=torch.uint8, device=DEV)
    ctx.smooth_cov_project(D.m, dev(C, torch.int32), dev(W, torch.float32), dev(V, torch.float32),
                           [h], p, gamma=G, status=st)
    ctx.sync()
    rG, rst = sm.smooth_cov_grid(D.m, h, C, W, V)
    gst = host(st)
    assert_status_band(gst, rst, grid_pairs(P), D.m, h, C, W, V, max_mismatch=P * P // 1000)
    ok = (rst == sm.STATUS_OK) & (gst == sm.STATUS_OK)
    assert rel_l2(host(G).astype(np.float64)[ok], rG[ok]) <= 1e-5
    fb = (rst == sm.STATUS_FALLBACK) & (gst == sm.STATUS_FALLBACK)
    if fb.any():
        assert rel_l2(host(G).astype(np.float64)[fb], rG[fb]) <= 1e-5


@pytest.mark.slow
def test_sparse_cv_pipeline_vs_oracle(ctx, B):
    """Sparse workload shape (Uniform{5..20} points per subject, 5 folds) on a
    16 x 16 bin grid: mean bins, mean fit, fold-split covariance bins and the CV
    grid through the ABI, against the oracle end to end."""
    from oracle import cv as ocv
    D = fs.sparse_2d(n=2000, m=16)
    m = D.m
    P = D.P
    hmu = (0.1, 0.1)
    hs = [0.06, 0.12, 0.24]
    offs, t, y = dev(D.offs), dev(D.t), dev(D.y)
    data = ctx.sparse(offs, t, y)
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(2))
    ctx.bin_mean(data, m, cnt, w, v)
    mu = torch.empty(P, dtype=torch.float64, device=DEV)
    ctx.smooth_mean(m, cnt, w, v, hmu, mu)
    C = torch.empty(5, P, P, dtype=torch.int32, device=DEV)
    W, V, Q = (torch.empty(5, P, P, dtype=torch.float32, device=DEV) for _ in range(3))
    ctx.bin_cov(data, m, mu, B.F32, C, W, V, q=Q, fold=dev(D.fold), nfold=5)
    cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
    ctx.smooth_cov_project(m, C, W, V, [(h, h) for h in hs], B.F32, q=Q, nfold=5, cv=cv)
    ctx.sync()
    rc, rw, rv, _ = sm.bin_mean_sparse(D.offs, D.t, D.y, m)
    rmu, _ = sm.smooth_mean(m, hmu, rc, rw, rv)
    assert np.allclose(host(mu), rmu, rtol=1e-10, atol=1e-12)
    r = sm.residuals_sparse(D.t, D.y, rmu, m)
    rC, rW, rV, rQ = sm.bin_cov_sparse(D.offs, D.t, r, m, D.fold, 5)
    assert np.array_equal(host(C), rC)
    ref = np.array([ocv.cv_score(m, [h, h], rC, rW, rV, rQ) for h in hs])
    got = host(cv)
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=1e-4)
    assert np.argmin(np.where(fin, got, np.inf)) == np.argmin(np.where(fin, ref, np.inf))
