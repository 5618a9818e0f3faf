"""GPU parity of the fused d = 3 smoother (fpca_bin_cov_factor, fpca_smooth_cov_apply,
fpca_smooth_cov_tiles, fpca_rproj_eig_factor) against the FP64 oracle.

The oracle's mean fit is handed to the factor so that the comparison isolates the
covariance smoother.  Residuals enter the tensor-core products in BF16 (FP32
accumulation): the stated tolerance for Gamma_hat and Gamma_hat X is a relative L2
error of 5e-3 (BF16 rounds to 2^-9 relative), for the leading eigenvalues 1e-2.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import block as ob
from oracle import eigen as oe
from oracle import smoother as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 5e-3


@pytest.fixture(scope="module")
def ctx():
    from paper_1510_04439_gb300 import binding as B
    return B.Context(0)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_mean(D, h):
    cnt, W, V, _ = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h, cnt, W, V)
    return mu


def make_factor(ctx, D, mu, y_dtype=np.float32):
    data = ctx.dense(dev(D.y.astype(y_dtype)))
    nbytes = ctx.cov_factor_bytes(D.m, D.n)
    assert nbytes > 0
    fac = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    ctx.bin_cov_factor(data, D.m, dev(mu), fac)
    return fac


SMALL = [
    ((8, 8, 8), 60, [0.3, 0.3, 0.3]),
    ((6, 5, 12), 45, [0.4, 0.45, 0.25]),     # ragged tiles on every axis
]


@pytest.mark.parametrize("m,n,h", SMALL)
def test_apply_and_tiles_small(ctx, m, n, h):
    D = fs.make_dense(3, m, n, [3.0, 2.0, 1.0], sigma=0.3, mean="exp", seed=31 + n)
    mu = oracle_mean(D, h)
    G, st = ob.smooth_cov_rows(D.y, None, mu, m, h, np.arange(D.P))
    assert np.all(st == sm.STATUS_OK)
    fac = make_factor(ctx, D, mu)
    rng = np.random.default_rng(7)
    for l in (5, 24, 64):
        X = rng.standard_normal((D.P, l)).astype(np.float32)
        Y = torch.empty(D.P, l, dtype=torch.float32, device=DEV)
        ctx.smooth_cov_apply(m, fac, n, h, dev(X), Y)
        ctx.sync()
        e = rel(host(Y), G @ X.astype(np.float64))
        assert e < TOL, (l, e)
    # every tile pair of the grid through the tile entry point
    tiles = []
    for a0 in range(0, m[0], 4):
        for a1 in range(0, m[1], 4):
            for a2 in range(0, m[2], 8):
                for b0 in range(0, m[0], 4):
                    for b1 in range(0, m[1], 4):
                        for b2 in range(0, m[2], 4):
                            tiles.append((a0, a1, a2, b0, b1, b2))
    out = torch.empty(len(tiles), 128, 64, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_tiles(m, fac, n, h, tiles, out)
    got = host(out)
    ref = np.full_like(got, np.nan, dtype=np.float64)
    Gg = G.reshape(m + m)
    for i, (a0, a1, a2, b0, b1, b2) in enumerate(tiles):
        blk = np.full((4, 4, 8, 4, 4, 4), np.nan)
        sub = Gg[a0:a0 + 4, a1:a1 + 4, a2:a2 + 8, b0:b0 + 4, b1:b1 + 4, b2:b2 + 4]
        blk[:sub.shape[0], :sub.shape[1], :sub.shape[2], :sub.shape[3], :sub.shape[4],
            :sub.shape[5]] = sub
        ref[i] = blk.reshape(128, 64)
    on = ~np.isnan(ref)
    assert np.array_equal(on, ~np.isnan(got))
    e = rel(got[on], ref[on])
    assert e < TOL, e


def test_rproj_eig_small(ctx):
    m, n, h = (8, 8, 8), 200, [0.3, 0.3, 0.3]
    lam = [4.0, 2.0, 1.0, 0.5]
    D = fs.make_dense(3, m, n, lam, sigma=0.2, mean="exp", seed=41)
    mu = oracle_mean(D, h)
    G, _ = ob.smooth_cov_rows(D.y, None, mu, m, h, np.arange(D.P))
    fac = make_factor(ctx, D, mu)
    k, l = 4, 16
    om = fs.gaussian_test_matrix(D.P, l, 5)
    ev = torch.empty(k, dtype=torch.float64, device=DEV)
    evec = torch.empty(k, D.P, dtype=torch.float64, device=DEV)
    fve = torch.empty(k, dtype=torch.float64, device=DEV)
    ctx.rproj_eig_factor(m, fac, n, h, dev(om.astype(np.float32)), k, ev, evec, fve,
                         power_iters=2)
    ctx.sync()
    lam_ref, phi_ref, fve_ref = oe.rproj_eig(G, m, np.ones(D.P, dtype=bool), om, k, 2)
    assert np.allclose(host(ev), lam_ref, rtol=1e-2)
    assert oe.subspace_angle(host(evec).T, phi_ref) <= 2e-2
    assert np.allclose(host(fve), fve_ref, rtol=1e-2)


H3 = [0.15, 0.15, 0.15]
ROWS3 = np.array([0, 31, 1023, 16912, 20000, 32767])


@pytest.fixture(scope="module")
def full3(ctx):
    """n = 2000 volumes on 32^3, the oracle's mean fit, the factored bins, and the
    oracle's Gamma_hat on the rows ROWS3 (every column)."""
    D = fs.dense_3d()
    mu = oracle_mean(D, H3)
    fac = make_factor(ctx, D, mu)
    G, st = ob.smooth_cov_rows(D.y, None, mu, D.m, H3, ROWS3)
    assert np.all(st == sm.STATUS_OK)
    return D, mu, fac, G


@pytest.mark.slow
def test_full_size_rows_and_tiles(ctx, full3):
    """n = 2000 volumes on 32^3 (1.07e9 covariance points): Gamma_hat Omega on sampled
    rows and Gamma_hat on 64 random tile pairs (4x4x8 s-box by 4x4x4 t-box) against
    the FP64 oracle evaluated at exactly those output pairs."""
    D, mu, fac, G = full3
    m, n, h = D.m, D.n, H3
    l = 64
    om = fs.gaussian_test_matrix(D.P, l, 3).astype(np.float32)
    Y = torch.empty(D.P, l, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_apply(m, fac, n, h, dev(om), Y)
    ctx.sync()
    Yh = host(Y)
    e = rel(Yh[ROWS3], G @ om.astype(np.float64))
    assert e < TOL, e
    rng = np.random.default_rng(2026)
    tiles = []
    for _ in range(64):
        s = (4 * rng.integers(0, 8), 4 * rng.integers(0, 8), 8 * rng.integers(0, 4))
        if rng.random() < 0.5:   # half of them near the diagonal
            t = tuple(int(np.clip(s[k] + 4 * rng.integers(-2, 3), 0, 28)) for k in range(3))
        else:
            t = tuple(4 * int(rng.integers(0, 8)) for _ in range(3))
        tiles.append(tuple(int(v) for v in s + t))
    out = torch.empty(64, 128, 64, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_tiles(m, fac, n, h, tiles, out)
    got = host(out)
    errs = []
    for i, (a0, a1, a2, b0, b1, b2) in enumerate(tiles):
        S = ob._box_nodes([a0, a1, a2], [a0 + 4, a1 + 4, a2 + 8], m)
        ref, st = ob.smooth_cov_block(D.y, None, mu, m, h, S, [b0, b1, b2], [b0 + 4, b1 + 4, b2 + 4])
        assert np.all(st == sm.STATUS_OK)
        errs.append(rel(got[i], ref))
    assert max(errs) < TOL, max(errs)


@pytest.mark.slow
def test_full_size_eigenpairs(ctx, full3):
    """The 32^3 step's own projection (k = 10, l = 64, no power step), too large for a
    whole-surface oracle, checked by what Rayleigh-Ritz fixes at any size: with
    psi = phi sqrt(dV) and theta = lambda / dV (Eq. 3.1), the psi are orthonormal, the
    theta descend, psi' Gamma_hat psi = diag(theta) with Gamma_hat psi from the fused
    apply, that product agrees on the sampled rows with the FP64 oracle's Gamma_hat, and
    FVE_j is the running sum of lambda over the trace of Gamma_hat times dV, with the
    diagonal agreeing with the oracle's on the sampled rows."""
    D, _, fac, G = full3
    m, n, h, P = D.m, D.n, H3, D.P
    k, l = 10, 64
    om = fs.gaussian_test_matrix(P, l, fs.SEED_BASE + 3).astype(np.float32)
    ev = torch.empty(k, dtype=torch.float64, device=DEV)
    evec = torch.empty(k, P, dtype=torch.float64, device=DEV)
    fve = torch.empty(k, dtype=torch.float64, device=DEV)
    ctx.rproj_eig_factor(m, fac, n, h, dev(om), k, ev, evec, fve, power_iters=0)
    diag = torch.empty(P, dtype=torch.float64, device=DEV)
    ctx.smooth_cov_diag(m, fac, n, h, diag)
    ctx.sync()
    lam, phi, fv, dg = host(ev), host(evec).T, host(fve), host(diag)
    dv = 1.0 / P
    psi, theta = phi * np.sqrt(dv), lam / dv
    assert np.all(np.diff(lam) <= 0) and lam[-1] > 0
    assert np.max(np.abs(psi.T @ psi - np.eye(k))) < 1e-6
    X = np.zeros((P, 16), dtype=np.float32)
    X[:, :k] = psi
    Y = torch.empty(P, 16, dtype=torch.float32, device=DEV)
    ctx.smooth_cov_apply(m, fac, n, h, dev(X), Y)
    ctx.sync()
    Z = host(Y)[:, :k].astype(np.float64)
    assert rel(psi.T @ Z, np.diag(theta)) < TOL
    assert rel(Z[ROWS3], G @ psi) < TOL
    assert rel(dg[ROWS3], G[np.arange(len(ROWS3)), ROWS3]) < TOL
    assert np.allclose(fv, np.cumsum(lam) / (dg.sum() * dv), rtol=1e-9)


def test_fused_rejects_what_it_does_not_cover(ctx):
    """Masked data, other dimensions, too many taps, bad tile corners and bad l are
    refused synchronously with a status, nothing launched."""
    from paper_1510_04439_gb300 import binding as B
    D = fs.make_dense(3, (8, 8, 8), 20, [2.0, 1.0], sigma=0.3, mean="exp", seed=3)
    mu = np.zeros(D.P)
    nbytes = ctx.cov_factor_bytes(D.m, D.n)
    fac = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
    masked = ctx.dense(dev(D.y.astype(np.float32)), dev(np.ones_like(D.mask, dtype=np.uint8)))
    with pytest.raises(B.FpcaError) as e:
        ctx.bin_cov_factor(masked, D.m, dev(mu), fac)
    assert e.value.status == B.E_UNSUPPORTED
    full = ctx.dense(dev(D.y.astype(np.float32)))
    with pytest.raises(B.FpcaError) as e:
        ctx.bin_cov_factor(full, D.m, dev(mu), fac[: nbytes // 2])
    assert e.value.status == B.E_INVALID_ARG
    ctx.bin_cov_factor(full, D.m, dev(mu), fac)
    X = torch.zeros(D.P, 4, dtype=torch.float32, device=DEV)
    Y = torch.empty_like(X)
    with pytest.raises(B.FpcaError) as e:          # 0.9 * 8 = 7.2 -> 7 taps
        ctx.smooth_cov_apply(D.m, fac, D.n, [0.9, 0.3, 0.3], X, Y)
    assert e.value.status == B.E_UNSUPPORTED
    with pytest.raises(B.FpcaError) as e:          # 0.1 * 8 < 1 -> no taps
        ctx.smooth_cov_apply(D.m, fac, D.n, [0.1, 0.3, 0.3], X, Y)
    assert e.value.status == B.E_UNSUPPORTED
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_cov_apply((16, 32), fac, D.n, [0.3, 0.3], X, Y)
    assert e.value.status == B.E_UNSUPPORTED
    wide = torch.zeros(D.P, 65, dtype=torch.float32, device=DEV)
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_cov_apply(D.m, fac, D.n, [0.3] * 3, wide, torch.empty_like(wide))
    assert e.value.status == B.E_INVALID_ARG
    out = torch.empty(1, 128, 64, dtype=torch.float32, device=DEV)
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_cov_tiles(D.m, fac, D.n, [0.3] * 3, [(0, 0, 4, 0, 0, 0)], out)
    assert e.value.status == B.E_INVALID_ARG
    # the context stays usable
    ctx.smooth_cov_apply(D.m, fac, D.n, [0.3] * 3, X, Y)
    ctx.sync()
    assert float(host(Y).std()) == 0.0
