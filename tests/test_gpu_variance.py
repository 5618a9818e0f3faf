"""GPU parity of the noise variance (fpca_sigma2, Eq. 2.5-2.6) and of the fused d = 3
surface's diagonal (fpca_smooth_cov_diag) against the FP64 oracle."""
import math

import numpy as np
import pytest

import fpca_synth as fs
from oracle import block as ob
from oracle import smoother as sm
from oracle import variance as ov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


def run_sigma2(ctx, D, h, bin_prec, smooth_prec):
    from paper_1510_04439_gb300 import binding as B
    from paper_1510_04439_gb300 import pipeline
    bufs = pipeline.alloc_dense(torch, DEV, D.P, 4, bin_prec, smooth_prec)
    pipeline.run_dense(ctx, D.m, dev(D.y), dev(D.mask), h, h, 4, bufs, bin_prec=bin_prec,
                       smooth_prec=smooth_prec, full=True)
    sig_t = torch.empty(D.P, dtype=torch.float64, device=DEV)
    st = torch.empty(D.P, dtype=torch.uint8, device=DEV)
    s2 = torch.empty(1, dtype=torch.float64, device=DEV)
    ctx.sigma2(D.m, bufs.cnt, bufs.w, bufs.v2, h, bufs.mu, bufs.gamma.reshape(-1), D.P + 1,
               sig_t, st, s2, domain=bufs.cnt)
    ctx.sync()
    return host(sig_t), host(st), float(host(s2)[0])


def test_sigma2_matches_oracle_fp64(ctx):
    from paper_1510_04439_gb300 import binding as B
    D = fs.make_dense(2, (16, 16), 120, [4.0, 2.0], sigma=0.5, seed=21, domain="disk", dropout=0.2)
    h = (0.15, 0.15)
    sig, st, s2 = run_sigma2(ctx, D, h, B.F64, B.F64)
    ref = sm.dense_gamma(D.y, D.mask, D.m, h, h)
    cnt, W, V, V2 = sm.bin_mean_dense(D.y, D.mask, D.m)
    gd = np.diag(ref["gamma"])          # NaN where the surface is EMPTY: sigma2 is NaN there
    rsig, rst = ov.sigma2_curve(D.m, h, cnt, W, V2, ref["mu"], gd)
    assert np.array_equal(st, rst)
    ok = np.isfinite(rsig)
    assert np.array_equal(np.isfinite(sig), ok)
    assert np.allclose(sig[ok], rsig[ok], rtol=1e-9, atol=1e-10)
    assert math.isclose(s2, ov.sigma2_scalar(rsig, cnt > 0), rel_tol=1e-9)


def test_sigma2_recovers_noise_variance(ctx):
    """Constant mean and covariance (reproduced without smoothing bias): the GPU
    estimate is within sampling error of sigma^2 = 0.25."""
    from paper_1510_04439_gb300 import binding as B
    rng = np.random.default_rng(11)
    n, P = 400, 256
    y = 1.5 + rng.normal(0, math.sqrt(2.0), (n, 1)) + 0.5 * rng.standard_normal((n, P))

    class Dset:
        pass
    D = Dset()
    D.m, D.P, D.y, D.mask = (16, 16), P, y, np.ones((n, P), dtype=np.uint8)
    _, _, s2 = run_sigma2(ctx, D, (0.15, 0.15), B.F64, B.F64)
    assert abs(s2 - 0.25) < 0.02, s2


def test_fused_diagonal_matches_oracle(ctx):
    D = fs.make_dense(3, (8, 8, 8), 80, [3.0, 1.0], sigma=0.3, mean="exp", seed=23)
    h = [0.3, 0.3, 0.3]
    cnt, W, V, V2 = sm.bin_mean_dense(D.y, D.mask, D.m)
    mu, _ = sm.smooth_mean(D.m, h, cnt, W, V)
    fac = torch.empty(ctx.cov_factor_bytes(D.m, D.n), dtype=torch.uint8, device=DEV)
    ctx.bin_cov_factor(ctx.dense(dev(D.y.astype(np.float32))), D.m, dev(mu), fac)
    diag = torch.empty(D.P, dtype=torch.float64, device=DEV)
    ctx.smooth_cov_diag(D.m, fac, D.n, h, diag)
    ctx.sync()
    G, _ = ob.smooth_cov_rows(D.y, None, mu, D.m, h, np.arange(D.P))
    ref = np.diag(G)
    assert np.linalg.norm(host(diag) - ref) / np.linalg.norm(ref) < 5e-3
