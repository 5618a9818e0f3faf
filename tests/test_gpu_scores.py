"""GPU parity of the principal component scores (PACE, Eq. 2.7; integration,
Section 2.1) and of the reconstruction against the FP64 oracle."""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import scores as osc

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


def basis(m, L):
    c = fs.grid_centres(m)
    return np.stack([fs.eval_fourier(s, c) for s in fs.fourier_basis_specs(len(m), L)], axis=1)


def gpu_pace_sparse(ctx, offs, t, y, m, mu, phi, lam, s2):
    from paper_1510_04439_gb300 import binding as B
    n, L = len(offs) - 1, phi.shape[1]
    data = B.Context.sparse(dev(offs), dev(t), dev(y))
    out = torch.empty((n, L), dtype=torch.float64, device=DEV)
    ctx.scores_pace(data, m, dev(mu), dev(lam), dev(phi.T), L, dev(np.array([s2])), out)
    ctx.sync()
    return host(out)


def gpu_pace_dense(ctx, y, mask, m, mu, phi, lam, s2, ydtype=torch.float64):
    from paper_1510_04439_gb300 import binding as B
    L = phi.shape[1]
    data = B.Context.dense(dev(y, ydtype), None if mask is None else dev(mask))
    out = torch.empty((y.shape[0], L), dtype=torch.float64, device=DEV)
    ctx.scores_pace(data, m, dev(mu), dev(lam), dev(phi.T), L, dev(np.array([s2])), out)
    ctx.sync()
    return host(out)


def close(a, b, rtol):
    """Max error relative to the largest score magnitude."""
    return float(np.max(np.abs(a - b))) <= rtol * max(1.0, float(np.max(np.abs(b))))


def test_pace_sparse_matches_oracle(ctx):
    D = fs.make_sparse(2, (16, 16), 300, [4.0, 2.0, 1.0, 0.5], nmin=1, nmax=20, seed=31)
    offs = np.insert(D.offs, [7, 7, 120], [D.offs[7], D.offs[7], D.offs[120]])  # empty subjects
    phi = basis(D.m, 4)
    mu = fs.mean_sincos(fs.grid_centres(D.m))
    for s2 in (0.25, 1e-3):
        got = gpu_pace_sparse(ctx, offs, D.t, D.y, D.m, mu, phi, D.lam, s2)
        ref = osc.pace_scores_sparse(offs, D.t, D.y, D.m, mu, phi, D.lam, s2)
        assert close(got, ref, 1e-9)
        assert np.all(got[[7, 8, 122]] == 0.0)


def test_pace_dense_matches_oracle_with_mask_and_16_components(ctx):
    m, L = (16, 16), 16
    D = fs.make_dense(2, m, 64, [2.0 ** (-k / 2) for k in range(L)], sigma=0.5, seed=32,
                      domain="disk", dropout=0.3)
    mask = D.mask.copy()
    mask[5] = 0        # a subject without observations
    mask[6] = 0
    mask[6, 100:103] = 1   # fewer observations than components
    phi = basis(m, L)
    mu = D.true_mean()
    for s2 in (0.25, 0.01):
        got = gpu_pace_dense(ctx, D.y, mask, m, mu, phi, D.lam, s2)
        ref = osc.pace_scores_dense(D.y, mask, mu, phi, D.lam, s2)
        assert close(got, ref, 1e-9)
        assert np.all(got[5] == 0.0)
    # FP32 observations: the oracle reads the same FP32 values
    y32 = D.y.astype(np.float32)
    got = gpu_pace_dense(ctx, y32, mask, m, mu, phi, D.lam, 0.25, torch.float32)
    ref = osc.pace_scores_dense(y32.astype(np.float64), mask, mu, phi, D.lam, 0.25)
    assert close(got, ref, 1e-9)
    # no mask: every node observed
    got = gpu_pace_dense(ctx, D.y, None, m, mu, phi, D.lam, 0.25)
    ref = osc.pace_scores_dense(D.y, np.ones_like(mask), mu, phi, D.lam, 0.25)
    assert close(got, ref, 1e-9)


def test_pace_recovers_true_scores(ctx):
    """Noise-free curves in the span of phi: sigma^2 -> 0 returns the scores."""
    m, L = (12, 12), 4
    rng = np.random.default_rng(33)
    phi = basis(m, L)
    lam = np.array([4.0, 2.0, 1.0, 0.5])
    a = rng.standard_normal((40, L)) * np.sqrt(lam)
    mu = rng.standard_normal(144)
    y = mu[None, :] + a @ phi.T
    got = gpu_pace_dense(ctx, y, None, m, mu, phi, lam, 1e-12)
    assert np.allclose(got, a, rtol=0, atol=1e-8)


def test_pace_full_size_sparse_2d(ctx):
    """20000 subjects with 5..20 points on a 64 x 64 grid, 6 components: every subject."""
    D = fs.sparse_2d()
    phi = basis(D.m, 6)
    mu = fs.mean_sincos(fs.grid_centres(D.m))
    got = gpu_pace_sparse(ctx, D.offs, D.t, D.y, D.m, mu, phi, D.lam, 0.25)
    ref = osc.pace_scores_sparse(D.offs, D.t, D.y, D.m, mu, phi, D.lam, 0.25)
    assert close(got, ref, 1e-9)


def test_pace_full_size_dense_2d_disk_sampled(ctx):
    """1000 surfaces on the 64 x 64 disk with 10% dropout, 8 components: GPU on all,
    the oracle's N_i x N_i solve on sampled subjects."""
    D = fs.dense_2d_disk()
    phi = basis(D.m, 8)
    mu = D.true_mean()
    got = gpu_pace_dense(ctx, D.y, D.mask, D.m, mu, phi, D.lam, 0.25)
    idx = np.array([0, 313, 999])
    ref = osc.pace_scores_dense(D.y[idx], D.mask[idx], mu, phi, D.lam, 0.25)
    assert close(got[idx], ref, 1e-9)
    assert np.all(np.isfinite(got))


def test_integral_scores_match_oracle(ctx):
    from paper_1510_04439_gb300 import binding as B
    for m, L, ydt, mean in (((16, 16), 16, torch.float64, "sincos"),
                            ((8, 8, 8), 5, torch.float32, "exp"), ((64,), 3, torch.float64, "1d")):
        D = fs.make_dense(len(m), m, 50, [1.0] * L, seed=34, dropout=0.2, mean=mean)
        y = D.y.astype(np.float32).astype(np.float64) if ydt == torch.float32 else D.y
        phi = basis(m, L)
        mu = D.true_mean()
        for mask in (D.mask, None):
            data = B.Context.dense(dev(D.y, ydt), None if mask is None else dev(mask))
            out = torch.empty((D.n, L), dtype=torch.float64, device=DEV)
            ctx.scores_integral(data, m, dev(mu), dev(phi.T), L, out)
            ctx.sync()
            mk = np.ones_like(D.mask) if mask is None else mask
            ref = osc.integral_scores(y, mk, mu, phi, m)
            assert np.allclose(host(out), ref, rtol=1e-11, atol=1e-12)


def test_integral_scores_of_the_basis_are_the_identity(ctx):
    """Orthonormal basis (sum_p phi_k phi_l / P = delta_kl): integrating
    mu + sum_l a_l phi_l returns a exactly up to rounding."""
    from paper_1510_04439_gb300 import binding as B
    m, L = (16, 16), 6
    phi = basis(m, L)
    a = np.random.default_rng(35).standard_normal((20, L))
    mu = np.linspace(-1, 1, 256)
    y = mu[None, :] + a @ phi.T
    out = torch.empty((20, L), dtype=torch.float64, device=DEV)
    ctx.scores_integral(B.Context.dense(dev(y)), m, dev(mu), dev(phi.T), L, out)
    ctx.sync()
    assert np.allclose(host(out), a, rtol=0, atol=1e-12)


def test_reconstruct_matches_oracle(ctx):
    m, L, n = (24, 20), 7, 33
    phi = basis(m, L)
    rng = np.random.default_rng(36)
    sc = rng.standard_normal((n, L))
    mu = rng.standard_normal(480)
    out = torch.empty((n, 480), dtype=torch.float32, device=DEV)
    ctx.reconstruct(m, dev(mu), dev(phi.T), L, dev(sc), n, out)
    ctx.sync()
    ref = osc.reconstruct(mu, phi, sc)
    assert np.allclose(host(out), ref, rtol=1e-6, atol=1e-6)


def test_scores_refusals(ctx):
    from paper_1510_04439_gb300 import binding as B
    m = (8, 8)
    phi = dev(basis(m, 4).T)
    mu = dev(np.zeros(64))
    lam = dev(np.ones(4))
    y = dev(np.zeros((3, 64)))
    out = torch.empty((3, 17), dtype=torch.float64, device=DEV)
    data = B.Context.dense(y)
    s2 = dev(np.array([0.25]))
    for L in (0, 17):
        with pytest.raises(B.FpcaError):
            ctx.scores_pace(data, m, mu, lam, phi, L, s2, out)
        with pytest.raises(B.FpcaError):
            ctx.scores_integral(data, m, mu, phi, L, out)
    with pytest.raises(B.FpcaError):
        ctx.scores_pace(data, m, mu, lam, phi, 4, None, out)
    sp = B.Context.sparse(dev(np.array([0, 2], dtype=np.int64)), dev(np.full((2, 2), 0.3)),
                          dev(np.ones(2)))
    with pytest.raises(B.FpcaError):
        ctx.scores_integral(sp, m, mu, phi, 4, out)
    # a zero eigenvalue (no Lambda^{-1}) or a negative sigma^2: reported at sync
    out4 = torch.zeros((3, 4), dtype=torch.float64, device=DEV)
    for bad_lam, bad_s2 in (([1.0, 1.0, 0.0, 1.0], 0.25), ([1.0] * 4, -0.1), ([1.0] * 4, np.nan)):
        ctx.scores_pace(data, m, mu, dev(np.array(bad_lam)), phi, 4, dev(np.array([bad_s2])), out4)
        with pytest.raises(B.FpcaError) as e:
            ctx.sync()
        assert e.value.status == B.E_NUMERIC
        assert np.all(np.isnan(host(out4)))
    ctx.sync()   # the error word was cleared


def test_mise_matches_oracle(ctx):
    m, n = (16, 12), 37
    rng = np.random.default_rng(37)
    x = rng.standard_normal((n, 192))
    xhat = (x + 0.1 * rng.standard_normal((n, 192))).astype(np.float32)
    out = torch.empty(1, dtype=torch.float64, device=DEV)
    for xd in (torch.float64, torch.float32):
        ref = osc.mise(xhat, x.astype(np.float32).astype(np.float64) if xd == torch.float32 else x, m)
        ctx.mise(m, dev(xhat), dev(x, xd), n, out)
        ctx.sync()
        assert np.isclose(float(host(out)[0]), ref, rtol=1e-12), (float(host(out)[0]), ref)
    # constant offset: exactly c^2 on the full grid
    ctx.mise(m, dev(np.full((n, 192), 0.25, dtype=np.float32)), dev(np.zeros((n, 192))), n, out)
    ctx.sync()
    assert np.isclose(float(host(out)[0]), 0.0625, rtol=1e-14)


def test_reconstruct_then_mise_of_true_scores_is_zero(ctx):
    """mu + sum A phi reconstructed from the true scores equals the noise-free
    curves up to FP32 rounding of the output."""
    m, L, n = (20, 20), 5, 25
    phi = basis(m, L)
    rng = np.random.default_rng(38)
    a = rng.standard_normal((n, L))
    mu = rng.standard_normal(400)
    x = mu[None, :] + a @ phi.T
    xh = torch.empty((n, 400), dtype=torch.float32, device=DEV)
    ctx.reconstruct(m, dev(mu), dev(phi.T), L, dev(a), n, xh)
    out = torch.empty(1, dtype=torch.float64, device=DEV)
    ctx.mise(m, xh, dev(x), n, out)
    ctx.sync()
    # every entry is the FP32 rounding of x (compensated sum): error within an ulp
    assert float(host(out)[0]) <= np.mean(np.sum((np.abs(x) * 2.0 ** -23) ** 2, axis=1)) / 400
