"""Pins of the score oracle (PACE Eq. 2.7, integration, reconstruction)."""
import numpy as np

import fpca_synth as fs
from oracle import scores as osc
from oracle import smoother as sm


def _basis(m, L):
    c = sm.centres(m)
    specs = fs.fourier_basis_specs(len(m), L)
    return np.stack([fs.eval_fourier(s, c) for s in specs], axis=1)


def test_pace_recovers_scores_of_noise_free_curves():
    """Y^C in the span of the L eigenfunctions at >= L points: as sigma^2 -> 0 the
    PACE predictor returns the scores; at any sigma^2 it equals the ridge form
    (sigma^2 Lambda^-1 + Phi'Phi)^-1 Phi' Y^C (the push-through identity)."""
    m = (12, 12)
    L = 4
    phi = _basis(m, L)
    rng = np.random.default_rng(2)
    n = 30
    lam = np.array([4.0, 2.0, 1.0, 0.5])
    a = rng.standard_normal((n, L)) * np.sqrt(lam)
    mu = rng.standard_normal(144)
    offs = np.zeros(n + 1, dtype=np.int64)
    ts, ys = [], []
    for i in range(n):
        while True:   # node sets on which the L functions are identifiable
            k = int(rng.integers(L + 1, 12))
            nodes = rng.choice(144, size=k, replace=False)
            if np.linalg.cond(phi[nodes]) < 1e6:
                break
        c = sm.centres(m)[nodes]
        ts.append(c)
        ys.append(mu[nodes] + phi[nodes] @ a[i])
        offs[i + 1] = offs[i] + k
    t, y = np.concatenate(ts), np.concatenate(ys)
    est = osc.pace_scores_sparse(offs, t, y, m, mu, phi, lam, 1e-9)
    assert np.allclose(est, a, rtol=0, atol=1e-4)
    s2 = 0.3
    est = osc.pace_scores_sparse(offs, t, y, m, mu, phi, lam, s2)
    for i in range(n):
        nodes = sm.bin_of(t[offs[i]:offs[i + 1]], m)
        Phi = phi[nodes]
        ridge = np.linalg.solve(s2 * np.diag(1.0 / lam) + Phi.T @ Phi, Phi.T @ (y[offs[i]:offs[i + 1]] - mu[nodes]))
        assert np.allclose(est[i], ridge, rtol=1e-10, atol=1e-12)


def test_pace_shrinks_to_the_prior_for_large_noise():
    """sigma^2 >> lambda |Phi|^2: Sigma ~ sigma^2 I, so A ~ lambda Phi' Y^C / sigma^2."""
    m = (10,)
    phi = _basis(m, 2)
    lam = np.array([1.0, 0.5])
    y = np.array([[0.3, -1.0, 2.0, 0.0, 1.0, 0.5, -0.2, 0.1, 0.7, -0.4]])
    mask = np.ones_like(y, dtype=bool)
    s2 = 1e8
    est = osc.pace_scores_dense(y, mask, np.zeros(10), phi, lam, s2)
    approx = lam * (phi.T @ y[0]) / s2
    assert np.allclose(est[0], approx, rtol=1e-6)


def test_dense_pace_equals_sparse_pace_on_the_same_points():
    m = (8, 8)
    phi = _basis(m, 3)
    D = fs.make_dense(2, m, 10, [2.0, 1.0, 0.5], sigma=0.3, seed=4, dropout=0.4)
    mu = np.zeros(64)
    dn = osc.pace_scores_dense(D.y, D.mask, mu, phi, np.array([2.0, 1.0, 0.5]), 0.09)
    c = sm.centres(m)
    offs = np.concatenate([[0], np.cumsum(D.mask.sum(1))]).astype(np.int64)
    rows, cols = np.nonzero(D.mask)
    sp = osc.pace_scores_sparse(offs, c[cols], D.y[rows, cols], m, mu, phi,
                                np.array([2.0, 1.0, 0.5]), 0.09)
    assert np.allclose(dn, sp, rtol=1e-12, atol=1e-12)


def test_integral_scores_and_reconstruction_are_exact_on_the_grid():
    """The Fourier eigenfunctions are orthonormal under the node Riemann sum, so the
    integral scores of mu + sum a_l phi_l are a, and reconstruction returns the data."""
    m = (16, 16)
    L = 5
    phi = _basis(m, L)
    rng = np.random.default_rng(7)
    a = rng.standard_normal((6, L))
    mu = rng.standard_normal(256)
    y = mu[None, :] + a @ phi.T
    est = osc.integral_scores(y, np.ones_like(y, dtype=bool), mu, phi, m)
    assert np.allclose(est, a, rtol=0, atol=1e-12)
    assert np.allclose(osc.reconstruct(mu, phi, est), y, rtol=0, atol=1e-12)


def test_mise_closed_forms():
    """A constant offset c over the full grid integrates to c^2; an error a*phi_l
    along an orthonormal eigenfunction integrates to a^2; the mean runs over
    subjects."""
    m = (12, 10)
    phi = _basis(m, 3)
    x = np.random.default_rng(5).standard_normal((4, 120))
    assert np.isclose(osc.mise(x + 0.3, x, m), 0.09, rtol=1e-13)
    err = np.stack([0.5 * phi[:, 0], -2.0 * phi[:, 2], np.zeros(120), phi[:, 1]])
    assert np.isclose(osc.mise(x + err, x, m), (0.25 + 4.0 + 0.0 + 1.0) / 4, rtol=1e-12)
