"""Pins of the noise-variance oracle (Eq. 2.5-2.6, oracle/variance.py)."""
import math

import numpy as np

from oracle import smoother as sm
from oracle import variance as ov


def test_sigma2_curve_exact_on_affine_second_moments():
    """Bins whose mean of Y^2 is affine in t: the local linear b0 reproduces it
    exactly, so sigma2(t) = f(t) - Gamma(t,t) - mu(t)^2 to rounding; the mean term
    enters with a minus sign."""
    m = (9, 7)
    P = 63
    c = sm.centres(m)
    rng = np.random.default_rng(3)
    W = rng.uniform(0.5, 2.0, P)
    cnt = np.ones(P, dtype=np.int64)
    f = 3.0 + 0.7 * c[:, 0] - 1.3 * c[:, 1]
    V2 = W * f
    mu = rng.uniform(-1.0, 1.0, P)
    gd = rng.uniform(0.0, 1.0, P)
    sig, st = ov.sigma2_curve(m, (0.3, 0.35), cnt, W, V2, mu, gd)
    assert np.all(st == sm.STATUS_OK)
    assert np.allclose(sig, f - gd - mu * mu, rtol=0, atol=1e-12)
    dom = np.zeros(P, dtype=bool)
    dom[::3] = True
    assert math.isclose(ov.sigma2_scalar(sig, dom), float(np.mean((f - gd - mu * mu)[dom])),
                        rel_tol=1e-13)


def test_sigma2_empty_nodes_are_left_out():
    m = (8,)
    cnt = np.array([1, 1, 0, 0, 0, 0, 1, 1])
    W = cnt.astype(float)
    V2 = 2.0 * W
    sig, st = ov.sigma2_curve(m, (0.2,), cnt, W, V2, np.zeros(8), np.zeros(8))
    assert np.isnan(sig[3]) and st[3] == sm.STATUS_EMPTY
    assert math.isclose(ov.sigma2_scalar(sig, np.ones(8, bool)), 2.0, rel_tol=1e-12)


def test_sigma2_recovers_the_noise_variance():
    """Y = c + xi_i + eps: mean and covariance are constant, which the local linear
    smoothers reproduce without bias, so the estimate is within sampling error."""
    rng = np.random.default_rng(11)
    m, n, sigma, lam = (16, 16), 400, 0.5, 2.0
    P = 256
    y = 1.5 + rng.normal(0, math.sqrt(lam), (n, 1)) + sigma * rng.standard_normal((n, P))
    mask = np.ones((n, P), dtype=bool)
    h = (0.15, 0.15)
    ref = sm.dense_gamma(y, mask, m, h, h)
    cnt, W, V, V2 = sm.bin_mean_dense(y, mask, m)
    sig, _ = ov.sigma2_curve(m, h, cnt, W, V2, ref["mu"], np.diag(ref["gamma"]))
    est = ov.sigma2_scalar(sig, cnt > 0)
    assert abs(est - sigma ** 2) < 0.08 * sigma ** 2, est
