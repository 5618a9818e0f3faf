"""Pins of the trust-region bandwidth search oracle (Section 3.3)."""
import itertools
import math

import numpy as np

from oracle import trust as otr


def test_box_qp_is_the_box_minimum():
    """Against a dense grid search, for definite, indefinite and singular quadratics."""
    rng = np.random.default_rng(1)
    for d in (1, 2):
        for trial in range(40):
            A = rng.standard_normal((d, d))
            H = A + A.T if trial % 3 else A @ A.T
            if trial % 7 == 0:
                H[:] = 0.0   # linear model: a vertex wins
            g = rng.standard_normal(d)
            lo = -rng.random(d)
            hi = rng.random(d)
            u = otr.box_qp(g, H, lo, hi)
            assert np.all(u >= lo - 1e-12) and np.all(u <= hi + 1e-12)
            grid = [np.linspace(lo[k], hi[k], 201) for k in range(d)]
            best = min(g @ np.array(p) + 0.5 * np.array(p) @ H @ np.array(p)
                       for p in itertools.product(*grid))
            assert g @ u + 0.5 * u @ H @ u <= best + 1e-9


def test_regression_recovers_a_quadratic():
    rng = np.random.default_rng(2)
    beta = rng.standard_normal(6)
    c, g, H = otr.unpack(beta, 2)
    pts = [np.array(v) for v in itertools.product((-1.0, 0.0, 1.0), repeat=2)]
    rows = np.array([otr.quad_terms(p) for p in pts])
    ys = np.array([otr.qval(c, g, H, p) for p in pts])
    fit = np.linalg.lstsq(rows, ys, rcond=None)[0]
    assert np.allclose(fit, beta, atol=1e-12)


def _batch(fun):
    return lambda pts: [fun(np.asarray(p)) for p in pts]


def test_convex_quadratic_minimum_inside_the_box():
    xs = np.log(np.array([0.11, 0.07]))
    A = np.array([[3.0, 0.8], [0.8, 1.5]])
    f = _batch(lambda x: 2.0 + (x - xs) @ A @ (x - xs))
    x, fx, trace = otr.trust_region_search(f, np.log([0.3, 0.3]), 2)
    assert np.allclose(x, xs, atol=2e-3), (x, xs)
    assert fx <= 2.0 + 1e-4
    pts = [tuple(p) for p, _ in trace]
    assert len(pts) == len(set(pts))        # every point evaluated once


def test_minimum_outside_the_box_lands_on_its_edge():
    f = _batch(lambda x: float(np.sum((x - math.log(0.01)) ** 2)))
    x, _, _ = otr.trust_region_search(f, np.log([0.2, 0.2]), 2)
    assert np.allclose(x, math.log(0.02), atol=1e-12)


def test_noisy_quadratic_and_infinite_region():
    """Noise of 1e-3 on a unit-curvature bowl, CV = inf below h = 0.04 (EMPTY points)."""
    rng = np.random.default_rng(3)
    xs = np.log(np.array([0.09, 0.15]))

    def fun(x):
        if np.any(np.exp(x) < 0.04):
            return math.inf
        return float((x - xs) @ (x - xs)) + 1e-3 * rng.standard_normal()
    x, _, _ = otr.trust_region_search(_batch(fun), np.log([0.3, 0.3]), 2)
    assert np.max(np.abs(x - xs)) < 0.15, (np.exp(x), np.exp(xs))


def test_one_dimension():
    f = _batch(lambda x: float((x[0] - math.log(0.13)) ** 2))
    x, _, _ = otr.trust_region_search(f, np.array([math.log(0.5)]), 1)
    assert abs(x[0] - math.log(0.13)) < 2e-3
