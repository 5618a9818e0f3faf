"""Oracle: derivative-free trust-region bandwidth search (Section 3.3), FP64.

Test infrastructure only: the library never imports this module.

Section 3.3 proposes to minimise the noisy CV criterion over the bandwidth
vector with the derivative-free trust-region method of Marazzi and Nocedal,
the gradient and Hessian coming from a local quadratic model, fitted by
least-squares regression instead of interpolation so that noise is averaged.
The paper gives no further detail; the reading below fixes every step.

Reading
-------
* Variables x = log h (one per axis, d <= 2), kept in the box
  [log h_lo, log h_hi]^d.  f(x) = CV(exp(x)); evaluations are cached by point.
* Trust region: the box |x - x_k|_inf <= Delta_k (Delta_0 = 0.4, in log units).
* Each iteration samples the 3^d stencil x_k + Delta_k v, v in {-1, 0, 1}^d
  (ordered lexicographically, clipped to the box, duplicates dropped) and fits
  q(u) = c + g'u + u'Hu/2 in u = (x - x_k)/Delta_k by least squares on the
  finite values.  Fewer finite values than parameters: Delta halves.
* The step minimises q over the trust-region box intersected with the bounds,
  exactly: every active set (each coordinate free, at its lower or at its upper
  bound) is tried, its stationary point kept when it is feasible, the smallest
  value wins (first in enumeration order on ties).
* pred = q(0) - q(u*) <= 0: Delta halves.  Otherwise the trial point is
  evaluated, rho = (f(x_k) - f(x_t)) / pred; rho >= 0.1 accepts it; rho < 0.25
  halves Delta, rho > 0.75 with a step on the trust-region boundary
  (|u*|_inf > 0.99) doubles it up to Delta_max = 1.
* Stop when Delta < Delta_min = 0.01 or after max_iter = 20 iterations; the
  result is the best point evaluated (lowest finite CV, first on ties).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

DEFAULTS = dict(delta0=0.4, delta_min=0.01, delta_max=1.0, h_lo=0.02, h_hi=0.6, max_iter=20)


def quad_terms(u):
    """Regression row of q at u: 1, u_k, then u_i u_j / 2 (i == j) or u_i u_j (i < j)."""
    d = len(u)
    row = [1.0] + [float(x) for x in u]
    for i in range(d):
        for j in range(i, d):
            row.append(0.5 * u[i] * u[i] if i == j else u[i] * u[j])
    return row


def unpack(beta, d):
    """c, g, H from the regression coefficients."""
    c = beta[0]
    g = np.array(beta[1:1 + d])
    H = np.zeros((d, d))
    k = 1 + d
    for i in range(d):
        for j in range(i, d):
            H[i, j] = H[j, i] = beta[k]
            k += 1
    return c, g, H


def qval(c, g, H, u):
    u = np.asarray(u, dtype=np.float64)
    return c + g @ u + 0.5 * u @ H @ u


def box_qp(g, H, lo, hi):
    """argmin over lo <= u <= hi of g'u + u'Hu/2 by enumerating active sets."""
    d = len(g)
    best, best_u = math.inf, None
    for state in itertools.product((0, 1, 2), repeat=d):   # 0 free, 1 lower, 2 upper
        u = np.zeros(d)
        free = [k for k in range(d) if state[k] == 0]
        for k in range(d):
            if state[k] == 1:
                u[k] = lo[k]
            elif state[k] == 2:
                u[k] = hi[k]
        if free:
            bound = [k for k in range(d) if state[k] != 0]
            Hff = H[np.ix_(free, free)]
            rhs = -(g[free] + (H[np.ix_(free, bound)] @ u[bound] if bound else 0.0))
            if abs(np.linalg.det(Hff)) < 1e-12 * max(1.0, np.abs(Hff).max()) ** len(free):
                continue
            u[free] = np.linalg.solve(Hff, rhs)
            if np.any(u[free] < lo[free] - 1e-12) or np.any(u[free] > hi[free] + 1e-12):
                continue
        v = g @ u + 0.5 * u @ H @ u
        if v < best:
            best, best_u = v, u.copy()
    return best_u


def trust_region_search(f, x0, d, options=None):
    """Minimise f over log-bandwidths; returns (x_best, f_best, trace).

    f maps a list of points (arrays of length d) to their values; trace lists
    every evaluated (x, f(x)) in evaluation order.
    """
    o = dict(DEFAULTS)
    if options:
        o.update(options)
    lo = np.full(d, math.log(o["h_lo"]))
    hi = np.full(d, math.log(o["h_hi"]))
    cache, trace = {}, []

    def evaluate(points):
        new = [p for p in points if tuple(p) not in cache]
        uniq = []
        for p in new:
            if all(tuple(p) != tuple(q) for q in uniq):
                uniq.append(p)
        if uniq:
            vals = f(uniq)
            for p, v in zip(uniq, vals):
                cache[tuple(p)] = float(v)
                trace.append((np.array(p), float(v)))
        return [cache[tuple(p)] for p in points]

    x = np.clip(np.asarray(x0, dtype=np.float64), lo, hi)
    delta = o["delta0"]
    fx = evaluate([x])[0]
    if not math.isfinite(fx):
        raise ValueError("the starting bandwidth has an infinite CV score")
    npar = (d + 1) * (d + 2) // 2
    for _ in range(o["max_iter"]):
        if delta < o["delta_min"]:
            break
        pts = []
        for v in itertools.product((-1.0, 0.0, 1.0), repeat=d):
            p = np.clip(x + delta * np.array(v), lo, hi)
            if all(tuple(p) != tuple(q) for q in pts):
                pts.append(p)
        vals = evaluate(pts)
        rows = [quad_terms((p - x) / delta) for p, v in zip(pts, vals) if math.isfinite(v)]
        ys = [v for v in vals if math.isfinite(v)]
        if len(ys) < npar:
            delta *= 0.5
            continue
        beta = np.linalg.lstsq(np.array(rows), np.array(ys), rcond=None)[0]
        c, g, H = unpack(beta, d)
        ulo = np.maximum(-1.0, (lo - x) / delta)
        uhi = np.minimum(1.0, (hi - x) / delta)
        u = box_qp(g, H, ulo, uhi)
        pred = -math.inf if u is None else qval(c, g, H, np.zeros(d)) - qval(c, g, H, u)
        if not pred > 0.0:
            delta *= 0.5
            continue
        xt = x + delta * u
        ft = evaluate([xt])[0]
        rho = (fx - ft) / pred if math.isfinite(ft) else -math.inf
        if rho >= 0.1:
            x, fx = xt, ft
        if rho < 0.25:
            delta *= 0.5
        elif rho > 0.75 and np.max(np.abs(u)) > 0.99:
            delta = min(2.0 * delta, o["delta_max"])
    best = min((v, k) for k, (p, v) in enumerate(trace) if math.isfinite(v))
    return trace[best[1]][0], best[0], trace
