"""Pins of the bandwidth-network oracle (CPU): central finite differences for
the manual backward pass, the GELU derivative, and the closed form of the
first AdamW step."""
import math

import numpy as np
import pytest

from oracle import mlp


def _problem(seed=0, B=7):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mlp.param_count()) * 0.05
    X = rng.standard_normal((B, mlp.NFEAT))
    Y = rng.standard_normal((B, mlp.NOUT))
    M = (rng.random((B, mlp.NOUT)) < 0.7).astype(float)
    return theta, X, Y, M


def test_param_count_and_layout():
    assert mlp.param_count() == 32 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 6 + 6
    theta = np.arange(mlp.param_count(), dtype=float)
    layers = mlp.unpack(theta)
    assert layers[0][0].shape == (32, 256) and layers[-1][1].shape == (6,)
    assert layers[1][0][0, 0] == 32 * 256 + 256


def test_gelu_grad_matches_numeric_derivative():
    z = np.linspace(-5, 5, 101)
    eps = 1e-6
    num = (mlp.gelu(z + eps) - mlp.gelu(z - eps)) / (2 * eps)
    assert np.max(np.abs(num - mlp.gelu_grad(z))) < 1e-8
    # gelu(z) = z Phi(z): exact values at 0 and the limit
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15


def _fd_check(loss_and_grad, seed=1, nprobe=60):
    theta, X, Y, M = _problem(seed)
    _, g = loss_and_grad(theta, X, Y, M)
    rng = np.random.default_rng(seed + 100)
    idx = rng.choice(theta.size, nprobe, replace=False)
    idx = np.concatenate([idx, [0, 32 * 256, theta.size - 1, theta.size - 7]])
    errs = []
    for i in idx:
        e = np.zeros_like(theta)
        h = 1e-6 * max(1.0, abs(theta[i]))
        e[i] = h
        lp, _ = loss_and_grad(theta + e, X, Y, M)
        lm, _ = loss_and_grad(theta - e, X, Y, M)
        num = (lp - lm) / (2 * h)
        errs.append(abs(num - g[i]) / max(1e-6, abs(num) + abs(g[i])))
    return max(errs)


def test_backward_matches_central_differences():
    # central differences with h = 1e-6 resolve relative errors to ~1e-5 here
    assert _fd_check(mlp.loss_and_grad) < 1e-4


def test_first_adamw_step_closed_form():
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, wd, eps = 1e-3, 1e-4, 1e-8
    t1, m1, v1 = mlp.adamw_step(theta, np.zeros(50), np.zeros(50), g, 1, lr, wd, eps=eps)
    # step 1: bias-corrected moments are g and g^2 exactly
    expect = theta - lr * (g / (np.abs(g) + eps) + wd * theta)
    assert np.allclose(t1, expect, rtol=1e-12, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_planted_wrong_gelu_derivative_fails(monkeypatch):
    monkeypatch.setattr(mlp, "gelu_grad", lambda z: 0.5 * (1.0 + np.tanh(z)))
    assert _fd_check(mlp.loss_and_grad) > 1e-3
