"""Oracle: the bandwidth-proposal network, FP64 (test infrastructure only).

The paper selects bandwidths by cross-validation over candidate values
(Section 3.3) and notes that a grid search is expensive.  The network here
regresses the CV-optimal log bandwidths from a 32-number summary of a
dataset's bins, so that one smoothing pass at the proposed bandwidth (plus a
CV check) can replace the grid.

Architecture: 32 -> 256 -> 256 -> 256 -> 6, exact GELU
gelu(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2)) after each hidden layer,
linear output.  Weights are used rounded to FP16 (the GPU stores them so);
all arithmetic here is FP64.

Loss: masked mean squared error, L = sum_bj m_bj (o_bj - y_bj)^2 / sum_bj m_bj.
Optimiser: AdamW (decoupled weight decay), bias-corrected moments.

Parameter vector layout (shared with the GPU): for each layer in order,
W (fan_in x fan_out, row-major) then b (fan_out).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYERS = [(32, 256), (256, 256), (256, 256), (256, 6)]
NFEAT = 32
NOUT = 6


def param_count():
    return sum(i * o + o for i, o in LAYERS)


def unpack(theta):
    """Split the flat parameter vector into [(W, b), ...]."""
    out = []
    off = 0
    for fi, fo in LAYERS:
        W = theta[off:off + fi * fo].reshape(fi, fo)
        off += fi * fo
        b = theta[off:off + fo]
        off += fo
        out.append((W, b))
    return out


def fp16_weights(theta):
    """The parameter vector with weights (not biases) rounded to FP16."""
    t = np.array(theta, dtype=np.float64, copy=True)
    off = 0
    for fi, fo in LAYERS:
        t[off:off + fi * fo] = t[off:off + fi * fo].astype(np.float16).astype(np.float64)
        off += fi * fo + fo
    return t


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """Output (B x 6) and the cache of pre-activations and activations."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    cache = [h]
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        if li < len(layers) - 1:
            cache.append(z)
            h = gelu(z)
            cache.append(h)
        else:
            h = z
    return h, cache


def loss_and_grad(theta, X, Y, M):
    """Masked MSE and its gradient with respect to the flat parameters."""
    theta = np.asarray(theta, dtype=np.float64)
    out, cache = forward(theta, X)
    M = np.asarray(M, dtype=np.float64)
    denom = max(M.sum(), 1.0)
    diff = (out - Y) * M
    loss = float(np.sum(diff * (out - Y)) / denom)
    g_out = 2.0 * diff / denom
    layers = unpack(theta)
    grads = []
    delta = g_out
    nl = len(layers)
    for li in range(nl - 1, -1, -1):
        W, b = layers[li]
        h_in = cache[0] if li == 0 else cache[2 * li]
        gW = h_in.T @ delta
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            z_prev = cache[2 * li - 1]
            delta = (delta @ W.T) * gelu_grad(z_prev)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adamw_step(theta, m, v, grad, step, lr, wd=1e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update (decoupled weight decay on every parameter)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
