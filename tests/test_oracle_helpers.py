"""Pins of the oracle's small helpers against hand-worked values.

Matrixisation of Eq. 3.1 (symmetrised, NaN and out-of-domain rows/columns
zeroed), the eigenvector sign convention, the orthonormal range basis, the
Riemann rescaling, the dense eigensolver on a matrix of known spectrum, the
sparse residuals R_ij = Y_ij - mu_hat(bin of t_ij) of Section 2, and the FP16
rounding of the bandwidth network's weights (biases kept).
"""
import math

import numpy as np
import pytest

from oracle import eigen as oe
from oracle import mlp as om
from oracle import smoother as sm


def test_matrixize_by_hand():
    G = np.array([[1.0, 2.0, np.nan],
                  [4.0, 5.0, 6.0],
                  [7.0, 8.0, 9.0]])
    S = oe.matrixize(G, np.array([True, True, False]))
    # (G + G')/2 with NaN -> 0, then row and column 2 zeroed
    want = np.array([[1.0, 3.0, 0.0],
                     [3.0, 5.0, 0.0],
                     [0.0, 0.0, 0.0]])
    assert np.array_equal(S, want)
    S = oe.matrixize(G, np.ones(3, bool))
    assert S[0, 2] == S[2, 0] == 3.5          # (0 + 7) / 2: the NaN counts as 0
    assert S[1, 2] == S[2, 1] == 7.0


def test_sign_convention_first_largest_entry_positive():
    V = np.array([[0.1, -2.0, 0.0],
                  [-0.9, 2.0, 1.0],
                  [0.3, 0.5, -1.0]])
    F = oe.fix_signs(V)
    assert np.array_equal(F[:, 0], -V[:, 0])   # -0.9 is the largest magnitude
    assert np.array_equal(F[:, 1], -V[:, 1])   # tie -2 / 2: the first one decides
    assert np.array_equal(F[:, 2], V[:, 2])    # tie 1 / -1: the first one is positive


def test_orth_is_an_orthonormal_basis_of_the_range():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((9, 4)) @ np.diag([1.0, 1e-3, 10.0, 2.0])
    Q = oe.orth(Y)
    assert Q.shape == (9, 4)
    assert np.allclose(Q.T @ Q, np.eye(4), atol=1e-13)
    assert np.allclose(Q @ (Q.T @ Y), Y, atol=1e-12)
    # an orthonormal input is returned up to column signs
    E = np.eye(9)[:, [2, 5]]
    Qe = oe.orth(E)
    assert np.allclose(np.abs(Qe), E)


def test_rescale_and_cell_volume():
    m = (8, 4)
    assert oe.cell_volume(m) == 1.0 / 32.0
    lam, phi = oe.rescale(np.array([64.0]), np.full((32, 1), 1.0 / math.sqrt(32.0)), m)
    assert lam[0] == pytest.approx(2.0)
    assert np.allclose(phi, 1.0)               # the unit-norm constant vector -> phi = 1


def test_eig_full_on_a_known_spectrum():
    # Sigma = sum_j theta_j u_j u_j' with orthonormal u_j, one node outside Omega
    m = (5,)
    U = np.zeros((5, 3))
    U[[0, 1], 0] = [3 / 5, 4 / 5]
    U[[0, 1], 1] = [-4 / 5, 3 / 5]
    U[2, 2] = -1.0
    theta = np.array([2.0, 5.0, 1.0])
    G = U @ np.diag(theta) @ U.T
    G[3, 3] = 7.0                              # node 3 outside the domain: dropped
    dom = np.array([True, True, True, False, True])
    lam, phi, fve = oe.eig_full(G, m, dom, 3)
    dv = 1.0 / 5.0
    assert np.allclose(lam, np.array([5.0, 2.0, 1.0]) * dv)
    # largest-magnitude entry made positive: (-4/5, 3/5) -> (4/5, -3/5)
    assert np.allclose(phi[:, 0], np.array([4 / 5, -3 / 5, 0, 0, 0]) / math.sqrt(dv))
    assert np.allclose(phi[:, 1], np.array([3 / 5, 4 / 5, 0, 0, 0]) / math.sqrt(dv))
    assert np.allclose(phi[:, 2], np.array([0, 0, 1.0, 0, 0]) / math.sqrt(dv))  # sign flipped
    assert np.allclose(fve, np.cumsum([5.0, 2.0, 1.0]) / 8.0)


def test_sparse_residuals_use_the_bin_of_each_time():
    m = (4,)
    mu = np.array([10.0, 20.0, 30.0, 40.0])
    t = np.array([[0.0], [0.26], [0.49], [0.999]])    # bins 0, 1, 1, 3 of width 1/4
    y = np.array([1.0, 2.0, 3.0, 4.0])
    r = sm.residuals_sparse(t, y, mu, m)
    assert np.array_equal(r, np.array([-9.0, -18.0, -17.0, -36.0]))


def test_fp16_rounding_of_weights_only():
    theta = np.full(om.param_count(), 1.0 + 2.0 ** -12)   # not representable in FP16
    t16 = om.fp16_weights(theta)
    off = 0
    for fi, fo in om.LAYERS:
        assert np.all(t16[off:off + fi * fo] == 1.0)                       # rounded
        assert np.all(t16[off + fi * fo:off + fi * fo + fo] == theta[0])  # bias kept
        off += fi * fo + fo
    assert off == om.param_count()
