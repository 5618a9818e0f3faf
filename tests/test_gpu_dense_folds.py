"""FP32 fold-split covariance bins of gridded data (fpca_bin_cov, FPCA_DENSE,
FPCA_F32) against the oracle.

The kernel puts subjects in fold order and forms each fold's four Gram matrices
C = M'M, W = M' D M, V = R' D R, Q = (R^2)' D (R^2) (D the fold's pair weights
1/(N_i(N_i - 1))) on CUDA cores, 128 x 128 outputs per block, upper tile pairs
only and the lower ones as transposes.  The oracle is the pair-by-pair
definition (oracle/smoother.py: bin_cov_sparse over the observed nodes listed as
points, which also gives Q) on small cases, and bin_cov_dense per fold (the
Gram form, pinned to the pair loop) at the 64 x 64 size.

Tolerances: counts bit-exact; W, V, Q within FP32 summation error,
rtol 2e-6 with atol 2e-6 of the largest magnitude (the bar of the scattered FP32
binning).  Cases: ragged last tiles (P = 143, 576), P % 4 != 0 (scalar stores),
no folds, empty folds, subjects with N_i < 2, no mask, FP32 y, and the full
64 x 64 grid with 5 folds.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import smoother as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_1510_04439_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    return B.Context(0)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def host(t):
    return t.cpu().numpy()


def as_points(D, r):
    """The observed nodes of gridded data as scattered points (subject order)."""
    c = fs.grid_centres(D.m)
    mk = D.mask.astype(bool)
    Ni = mk.sum(axis=1)
    offs = np.zeros(len(Ni) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(Ni)
    rows, cols = np.nonzero(mk)
    return offs, c[cols], r[rows, cols]


def close(a, b, tol=2e-6):
    a = a.astype(np.float64)
    return np.allclose(a, b, rtol=tol, atol=tol * max(np.abs(b).max(), 1e-300))


def run(ctx, B, D, mu, nfold, fold, y_dtype=torch.float64, with_mask=True, with_q=True):
    P = D.P
    F = max(nfold, 1)
    C = torch.empty(F, P, P, dtype=torch.int32, device=DEV)
    W, V, Q = (torch.empty(F, P, P, dtype=torch.float32, device=DEV) for _ in range(3))
    y = dev(D.y, y_dtype)
    data = ctx.dense(y, dev(D.mask) if with_mask else None)
    ctx.bin_cov(data, D.m, dev(mu), B.F32, C, W, V, q=Q if with_q else None,
                fold=None if nfold == 0 else dev(fold, torch.int32), nfold=nfold)
    ctx.sync()
    return host(C), host(W), host(V), host(Q)


@pytest.mark.parametrize("m,nfold", [((13, 11), 5), ((13, 11), 0), ((24, 24), 3)])
def test_dense_fold_bins_vs_pair_definition(ctx, B, m, nfold):
    D = fs.make_dense(2, m, 37, [2.0, 1.0], sigma=0.4, seed=41, domain="disk", dropout=0.3)
    D.mask[3, :] = 0                      # a subject with no observation
    D.mask[5, :] = 0
    D.mask[5, 7] = 1                      # and one with a single observation
    mu = np.linspace(-0.3, 0.4, D.P)
    fold = np.random.default_rng(2).integers(0, max(nfold, 1), size=D.y.shape[0]).astype(np.int32)
    C, W, V, Q = run(ctx, B, D, mu, nfold, fold)
    r = sm.residuals_dense(D.y, D.mask, mu)
    offs, t, rr = as_points(D, r)
    rC, rW, rV, rQ = sm.bin_cov_sparse(offs, t, rr, D.m, fold if nfold else None, nfold)
    assert np.array_equal(C, rC)
    assert close(W, rW) and close(V, rV) and close(Q, rQ)


def test_dense_fold_bins_empty_folds_no_mask_f32_y(ctx, B):
    """Every subject in fold 2 of 4 (folds 0, 1, 3 empty: all-zero slices), fully
    observed data without a mask, FP32 responses, no q."""
    D = fs.make_dense(2, (8, 16), 21, [2.0, 1.0], sigma=0.4, seed=5)
    mu = np.zeros(D.P)
    fold = np.full(D.y.shape[0], 2, dtype=np.int32)
    C, W, V, _ = run(ctx, B, D, mu, 4, fold, y_dtype=torch.float32, with_mask=False,
                     with_q=False)
    for f in (0, 1, 3):
        assert not C[f].any() and not W[f].any() and not V[f].any()
    y32 = D.y.astype(np.float32).astype(np.float64)
    rC, rW, rV = sm.bin_cov_dense(y32, np.ones_like(D.mask))
    assert np.array_equal(C[2], rC)
    assert close(W[2], rW) and close(V[2], rV)


def test_dense_fold_bins_64x64_five_folds(ctx, B):
    """The 64 x 64 disk grid (32 tiles a side) with 5 folds against the oracle's
    Gram form, fold by fold."""
    D = fs.make_dense(2, (64, 64), 300, [4.0, 2.0, 1.0], sigma=0.5, seed=8, domain="disk",
                      dropout=0.2)
    mu = np.sin(np.linspace(0.0, 3.0, D.P))
    fold = (np.random.default_rng(9).permutation(300) % 5).astype(np.int32)
    C, W, V, _ = run(ctx, B, D, mu, 5, fold, with_q=False)
    r = sm.residuals_dense(D.y, D.mask, mu)
    for f in range(5):
        sel = fold == f
        rC, rW, rV = sm.bin_cov_dense(r[sel], D.mask[sel])
        assert np.array_equal(C[f], rC)
        assert close(W[f], rW) and close(V[f], rV)


def test_dense_fold_bins_reject_bad_arguments(ctx, B):
    D = fs.make_dense(2, (8, 8), 10, [1.0], seed=1)
    P = D.P
    C = torch.empty(2, P, P, dtype=torch.int32, device=DEV)
    W = torch.empty(2, P, P, dtype=torch.float32, device=DEV)
    data = ctx.dense(dev(D.y), dev(D.mask))
    mu = torch.zeros(P, dtype=torch.float64, device=DEV)
    with pytest.raises(B.FpcaError) as e:           # folds need the fold ids
        ctx.bin_cov(data, D.m, mu, B.F32, C, W, W, nfold=2)
    assert e.value.status == B.E_INVALID_ARG
    with pytest.raises(B.FpcaError) as e:           # folds are FP32 only for gridded data
        ctx.bin_cov(data, D.m, mu, B.F64, C, W, W, fold=dev(np.zeros(10, np.int32)), nfold=2)
    assert e.value.status == B.E_UNSUPPORTED
