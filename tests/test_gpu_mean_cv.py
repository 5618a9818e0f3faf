"""Cross-validation of the mean smoother (fpca_smooth_mean_cv) against the oracle.

The oracle's score (oracle/cv.py mean_cv_score) is pinned on the CPU to the
held-out error summed observation by observation.  FP64 on both sides:
rel <= 1e-9, the same argmin, +inf at the same bandwidths.
"""
import numpy as np
import pytest

import fpca_synth as fs
from oracle import cv as ocv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("d,m,n", [(1, (64,), 300), (2, (16, 16), 800), (2, (64, 64), 4000)])
def test_mean_cv_matches_oracle(d, m, n):
    from paper_1510_04439_gb300 import binding as B
    ctx = B.Context(0)
    D = fs.make_sparse(d, m, n, [2.0, 1.0, 0.5], nmin=5, nmax=20, sigma=0.5, seed=31 + d, nfold=5,
                       mean="1d" if d == 1 else "sincos")
    hs = [0.03, 0.06, 0.12, 0.25, 0.5]
    data = ctx.sparse(torch.from_numpy(D.offs).to(DEV), torch.from_numpy(D.t).to(DEV),
                      torch.from_numpy(D.y).to(DEV))
    cv = torch.empty(len(hs), dtype=torch.float64, device=DEV)
    ctx.smooth_mean_cv(data, m, torch.from_numpy(D.fold.astype(np.int32)).to(DEV), 5, hs, cv)
    ctx.sync()
    bins = ocv.mean_fold_bins(D.offs, D.t, D.y, m, D.fold, 5)
    ref = np.array([ocv.mean_cv_score(m, [h] * d, *bins) for h in hs])
    got = cv.cpu().numpy()
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    fin = np.isfinite(ref)
    assert fin.sum() >= 3
    assert np.allclose(got[fin], ref[fin], rtol=1e-9)
    assert np.argmin(np.where(fin, got, np.inf)) == np.argmin(np.where(fin, ref, np.inf))


def test_mean_cv_rejects_dense_data():
    from paper_1510_04439_gb300 import binding as B
    ctx = B.Context(0)
    y = torch.zeros(4, 16, dtype=torch.float64, device=DEV)
    fold = torch.zeros(4, dtype=torch.int32, device=DEV)
    cv = torch.empty(1, dtype=torch.float64, device=DEV)
    with pytest.raises(B.FpcaError) as e:
        ctx.smooth_mean_cv(ctx.dense(y), (16,), fold, 2, [0.1], cv)
    assert e.value.status == B.E_UNSUPPORTED
