"""GPU trust-region bandwidth search (Section 3.3) against the FP64 oracle's run of
the same steps on the oracle's CV score."""
import math

import numpy as np
import pytest

import fpca_synth as fs
from oracle import cv as ocv
from oracle import smoother as sm
from oracle import trust as otr

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


def _bins():
    D = fs.make_sparse(2, (8, 8), 400, [2.0, 1.0], nmin=3, nmax=12, sigma=0.4, seed=77, nfold=5)
    mu = np.linspace(-0.2, 0.3, D.P)
    r = sm.residuals_sparse(D.t, D.y, mu, D.m)
    return D.m, sm.bin_cov_sparse(D.offs, D.t, r, D.m, D.fold, 5)


def test_trust_region_follows_the_oracle_step_by_step(ctx):
    from paper_1510_04439_gb300 import binding as B
    m, (C, W, V, Q) = _bins()
    opts = {"max_iter": 4}
    h, cv, trace = ctx.bw_trust_region(m, dev(C, torch.int32), dev(W), dev(V), dev(Q), 5, B.F64,
                                       (0.3, 0.3), options=opts)

    def f(points):
        return [ocv.cv_score(m, list(np.exp(p)), C, W, V, Q) for p in points]
    x_ref, cv_ref, tr_ref = otr.trust_region_search(f, np.log([0.3, 0.3]), 2, opts)
    assert len(trace) == len(tr_ref)
    for (hg, vg), (xr, vr) in zip(trace, tr_ref):
        assert np.allclose(hg, np.exp(xr), rtol=1e-9)
        assert (math.isinf(vg) and math.isinf(vr)) or math.isclose(vg, vr, rel_tol=1e-9)
    assert np.allclose(h, np.exp(x_ref), rtol=1e-9)
    assert math.isclose(cv, cv_ref, rel_tol=1e-9)
    # the search improves on its start
    assert cv <= trace[0][1]


def test_trust_region_refusals(ctx):
    from paper_1510_04439_gb300 import binding as B
    m, (C, W, V, Q) = _bins()
    with pytest.raises(B.FpcaError):   # an infinite CV score at the start (h far too small)
        ctx.bw_trust_region(m, dev(C, torch.int32), dev(W), dev(V), dev(Q), 5, B.F64,
                            (0.001, 0.001), options={"h_lo": 0.0005})
    with pytest.raises(B.FpcaError):   # inconsistent options
        ctx.bw_trust_region(m, dev(C, torch.int32), dev(W), dev(V), dev(Q), 5, B.F64,
                            (0.3, 0.3), options={"h_lo": 0.5, "h_hi": 0.1})
