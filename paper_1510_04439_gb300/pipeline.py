"""The dense FPCA path as a sequence of C-ABI calls (allocation and marshalling only).

Steps (all in libfpca.so kernels):
  fpca_bin_mean -> fpca_smooth_mean -> fpca_bin_cov -> fpca_smooth_cov_project
  -> fpca_rproj_eig
Torch provides device memory and the stream; no arithmetic of the method runs
in Python.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import binding as B


@dataclass
class DenseBuffers:
    cnt: object
    w: object
    v: object
    v2: object
    mu: object
    mu_status: object
    ccnt: object
    cw: object
    cv: object
    gamma: object
    status: object
    evals: object
    evecs: object
    fve: object


def alloc_dense(torch, device, P, k, bin_prec, smooth_prec):
    f = torch.float64 if smooth_prec == B.F64 else torch.float32
    fb = torch.float64 if bin_prec == B.F64 else torch.float32
    z = lambda *s, dt=torch.float64: torch.empty(*s, dtype=dt, device=device)  # noqa: E731
    return DenseBuffers(
        cnt=z(P, dt=torch.int32), w=z(P), v=z(P), v2=z(P), mu=z(P),
        mu_status=z(P, dt=torch.uint8),
        ccnt=z(P, P, dt=torch.int32), cw=z(P, P, dt=fb), cv=z(P, P, dt=fb),
        gamma=z(P, P, dt=f), status=z(P, P, dt=torch.uint8),
        evals=z(k), evecs=z(k, P), fve=z(k))


def run_dense(ctx, m, y, mask, h_mu, h_cov, k, bufs, bin_prec=B.BF16, smooth_prec=B.F32,
              omega=None, power_iters=2, full=False, mode=B.COV_RESIDUAL):
    """One pass of the dense path; results land in ``bufs`` (device tensors)."""
    data = ctx.dense(y, mask)
    ctx.bin_mean(data, m, bufs.cnt, bufs.w, bufs.v, bufs.v2)
    ctx.smooth_mean(m, bufs.cnt, bufs.w, bufs.v, h_mu, bufs.mu, bufs.mu_status)
    ctx.bin_cov(data, m, bufs.mu, bin_prec, bufs.ccnt, bufs.cw, bufs.cv, mode=mode)
    ctx.smooth_cov_project(m, bufs.ccnt, bufs.cw, bufs.cv, [list(h_cov)], smooth_prec,
                           mu_raw=bufs.mu if mode == B.COV_RAW else None,
                           gamma=bufs.gamma, status=bufs.status)
    ctx.rproj_eig(m, bufs.gamma, k, bufs.evals, bufs.evecs, bufs.fve, domain=bufs.cnt,
                  omega=omega, power_iters=power_iters, full=full)
    return bufs


@dataclass
class SparseCVBuffers:
    cnt: object
    w: object
    v: object
    mu: object
    ccnt: object
    cw: object
    cv_: object
    cq: object
    scores: object


def alloc_sparse_cv(torch, device, P, nfold, nh):
    z = lambda *s, dt=torch.float64: torch.empty(*s, dtype=dt, device=device)  # noqa: E731
    return SparseCVBuffers(
        cnt=z(P, dt=torch.int32), w=z(P), v=z(P), mu=z(P),
        ccnt=z(nfold, P, P, dt=torch.int32), cw=z(nfold, P, P, dt=torch.float32),
        cv_=z(nfold, P, P, dt=torch.float32), cq=z(nfold, P, P, dt=torch.float32),
        scores=z(nh))


def run_sparse_cv(ctx, m, offs, t, y, fold, nfold, h_mu, hs, bufs, prec=B.F32C):
    """Mean bins and fit, fold-split covariance bins, and the CV score of every
    isotropic bandwidth in ``hs`` (one smoothing pass per bandwidth and fold)."""
    data = ctx.sparse(offs, t, y)
    ctx.bin_mean(data, m, bufs.cnt, bufs.w, bufs.v)
    ctx.smooth_mean(m, bufs.cnt, bufs.w, bufs.v, h_mu, bufs.mu)
    ctx.bin_cov(data, m, bufs.mu, B.F32, bufs.ccnt, bufs.cw, bufs.cv_, q=bufs.cq, fold=fold,
                nfold=nfold)
    d = len(m)
    ctx.smooth_cov_project(m, bufs.ccnt, bufs.cw, bufs.cv_, [[h] * d for h in hs], prec,
                           q=bufs.cq, nfold=nfold, cv=bufs.scores)
    return bufs
