"""Learned bandwidth proposal: labels, training and evaluation (GPU).

Section 3.3 selects bandwidths by cross-validation and calls grid search
expensive.  Here a small network (fpca_bw_predict / fpca_bw_train_step)
proposes the CV-optimal covariance bandwidth from 32 summary numbers of the
binned data (fpca_bw_features); a CV check at the proposal and two
neighbours (h x {0.8, 1, 1.25}) replaces the 16-bandwidth grid, and the grid
is kept as the fallback when a neighbour beats the proposal by more than 5%.

Everything numerical runs in libfpca.so kernels through the ABI; this module
draws datasets (fpca_synth), moves arrays and runs the training loop.

Labels: the argmin of the 5-fold subject-level CV score over 16 isotropic
bandwidths log-spaced in [0.03, 0.3] (covariance smoother).  Output entries
3..5 (log h_Gamma per axis) carry the label for axes < d; the mean-bandwidth
entries 0..2 are masked (no CV of the mean smoother is built).

CLI:  python -m paper_1510_04439_gb300.bandwidth --train 2000 --eval 200 --out run.npz
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding as B
from . import pipeline

HGRID = np.exp(np.linspace(math.log(0.03), math.log(0.3), 16))
NFOLD = 5


def draw_dataset(seed):
    """One synthetic dataset from the workload generators (d = 1 or 2, n log-uniform,
    sigma uniform in [0.1, 1.0]), returned in scattered (offsets) form."""
    import fpca_synth as fs
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 3))
    sigma = float(rng.uniform(0.1, 1.0))
    kind = rng.choice(["dense", "sparse"])
    if d == 1:
        m = (64,)
        lam = [4.0, 2.0, 1.0, 0.5][: int(rng.integers(2, 5))]
        mean = "1d"
    else:
        m = (32, 32)
        lam = [8.0 * 2.0 ** (-k) for k in range(int(rng.integers(2, 7)))]
        mean = "sincos"
    if kind == "dense":
        n = int(np.exp(rng.uniform(math.log(50), math.log(2000))))
        D = fs.make_dense(d, m, n, lam, sigma=sigma, mean=mean, seed=seed,
                          domain="disk" if (d == 2 and rng.random() < 0.5) else "full",
                          dropout=float(rng.choice([0.0, 0.1, 0.3])))
        c = fs.grid_centres(m)
        Ni = D.mask.sum(axis=1).astype(np.int64)
        offs = np.zeros(n + 1, dtype=np.int64)
        offs[1:] = np.cumsum(Ni)
        rows, cols = np.nonzero(D.mask)
        t = c[cols]
        y = D.y[rows, cols]
    else:
        n = int(np.exp(rng.uniform(math.log(200), math.log(20000))))
        D = fs.make_sparse(d, m, n, lam, sigma=sigma, mean=mean, seed=seed, nfold=0)
        offs, t, y = D.offs, D.t, D.y
    fold = (np.random.default_rng(seed + 7).permutation(n) % NFOLD).astype(np.int32)
    return dict(d=d, m=m, offs=offs, t=np.ascontiguousarray(t), y=np.ascontiguousarray(y),
                fold=fold, specs=D.specs, lam=np.asarray(lam), seed=seed)


class Labeller:
    """GPU bins, features, CV scores and final FPCA fits of datasets on one context."""

    def __init__(self, ctx, torch):
        self.ctx = ctx
        self.torch = torch
        self.dev = ctx.device

    def upload(self, ds):
        return {k: self.torch.from_numpy(ds[k]).to(self.dev) for k in ("offs", "t", "y", "fold")}

    def prepare(self, ds, tensors=None, features=True):
        """Mean bins and fit, fold-split covariance bins, and (optionally) the features."""
        torch = self.torch
        m = ds["m"]
        P = int(np.prod(m))
        bufs = pipeline.alloc_sparse_cv(torch, self.dev, P, NFOLD, len(HGRID))
        t = tensors if tensors is not None else self.upload(ds)
        data = self.ctx.sparse(t["offs"], t["t"], t["y"])
        v2 = torch.empty_like(bufs.w)
        self.ctx.bin_mean(data, m, bufs.cnt, bufs.w, bufs.v, v2)
        hmu = [0.1] * len(m)
        self.ctx.smooth_mean(m, bufs.cnt, bufs.w, bufs.v, hmu, bufs.mu)
        self.ctx.bin_cov(data, m, bufs.mu, B.F32, bufs.ccnt, bufs.cw, bufs.cv_, q=bufs.cq,
                         fold=t["fold"], nfold=NFOLD)
        prep = dict(bufs=bufs, tensors=t, data=data, m=m, d=len(m), v2=v2, feat=None)
        if features:
            self.features(prep)
        return prep

    def features(self, prep):
        b = prep["bufs"]
        feat = self.torch.empty(32, dtype=self.torch.float32, device=self.dev)
        self.ctx.bw_features(prep["data"], prep["m"], b.cnt, b.w, b.v, prep["v2"], b.ccnt, b.cw,
                             b.cv_, feat, nfold=NFOLD)
        prep["feat"] = feat
        return feat

    def cv(self, prep, hs):
        """CV score of each isotropic bandwidth in hs (one pass per bandwidth and fold)."""
        torch = self.torch
        b = prep["bufs"]
        out = torch.empty(len(hs), dtype=torch.float64, device=self.dev)
        d = prep["d"]
        self.ctx.smooth_cov_project(prep["m"], b.ccnt, b.cw, b.cv_, [[float(h)] * d for h in hs],
                                    B.F32C, q=b.cq, nfold=NFOLD, cv=out)
        return out

    def fit(self, prep, h, k, omega):
        """Final covariance surface at bandwidth h on the pooled bins and its top-k
        eigenpairs by random projection (k + 10 columns, 2 power iterations)."""
        torch = self.torch
        b = prep["bufs"]
        m = prep["m"]
        P = int(np.prod(m))
        gamma = torch.empty(P, P, dtype=torch.float32, device=self.dev)
        self.ctx.smooth_cov_project(m, b.ccnt, b.cw, b.cv_, [[float(h)] * prep["d"]], B.F32C,
                                    nfold=NFOLD, gamma=gamma)
        evals = torch.empty(k, dtype=torch.float64, device=self.dev)
        evecs = torch.empty(k, P, dtype=torch.float64, device=self.dev)   # vector j in row j
        self.ctx.rproj_eig(m, gamma, k, evals, evecs, omega=omega, power_iters=2)
        return evals, evecs


def subspace_sine(a, b):
    """Largest principal-angle sine between the column spaces of a and b."""
    qa, _ = np.linalg.qr(a)
    qb, _ = np.linalg.qr(b)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(math.sqrt(max(0.0, 1.0 - float(np.min(s)) ** 2)))


def make_table(ctx, torch, seeds, log_every=0):
    """Features and CV-grid labels of datasets drawn with ``seeds``."""
    lab = Labeller(ctx, torch)
    feats, targets, masks, best = [], [], [], []
    t0 = time.time()
    for k, s in enumerate(seeds):
        ds = draw_dataset(int(s))
        prep = lab.prepare(ds)
        scores = lab.cv(prep, HGRID).cpu().numpy()
        fin = np.isfinite(scores)
        j = int(np.argmin(np.where(fin, scores, np.inf))) if fin.any() else len(HGRID) // 2
        tgt = np.zeros(6, np.float32)
        msk = np.zeros(6, np.uint8)
        for a in range(ds["d"]):
            tgt[3 + a] = math.log(HGRID[j])
            msk[3 + a] = 1
        feats.append(prep["feat"].cpu().numpy())
        targets.append(tgt)
        masks.append(msk if fin.any() else np.zeros(6, np.uint8))
        best.append(j)
        if log_every and (k + 1) % log_every == 0:
            print(f"labelled {k + 1}/{len(seeds)} in {time.time() - t0:.1f} s", flush=True)
    return (np.stack(feats), np.stack(targets), np.stack(masks), np.array(best))


def standardize(X, mu=None, sd=None):
    if mu is None:
        mu = X.mean(0)
        sd = X.std(0)
        sd[sd == 0] = 1.0
    return (X - mu) / sd, mu, sd


def train(ctx, torch, X, Y, M, epochs=200, batch=256, lr=1e-3, wd=1e-4, seed=0):
    """AdamW on (X, Y, M) with the GPU kernels; returns params and loss history."""
    dev = ctx.device
    th = torch.empty(ctx.bw_param_count(), dtype=torch.float32, device=dev)
    ctx.bw_mlp_init(th, seed)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    Yd = torch.from_numpy(Y.astype(np.float32)).to(dev)
    Md = torch.from_numpy(M.astype(np.uint8)).to(dev)
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    step = 0
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        for s in range(0, n, batch):
            idx = perm[s:s + batch]
            step += 1
            ctx.bw_train_step(th, m, v, step, Xd[idx].contiguous(), Yd[idx].contiguous(),
                              Md[idx].contiguous(), lr=lr, wd=wd, loss=loss)
        hist.append(float(loss.item()))
    return th, hist


def predict(ctx, torch, th, X):
    out = torch.empty(X.shape[0], 6, dtype=torch.float32, device=ctx.device)
    ctx.bw_predict(th, torch.from_numpy(X.astype(np.float32)).to(ctx.device), out)
    return out.cpu().numpy()


def evaluate(ctx, torch, th, mu, sd, seeds):
    """Per held-out dataset, the whole FPCA (bins, bandwidth choice, final surface and
    top-k eigenfunctions, k = the true number of components) by both methods:

      grid:    CV over the 16 bandwidths, fit at the best one;
      learned: features -> network -> CV check at h x {0.8, 1, 1.25} -> fit at the
               best checked bandwidth, or the grid when a neighbour beats the
               proposal by more than 5% (fallback).

    Records wall times of each stage (GPU work plus host overhead, synchronised),
    CV scores, and the eigenfunction subspace error of both fits against the truth."""
    import fpca_synth as fs
    lab = Labeller(ctx, torch)
    rows = []

    def clock():
        torch.cuda.synchronize()
        return time.perf_counter()

    for s in seeds:
        ds = draw_dataset(int(s))
        m = ds["m"]
        P = int(np.prod(m))
        k = len(ds["lam"])
        omega = torch.from_numpy(fs.gaussian_test_matrix(P, k + 10, int(s)).astype(np.float32)).to(ctx.device)
        tens = lab.upload(ds)
        t0 = clock()
        prep = lab.prepare(ds, tens, features=False)
        t1 = clock()
        grid = lab.cv(prep, HGRID).cpu().numpy()
        t2 = clock()
        fin = np.isfinite(grid)
        jb = int(np.argmin(np.where(fin, grid, np.inf))) if fin.any() else len(HGRID) // 2
        _, vec_g = lab.fit(prep, HGRID[jb], k, omega)
        vec_g = vec_g.cpu().numpy().T
        t3 = clock()
        feat = lab.features(prep).cpu().numpy()
        f = (feat[None, :] - mu) / sd
        out = predict(ctx, torch, th, f)[0]
        hp = float(np.exp(np.mean(out[3:3 + ds["d"]])))
        hp = float(np.clip(hp, HGRID[0], HGRID[-1]))
        cand = [hp * 0.8, hp, hp * 1.25]
        chk = lab.cv(prep, cand).cpu().numpy()
        t4 = clock()
        fallback = (not np.isfinite(chk[1])) or bool(min(chk[0], chk[2]) < 0.95 * chk[1])
        if fallback:
            h_l = float(HGRID[jb])       # the grid scores computed above stand in for a rerun
        else:
            h_l = float(cand[int(np.nanargmin(np.where(np.isfinite(chk), chk, np.nan)))])
        t5 = clock()
        _, vec_l = lab.fit(prep, h_l, k, omega)
        vec_l = vec_l.cpu().numpy().T
        t6 = clock()
        best = float(np.min(grid[fin])) if fin.any() else math.inf
        prop = float(np.nanmin(np.where(np.isfinite(chk), chk, np.nan))) if np.isfinite(chk).any() \
            else math.inf
        c = fs.grid_centres(m)
        phi = np.stack([fs.eval_fourier(sp, c) for sp in ds["specs"]], axis=1)
        t_prep, t_cv, t_fit_g = t1 - t0, t2 - t1, t3 - t2
        t_sel, t_fit_l = t4 - t3, t6 - t5
        rows.append(dict(
            seed=int(s), d=ds["d"], k=k, grid_best=best, grid_h=float(HGRID[jb]), prop_h=hp,
            prop_score=prop, fallback=fallback, final_h=h_l,
            final_score=best if fallback else prop,
            t_grid=t_cv, t_prop=t_sel,
            t_final=t_sel + (t_cv if fallback else 0.0),
            fpca_grid=t_prep + t_cv + t_fit_g,
            fpca_learned=t_prep + t_sel + (t_cv if fallback else 0.0) + t_fit_l,
            sine_grid=subspace_sine(vec_g, phi), sine_learned=subspace_sine(vec_l, phi)))
    return rows


def summarize(rows):
    """Share of datasets whose final CV score is within 5% of the grid optimum, mean
    wall times of both selections and of both whole FPCA runs, and the eigenfunction
    subspace errors of both fits."""
    ok = [r for r in rows if np.isfinite(r["grid_best"])]
    ratio = np.array([r["final_score"] / r["grid_best"] for r in ok])
    pratio = np.array([r["prop_score"] / r["grid_best"] for r in ok])
    sg = np.array([r["sine_grid"] for r in rows])
    sl = np.array([r["sine_learned"] for r in rows])
    mean = lambda key: float(np.mean([r[key] for r in rows]))  # noqa: E731
    return dict(n=len(rows), within5=float(np.mean(ratio <= 1.05)),
                median_ratio=float(np.median(ratio)), proposal_within5=float(np.mean(pratio <= 1.05)),
                fallback_rate=mean("fallback"), t_grid=mean("t_grid"), t_final=mean("t_final"),
                fpca_grid_s=mean("fpca_grid"), fpca_learned_s=mean("fpca_learned"),
                fpca_speedup=mean("fpca_grid") / mean("fpca_learned"),
                sine_grid_median=float(np.median(sg)), sine_learned_median=float(np.median(sl)),
                sine_grid_mean=float(np.mean(sg)), sine_learned_mean=float(np.mean(sl)),
                sine_worse_by_0p01=float(np.mean(sl > sg + 0.01)))


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--out", default="bandwidth_run.npz")
    ap.add_argument("--rows", default=None, help="write the per-dataset evaluation rows (JSON)")
    ap.add_argument("--table", default=None,
                    help="reuse the labelled table (X, Y, M, best) of an earlier run's output")
    a = ap.parse_args()
    ctx = B.Context(0)
    t0 = time.time()
    if a.table:
        z = np.load(a.table)
        X, Y, M, best = z["X"], z["Y"], z["M"], z["best"]
    else:
        X, Y, M, best = make_table(ctx, torch, np.arange(a.train), log_every=200)
    t_label = time.time() - t0
    Xs, mu, sd = standardize(X)
    t0 = time.time()
    th, hist = train(ctx, torch, Xs, Y, M, epochs=a.epochs)
    t_train = time.time() - t0
    rows = evaluate(ctx, torch, th, mu, sd, 10 ** 6 + np.arange(a.eval))
    summ = summarize(rows)
    summ.update(t_label=t_label, t_train=t_train, final_loss=hist[-1], first_loss=hist[0],
                train=int(X.shape[0]), epochs=a.epochs)
    np.savez(a.out, params=th.cpu().numpy(), mu=mu, sd=sd, X=X, Y=Y, M=M, best=best,
             loss=np.array(hist))
    if a.rows:
        with open(a.rows, "w") as fh:
            json.dump(rows, fh)
    print(json.dumps(summ), flush=True)


if __name__ == "__main__":
    main()
