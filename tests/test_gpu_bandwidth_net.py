"""The bandwidth network and its input features on the GPU against the FP64 oracle.

Tolerances: forward outputs rel <= 1e-4, gradient rel-L2 <= 1e-3 (FP32
accumulation against FP64 at the same FP16-rounded weights), one AdamW step
rel <= 1e-5 where the gradient is not negligible, features abs <= 1e-4.
"""
import json

import numpy as np
import pytest

import fpca_synth as fs
from oracle import features as ofeat
from oracle import mlp as omlp
from oracle import smoother as sm

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


def host(t):
    return t.detach().cpu().numpy()


def init_params(seed):
    """He-style initial parameters drawn on the host (passed in as inputs)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in omlp.LAYERS:
        parts.append(rng.standard_normal(fi * fo) * np.sqrt(2.0 / fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts)


def test_param_count_matches_oracle(ctx):
    assert ctx.bw_param_count() == omlp.param_count()


def test_forward_and_gradient_vs_oracle(ctx):
    rng = np.random.default_rng(5)
    theta = init_params(1).astype(np.float32).astype(np.float64)
    B = 37
    X = rng.standard_normal((B, 32))
    Y = rng.standard_normal((B, 6))
    M = (rng.random((B, 6)) < 0.8).astype(np.uint8)
    th = dev(theta, torch.float32)
    out = torch.empty(B, 6, dtype=torch.float32, device=DEV)
    ctx.bw_predict(th, dev(X, torch.float32), out)
    ctx.sync()
    t16 = omlp.fp16_weights(theta)
    ref, _ = omlp.forward(t16, X.astype(np.float32).astype(np.float64))
    assert np.allclose(host(out), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    grad = torch.empty(omlp.param_count(), dtype=torch.float32, device=DEV)
    ctx.bw_train_step(th, None, None, 0, dev(X, torch.float32), dev(Y, torch.float32), dev(M),
                      loss=loss, grad=grad)
    ctx.sync()
    rl, rg = omlp.loss_and_grad(t16, X.astype(np.float32).astype(np.float64),
                                Y.astype(np.float32).astype(np.float64), M)
    assert abs(float(host(loss)[0]) - rl) <= 1e-4 * abs(rl)
    g = host(grad).astype(np.float64)
    assert np.linalg.norm(g - rg) <= 1e-3 * np.linalg.norm(rg)


def test_adamw_step_vs_oracle(ctx):
    rng = np.random.default_rng(6)
    theta = init_params(2).astype(np.float32).astype(np.float64)
    B = 64
    X = rng.standard_normal((B, 32)).astype(np.float32)
    Y = rng.standard_normal((B, 6)).astype(np.float32)
    M = np.ones((B, 6), dtype=np.uint8)
    th = dev(theta, torch.float32)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    grad = torch.empty_like(th)
    lr, wd = 1e-3, 1e-4
    ctx.bw_train_step(th, m, v, 1, dev(X), dev(Y), dev(M), lr=lr, wd=wd, grad=grad)
    ctx.sync()
    g = host(grad).astype(np.float64)
    ref, _, _ = omlp.adamw_step(theta, np.zeros_like(theta), np.zeros_like(theta), g, 1, lr, wd)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.allclose(host(th)[big], ref[big], rtol=1e-5, atol=1e-7)


def test_training_reduces_loss(ctx):
    rng = np.random.default_rng(7)
    B = 256
    X = rng.standard_normal((B, 32)).astype(np.float32)
    Wt = rng.standard_normal((32, 6)) * 0.3
    Y = np.tanh(X @ Wt).astype(np.float32)
    M = np.ones((B, 6), dtype=np.uint8)
    th = dev(init_params(3), torch.float32)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    Xd, Yd, Md = dev(X), dev(Y), dev(M)
    first = None
    for step in range(1, 301):
        ctx.bw_train_step(th, m, v, step, Xd, Yd, Md, lr=1e-3, wd=1e-4, loss=loss)
        if step == 1:
            ctx.sync()
            first = float(host(loss)[0])
    ctx.sync()
    last = float(host(loss)[0])
    assert last < 0.05 * first


@pytest.mark.parametrize("kind", ["dense", "sparse", "dense1d", "sparse_folds"])
def test_features_vs_oracle(ctx, kind):
    from paper_1510_04439_gb300 import binding as B
    if kind == "dense":
        D = fs.make_dense(2, (16, 16), 120, [2.0, 1.0], sigma=0.5, seed=3, domain="disk", dropout=0.2)
    elif kind == "dense1d":
        D = fs.make_dense(1, (48,), 90, [2.0, 1.0], sigma=0.3, mean="1d", seed=4, dropout=0.3)
    else:
        D = fs.make_sparse(2, (12, 12), 700, [2.0, 1.0], seed=8, nfold=0)
    m, P = D.m, D.P
    nfold = 0
    if kind == "sparse_folds":
        # the fold slices are pooled by the kernel: the expected value uses their sums
        nfold = 3
        fold = (np.arange(D.n) % nfold).astype(np.int32)
        data = ctx.sparse(dev(D.offs), dev(D.t), dev(D.y))
        cnt, Wm, Vm, V2m = sm.bin_mean_sparse(D.offs, D.t, D.y, m)
        Ni = np.diff(D.offs)
        r = sm.residuals_sparse(D.t, D.y, np.zeros(P), m)
        Cf, Wf, Vf, _ = sm.bin_cov_sparse(D.offs, D.t, r, m, fold=fold, nfold=nfold)
        C, W, V = Cf.sum(0), Wf.sum(0), Vf.sum(0)
        ref = ofeat.features(len(m), m, Ni, cnt, Wm, Vm, V2m, C, W, V)
        feat = torch.empty(32, dtype=torch.float32, device=DEV)
        ctx.bw_features(data, m, dev(cnt, torch.int32), dev(Wm), dev(Vm), dev(V2m),
                        dev(Cf, torch.int32), dev(Wf), dev(Vf), feat, nfold=nfold)
        ctx.sync()
        assert np.allclose(host(feat), ref, rtol=1e-5, atol=1e-4), np.abs(host(feat) - ref).max()
        return
    if kind == "sparse":
        data = ctx.sparse(dev(D.offs), dev(D.t), dev(D.y))
        cnt, Wm, Vm, V2m = sm.bin_mean_sparse(D.offs, D.t, D.y, m)
        Ni = np.diff(D.offs)
        r = sm.residuals_sparse(D.t, D.y, np.zeros(P), m)
        C, W, V, _ = sm.bin_cov_sparse(D.offs, D.t, r, m)
        C, W, V = C[0], W[0], V[0]
    else:
        data = ctx.dense(dev(D.y), dev(D.mask))
        cnt, Wm, Vm, V2m = sm.bin_mean_dense(D.y, D.mask, m)
        Ni = D.mask.sum(axis=1)
        C, W, V = sm.bin_cov_dense(D.y, D.mask)
    ref = ofeat.features(len(m), m, Ni, cnt, Wm, Vm, V2m, C, W, V)
    feat = torch.empty(32, dtype=torch.float32, device=DEV)
    ctx.bw_features(data, m, dev(cnt, torch.int32), dev(Wm), dev(Vm), dev(V2m), dev(C, torch.int32),
                    dev(W), dev(V), feat)
    ctx.sync()
    assert np.allclose(host(feat), ref, rtol=1e-5, atol=1e-4), np.abs(host(feat) - ref).max()


def test_bandwidth_workflow_small(ctx):
    """Labels, training and the proposal + check evaluation end to end on a few datasets:
    the batched CV grids agree with single-bandwidth CV calls, labels are the grid
    argmins of both smoothers (the covariance one on bins at the mean's best
    bandwidth), and the evaluation rows are complete."""
    from paper_1510_04439_gb300 import bandwidth as bw
    lab = bw.Labeller(ctx, torch)
    ds = bw.draw_dataset(11)
    prep = lab.prepare(ds)
    gm = host(lab.mean_cv(prep, bw.HGRID))
    for j in (0, 7, 15):
        one = host(lab.mean_cv(prep, [bw.HGRID[j]]))[0]
        assert (not np.isfinite(gm[j]) and not np.isfinite(one)) or abs(one - gm[j]) <= 1e-12 * abs(gm[j])
    jm = int(np.argmin(np.where(np.isfinite(gm), gm, np.inf)))
    lab.cov_bins(prep, bw.HGRID[jm])
    grid = host(lab.cv(prep, bw.HGRID))
    for j in (0, 7, 15):
        one = host(lab.cv(prep, [bw.HGRID[j]]))[0]
        if np.isfinite(grid[j]):
            assert abs(one - grid[j]) <= 1e-9 * abs(grid[j])
        else:
            assert not np.isfinite(one)
    X, Y, M, best = bw.make_table(ctx, torch, [11, 12, 13, 14])
    assert X.shape == (4, 32) and np.isfinite(X).all()
    assert best[0, 0] == jm
    assert best[0, 1] == int(np.argmin(np.where(np.isfinite(grid), grid, np.inf)))
    for k in range(4):
        d = int(round(X[k, 0]))
        assert M[k, :d].all() and not M[k, d:3].any()
        assert M[k, 3:3 + d].all() and not M[k, 3 + d:].any()
        assert np.allclose(Y[k, :d], np.log(bw.HGRID[best[k, 0]]))
        assert np.allclose(Y[k, 3:3 + d], np.log(bw.HGRID[best[k, 1]]))
    Xs, mu, sd = bw.standardize(X)
    th, hist = bw.train(ctx, torch, Xs, Y, M, epochs=20, batch=4)
    assert hist[-1] < hist[0]
    const = bw.median_labels(Y, M, np.rint(X[:, 0]).astype(int))
    rows = bw.evaluate(ctx, torch, th, mu, sd, [21, 22], const=const)
    assert len(rows) == 2
    for r in rows:
        assert bw.HGRID[0] * 0.8 <= r["final_h"] <= bw.HGRID[-1] * 1.25
        if r["fallback"]:
            assert r["final_score"] == r["grid_best"]
        assert np.isfinite(r["sine_const"]) and np.isfinite(r["fpca_const"])


@pytest.mark.slow
def test_learned_bandwidth_gain(ctx):
    """What the trained network gains: on held-out datasets the whole FPCA with the
    learned proposals (each with its 3-bandwidth CV check) is faster than the
    16-bandwidth CV grids, its covariance CV score stays within 5% of the grid
    optimum, its eigenfunctions are as accurate as the grid method's (subspace sine
    against the truth), and it beats the constant proposal (the median training
    labels through the same checks) on accuracy or on time."""
    from paper_1510_04439_gb300 import bandwidth as bw
    X, Y, M, _ = bw.make_table(ctx, torch, np.arange(300))
    Xs, mu, sd = bw.standardize(X)
    th, hist = bw.train(ctx, torch, Xs, Y, M, epochs=150)
    assert hist[-1] < 0.2 * hist[0]
    const = bw.median_labels(Y, M, np.rint(X[:, 0]).astype(int))
    rows = bw.evaluate(ctx, torch, th, mu, sd, 10 ** 6 + np.arange(40), const=const)
    s = bw.summarize(rows)
    print(json.dumps(s))
    assert s["within5"] >= 0.9, s
    assert s["fpca_learned_s"] < s["fpca_grid_s"], s
    assert s["sine_learned_median"] <= s["sine_grid_median"] + 0.02, s
    assert s["sine_grid_median"] < 0.5, s          # the fits do recover the eigenfunctions
    c = s["constant_proposal"]
    better_accuracy = (s["within5"] > c["within5"] or s["fallback_rate"] < c["fallback_rate"]
                       or s["sine_learned_mean"] < c["sine_mean"])
    assert better_accuracy or s["fpca_learned_s"] < c["fpca_s"], s
    for r in rows:
        assert np.isfinite(r["sine_grid"]) and np.isfinite(r["sine_learned"])


def test_mlp_init_is_he_normal_and_seeded(ctx):
    """fpca_bw_mlp_init: biases zero, each layer's weights N(0, 2/fan_in) (sample
    mean and variance within a few standard errors), same seed same vector."""
    n = omlp.param_count()
    a = torch.empty(n, dtype=torch.float32, device=DEV)
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    ctx.bw_mlp_init(a, 7)
    ctx.bw_mlp_init(b, 7)
    ctx.bw_mlp_init(c, 8)
    ctx.sync()
    assert torch.equal(a, b)
    assert not torch.equal(a, c)
    layers = omlp.unpack(host(a).astype(np.float64))
    for (W, bias), (fi, fo) in zip(layers, omlp.LAYERS):
        assert np.all(bias == 0.0)
        var = 2.0 / fi
        k = W.size
        assert abs(W.mean()) <= 5.0 * np.sqrt(var / k)
        assert abs(W.var() / var - 1.0) <= 5.0 * np.sqrt(2.0 / k)
        # normal shape: the fraction inside one standard deviation is 0.6827
        inside = np.mean(np.abs(W) <= np.sqrt(var))
        assert abs(inside - 0.6827) <= 5.0 * np.sqrt(0.6827 * 0.3173 / k)


def test_mlp_save_and_load_round_trip(ctx, tmp_path):
    from paper_1510_04439_gb300 import binding as B
    n = omlp.param_count()
    th = torch.empty(n, dtype=torch.float32, device=DEV)
    ctx.bw_mlp_init(th, 3)
    mu = torch.linspace(-1, 1, 32, dtype=torch.float32, device=DEV)
    sd = torch.linspace(0.5, 2, 32, dtype=torch.float32, device=DEV)
    path = tmp_path / "net.bin"
    ctx.bw_mlp_io(th, path, True, mu, sd)
    th2 = torch.zeros_like(th)
    mu2 = torch.zeros_like(mu)
    sd2 = torch.zeros_like(sd)
    ctx.bw_mlp_io(th2, path, False, mu2, sd2)
    ctx.sync()
    assert torch.equal(th, th2) and torch.equal(mu, mu2) and torch.equal(sd, sd2)
    # the loaded network predicts what the saved one did
    X = torch.randn(16, 32, device=DEV)
    o1 = torch.empty(16, 6, device=DEV)
    o2 = torch.empty(16, 6, device=DEV)
    ctx.bw_predict(th, X, o1)
    ctx.bw_predict(th2, X, o2)
    ctx.sync()
    assert torch.equal(o1, o2)
    # a file of another layout is refused and leaves the arrays alone
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"FPCABW01" + (123).to_bytes(8, "little") + bytes(64))
    with pytest.raises(B.FpcaError) as e:
        ctx.bw_mlp_io(th2, bad, False)
    assert e.value.status == B.E_INVALID_ARG
    assert torch.equal(th, th2)
