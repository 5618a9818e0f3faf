"""CUDA graphs of library call sequences (fpca_graph_begin / _end / _launch).

A recorded dense step (mean bins and fit, BF16 tensor-core covariance bins, the
FP32 compensated smoother, the random-projection eigenpairs) replayed on new
inputs written into the same buffers must give what the same calls give when run
directly: the kernels and their order are the same, so Gamma_hat and the statuses
are bit-identical and the eigenpairs agree to rounding (one FP64 atomic sum).
Calls that cannot be recorded (a host read-back) refuse, the capture then yields
no graph, and the context keeps working; a context on the legacy default stream
cannot record.
"""
import numpy as np
import pytest

import fpca_synth as fs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    from paper_1510_04439_gb300 import binding
    return binding


def make_inputs(seed):
    D = fs.make_dense(2, (32, 32), 200, [4.0, 2.0, 1.0], sigma=0.4, seed=seed, domain="disk",
                      dropout=0.1)
    return D, D.y.astype(np.float32), D.mask


def test_recorded_dense_step_matches_direct_calls(B):
    from paper_1510_04439_gb300 import pipeline
    stream = torch.cuda.Stream()
    ctx = B.Context(0, stream)
    D, y0, m0 = make_inputs(3)
    _, y1, m1 = make_inputs(4)
    P, k, h = D.P, 4, (0.15, 0.15)
    om = torch.from_numpy(fs.gaussian_test_matrix(P, k + 10, 5).astype(np.float32)).to(DEV)
    y = torch.from_numpy(y0).to(DEV)
    mask = torch.from_numpy(m0).to(DEV)
    bufs = pipeline.alloc_dense(torch, torch.device(DEV), P, k, B.BF16, B.F32)

    def step():
        pipeline.run_dense(ctx, D.m, y, mask, h, h, k, bufs, bin_prec=B.BF16,
                           smooth_prec=B.F32C, omega=om, power_iters=2)

    with torch.cuda.stream(stream):
        step()                      # settles the workspace and the autotuners
        ctx.sync()
        l0 = ctx.launches
        step()
        ctx.sync()
        direct_launches = ctx.launches - l0
        ctx.graph_begin()
        step()                      # recorded, not run
        g = ctx.graph_end()
        assert g.launches == direct_launches
        # new inputs in the same buffers: the direct calls, then the replay
        y.copy_(torch.from_numpy(y1))
        mask.copy_(torch.from_numpy(m1))
        step()
        ctx.sync()
        ref = [t.clone() for t in (bufs.gamma, bufs.status, bufs.evals, bufs.evecs)]
        bufs.gamma.zero_()
        bufs.evals.zero_()
        l0 = ctx.launches
        ctx.graph_launch(g)
        ctx.sync()
        assert ctx.launches - l0 == g.launches
    # (EMPTY points outside the disk hold NaN on both sides)
    assert torch.allclose(bufs.gamma, ref[0], rtol=0, atol=0, equal_nan=True)
    assert torch.equal(bufs.status, ref[1])
    # the domain trace is an atomic FP64 sum, so the eigen step may differ in the last bits
    assert torch.allclose(bufs.evals, ref[2], rtol=1e-12, atol=0)
    assert torch.allclose(bufs.evecs, ref[3], rtol=1e-10, atol=1e-12)


def test_capture_refuses_host_read_back_and_context_recovers(B):
    stream = torch.cuda.Stream()
    ctx = B.Context(0, stream)
    Ds = fs.make_sparse(2, (8, 8), 50, [1.0], nmin=3, nmax=6, seed=2, nfold=0)
    t = {k: torch.from_numpy(getattr(Ds, k)).to(DEV) for k in ("offs", "t", "y")}
    data = ctx.sparse(t["offs"], t["t"], t["y"])
    P = Ds.P
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(2))
    with torch.cuda.stream(stream):
        ctx.bin_mean(data, Ds.m, cnt, w, v)     # scattered binning reads offs[n] back
        ctx.sync()
        ref = cnt.clone()
        ctx.graph_begin()
        with pytest.raises(B.FpcaError) as e:
            ctx.bin_mean(data, Ds.m, cnt, w, v)
        assert e.value.status == B.E_UNSUPPORTED
        with pytest.raises(B.FpcaError) as e:
            ctx.graph_end()
        assert e.value.status == B.E_UNSUPPORTED
        cnt.zero_()
        ctx.bin_mean(data, Ds.m, cnt, w, v)     # the context works as before
        ctx.sync()
    assert torch.equal(cnt, ref)


def test_capture_needs_a_created_stream(B):
    ctx = B.Context(0)                          # legacy default stream
    with pytest.raises(B.FpcaError) as e:
        ctx.graph_begin()
    assert e.value.status == B.E_UNSUPPORTED
