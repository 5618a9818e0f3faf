"""Failure detection without a GPU fault: a device-side bounded wait that runs out.

Every kernel of the library that waits (on a bulk copy, a tensor-core commit or
a barrier) does so with a wait that gives up after about 2 s of GPU time,
records a timeout in the context's error word and returns.  fpca_check_wait
runs that same wait on a barrier that nothing completes; the next sync must
report FPCA_E_TIMEOUT, the error word must be cleared by reading it, and the
context must go on working.  Nothing here faults, traps or hangs the GPU: the
waiting thread returns by itself.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_recovers():
    from paper_1510_04439_gb300 import binding as B
    ctx = B.Context(0)
    ctx.check_wait(True)           # completed barrier: no error
    ctx.sync()
    t0 = time.perf_counter()
    ctx.check_wait(False)          # nothing arrives: the wait gives up
    with pytest.raises(B.FpcaError) as e:
        ctx.sync()
    waited = time.perf_counter() - t0
    assert e.value.status == B.E_TIMEOUT
    assert 1.0 <= waited <= 30.0, waited
    ctx.sync()                     # the error word was cleared by the read
    # the context still computes: mean bins of a tiny grid
    y = torch.arange(12, dtype=torch.float64, device="cuda:0").reshape(3, 4)
    cnt = torch.empty(4, dtype=torch.int32, device="cuda:0")
    w, v = (torch.empty(4, dtype=torch.float64, device="cuda:0") for _ in range(2))
    ctx.bin_mean(ctx.dense(y), (4,), cnt, w, v)
    ctx.sync()
    assert np.array_equal(cnt.cpu().numpy(), [3, 3, 3, 3])
    assert np.allclose(v.cpu().numpy(), (y.sum(0) / 4).cpu().numpy())
