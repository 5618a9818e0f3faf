"""The allocation-free mean binning entry point against the allocating one.

fpca_bin_mean_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or allocation is not allowed
where they run).  Its scratch is a fixed file-scope device array shared by
all calls; two calls in a row on different data must each match
fpca_bin_mean on the same data.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import fpca_synth as fs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


# The two entry points add the same terms in different orders (one FP64 chain
# per bin here, float-float subject slices and an FP64 tree in fpca_bin_mean):
# counts are bit-identical, the sums agree to about 1e-13 relative.
RTOL = 1e-13


def _bins_allocating(ctx, y, mask, m, with_v2=True):
    P = y.shape[1]
    cnt = torch.empty(P, dtype=torch.int32, device=DEV)
    w, v, v2 = (torch.empty(P, dtype=torch.float64, device=DEV) for _ in range(3))
    ctx.bin_mean(ctx.dense(y, mask), m, cnt, w, v, v2 if with_v2 else None)
    ctx.sync()
    return (cnt, w, v, v2) if with_v2 else (cnt, w, v)


def _bins_static(lib, B, y, mask, with_v2=True):
    n, P = y.shape
    cnt = torch.full((P,), -7, dtype=torch.int32, device=DEV)
    w, v, v2 = (torch.full((P,), np.nan, dtype=torch.float64, device=DEV) for _ in range(3))
    stream = torch.cuda.current_stream()
    st = lib.fpca_bin_mean_static(ctypes.c_void_p(stream.cuda_stream), n, P,
                                  ctypes.c_void_p(y.data_ptr()),
                                  B.F64 if y.dtype == torch.float64 else B.F32,
                                  ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
                                  ctypes.c_void_p(cnt.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                  ctypes.c_void_p(v.data_ptr()),
                                  ctypes.c_void_p(v2.data_ptr()) if with_v2 else None)
    assert st == B.OK
    stream.synchronize()
    if not with_v2:
        assert torch.all(torch.isnan(v2)), "v2 = NULL must leave the buffer untouched"
        return cnt, w, v
    return cnt, w, v, v2


def _assert_same(got, ref):
    assert torch.equal(got[0], ref[0])
    for a, b in zip(got[1:], ref[1:]):
        assert torch.allclose(a, b, rtol=RTOL, atol=RTOL)


def test_static_mean_bins_match_allocating_entry_point_twice():
    from paper_1510_04439_gb300 import binding as B
    lib = B.load()
    ctx = B.Context(0)
    # two different datasets in a row: the shared scratch must not leak state
    cases = [fs.dense_2d_disk(n=700, m=32), fs.make_dense(2, (16, 24), 90, [2.0, 1.0], seed=4,
                                                          dropout=0.3)]
    for D, dtype in zip(cases, (torch.float32, torch.float64)):
        y = torch.from_numpy(D.y).to(dtype).to(DEV)
        mask = torch.from_numpy(D.mask).to(DEV)
        ref = _bins_allocating(ctx, y, mask, D.m)
        got = _bins_static(lib, B, y, mask)
        _assert_same(got, ref)


def test_static_mean_bins_null_mask_null_v2_and_empty_subject():
    """mask = NULL (every node observed), v2 = NULL, and a subject whose mask row is
    all zero (N_i = 0, skipped by both entry points), each against fpca_bin_mean."""
    from paper_1510_04439_gb300 import binding as B
    lib = B.load()
    ctx = B.Context(0)
    D = fs.make_dense(2, (12, 20), 50, [2.0, 1.0], seed=8)
    y = torch.from_numpy(D.y).to(DEV)
    _assert_same(_bins_static(lib, B, y, None), _bins_allocating(ctx, y, None, D.m))
    _assert_same(_bins_static(lib, B, y, None, with_v2=False),
                 _bins_allocating(ctx, y, None, D.m, with_v2=False))
    D2 = fs.make_dense(2, (16, 16), 40, [2.0, 1.0], seed=9, dropout=0.2)
    mask = D2.mask.copy()
    mask[3, :] = 0
    mask[17, :] = 0
    y2 = torch.from_numpy(D2.y).to(torch.float32).to(DEV)
    m2 = torch.from_numpy(mask).to(DEV)
    got = _bins_static(lib, B, y2, m2)
    _assert_same(got, _bins_allocating(ctx, y2, m2, D2.m))
    _assert_same(_bins_static(lib, B, y2, m2, with_v2=False),
                 _bins_allocating(ctx, y2, m2, D2.m, with_v2=False))


def test_static_mean_bins_reject_oversize_n():
    from paper_1510_04439_gb300 import binding as B
    lib = B.load()
    buf = torch.zeros(8, dtype=torch.float64, device=DEV)
    st = lib.fpca_bin_mean_static(None, (1 << 20) + 1, 1, ctypes.c_void_p(buf.data_ptr()), B.F64,
                                  None, ctypes.c_void_p(buf.data_ptr()),
                                  ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                  None)
    assert st == B.E_UNSUPPORTED
