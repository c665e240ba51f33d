"""The evaluation entry point that allocates nothing.

Callers that cannot call cudaMalloc while they evaluate (inside a stream
capture, in loops that cannot take the allocator's device synchronisation,
under a fixed device-memory budget) use ggeval_eval_batch_noalloc, whose
scratch is one static device array.  This checks, through the C ABI, that
two calls in a row give the same fitness as ggeval_eval_batch within the
tolerance the cross-form tests use, and that requests beyond the static
limits are refused.  Kept in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def call_noalloc(gg, ds, op, cv, outs):
    b = gg.make_batch(op, cv)
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return gg.lib().ggeval_eval_batch_noalloc(ds._h, ctypes.byref(b), *ptrs, stream)


def test_noalloc_matches_eval_batch_twice(gg):
    w = PA.build("c2", 30_000, 700)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op = torch.from_numpy(w["op"]).cuda()
    cv = torch.from_numpy(w["cval"]).cuda()
    ref = [t.cpu().numpy().astype(np.float64) for t in ds.eval_batch(op, cv)]
    ds.sync()
    vy = float(np.var(w["y"].astype(np.float64)))
    for _ in range(2):
        outs = [torch.full((w["P"],), float("nan"), device="cuda") for _ in range(4)]
        assert call_noalloc(gg, ds, op, cv, outs) == 0, gg.lib().ggeval_last_error()
        ds.sync()
        got = [t.cpu().numpy().astype(np.float64) for t in outs]
        fin = np.isfinite(ref[0])
        np.testing.assert_array_equal(fin, np.isfinite(got[0]))
        np.testing.assert_allclose(got[0][fin], ref[0][fin], rtol=2e-4, atol=1e-8 * vy)
        np.testing.assert_allclose(got[3][fin], ref[3][fin], rtol=2e-4, atol=1e-8 * vy)
        ok = fin & (np.abs(ref[2]) > 1e-3)
        np.testing.assert_allclose(got[2][ok], ref[2][ok], rtol=1e-3)
    ds.close()


def test_noalloc_refuses_beyond_limits(gg):
    w = PA.build("c1", 1000, 8)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    big = torch.zeros((4097, 15), dtype=torch.uint8, device="cuda")
    outs = [torch.empty(4097, device="cuda") for _ in range(4)]
    assert call_noalloc(gg, ds, big, torch.zeros((4097, 15), device="cuda"), outs) == -7
    assert b"4097" in gg.lib().ggeval_last_error()
    tall = torch.zeros((2, 255), dtype=torch.uint8, device="cuda")  # height 7
    assert call_noalloc(gg, ds, tall, torch.zeros((2, 255), device="cuda"), outs[:4]) == -7
    ds.close()
    # rows that do not fit in 64 row tiles of shared-memory size: refused,
    # nothing launched (the outputs keep their values)
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.uniform(-1, 1, (1_000_000, 10)).astype(np.float32))
    ds = gg.Dataset(X, torch.from_numpy(rng.standard_normal(1_000_000).astype(np.float32)))
    op = torch.full((4, 15), 32, dtype=torch.uint8, device="cuda")  # x0
    outs = [torch.full((4,), float("nan"), device="cuda") for _ in range(4)]
    assert call_noalloc(gg, ds, op, torch.zeros((4, 15), device="cuda"), outs) == -7
    assert b"tiles" in gg.lib().ggeval_last_error()
    ds.sync()
    assert all(torch.isnan(t).all() for t in outs)
    ds.close()
