"""Failure detection on the GPU without a fault: a bounded device wait that
runs out reports GGEVAL_ERR_TIMEOUT through the status word, and the context
stays usable.  The test hook GGEVAL_F_TEST_STALL makes the batched forward
kernel issue no tile copy, so nothing is in flight while its waits give up
(no trap, no hang, no bad address)."""
import time

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


def test_bounded_wait_gives_up_and_the_context_survives(gg):
    w = PA.build("c2", 20_000, 64)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda()
    ref = [t.clone() for t in ds.eval_batch(op, cv)]
    ds.sync()
    t0 = time.perf_counter()
    ds.eval_batch(op, cv, flags=gg.F_TEST_STALL)
    with pytest.raises(gg.GGEvalError) as e:
        ds.sync()
    took = time.perf_counter() - t0
    assert e.value.status == gg.ERR_TIMEOUT
    assert took < 30.0, took
    ds.sync()  # the status word was cleared
    again = ds.eval_batch(op, cv)
    ds.sync()
    for r, a in zip(ref, again):
        assert torch.equal(r, a)
    # a graph-replayed call and the end-to-end path still work too
    st = torch.cuda.Stream()
    outs = [torch.empty(64, device="cuda") for _ in range(4)]
    ds.eval_batch(op, cv, flags=gg.F_GRAPH, stream=st, out=outs)
    ds.sync(st)
    assert torch.equal(outs[0], ref[0])
    ds.close()
