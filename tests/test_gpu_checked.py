"""The bounds-checked build (GGEVAL_CHECKED, built by build() next to the
library): the C++ interpreter with every shared-memory stack and feature
access and every tile copy tested first, a violation recorded in the status
word (GGEVAL_ERR_CHECKED from ggeval_sync), never trapped.  On small cases
of every workload it must report nothing, match the oracle, and give
per-row values bit-identical to the library's PTX interpreter (the same
operations in the same order)."""
import contextlib
import os

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


@pytest.fixture(scope="module")
def checked_lib(gg):
    path = os.path.join(os.path.dirname(gg.ggeval.LIB_PATH), "libggeval_checked.so")
    return gg.ggeval.load_library(path)  # ImportError if build() did not make it


@contextlib.contextmanager
def using(gg, lib):
    saved = gg.ggeval._LIB
    gg.ggeval._LIB = lib
    try:
        yield
    finally:
        gg.ggeval._LIB = saved


def run(gg, w, flags):
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda()
    hs = torch.from_numpy(w["heights"]).cuda()
    rows = ds.eval_rows(op, cv, hs, flags=flags).cpu().numpy()
    outs = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=flags)]
    ds.sync()  # raises GGEVAL_ERR_CHECKED if a bounds check failed
    ds.close()
    return rows, outs


@pytest.mark.parametrize("cfg,n_rows,n_trials", [
    ("c1", 1000, 64), ("c2", 5003, 64), ("c3", 4099, 48), ("c5", 3000, 32),
    ("t2", 5003, 64), ("l8_squ", 2000, 24)])
def test_checked_build_is_clean_and_identical(gg, checked_lib, cfg, n_rows, n_trials):
    w = PA.build(cfg, n_rows, n_trials)
    flags = gg.F_POW if w.get("uses_pow") else 0
    with using(gg, checked_lib):
        rows_c, outs_c = run(gg, w, flags)
    rows_p, outs_p = run(gg, w, flags)
    same = (rows_c.view(np.uint32) == rows_p.view(np.uint32)) | (np.isnan(rows_c) &
                                                                   np.isnan(rows_p))
    assert same.all(), np.argwhere(~same)[:5]
    for a, b in zip(outs_c, outs_p):
        np.testing.assert_array_equal(a, b)
    t = PA.check_fitness(w, range(w["P"]), outs_c[0], outs_c[3], processes=1)
    PA.report(f"checked build {w['name']} ({n_rows} rows)", "trials", t)
    assert t.failed == 0, repr(t)
