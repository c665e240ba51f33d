"""Randomised GPU parity of the adjoint: the configurations of the
randomised fitness test (heights to 5, both layouts, random operator sets
with pow, both objectives), each trial's d fitness / d ERC compared with
the FP64 oracle's reverse mode under the gradient tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
import parity as PA
from test_gpu_fuzz import random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("seed", range(16))
def test_random_gradients(gg, seed):
    run_gradients(gg, random_case(seed), seed)


@pytest.mark.parametrize("seed", range(6))
def test_random_gradients_wide(gg, seed):
    """More than 16 features: the adjoint reads the features from global
    memory (the kernel with 1, 2 or 4 rows per lane), per length class."""
    run_gradients(gg, random_case(seed, wide=True), seed)


def run_gradients(gg, w, seed):
    if int(w["heights"].max()) > 5 or w["N"] < 2:
        pytest.skip("the oracle's reverse mode is kept to heights up to 5 and two rows")
    mode = "mse" if seed % 3 == 2 else "smse"
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    flags = (gg.F_GRAD_MSE if mode == "mse" else 0) | (gg.F_POW if synth.POW in w["funcs"] else 0)
    smse, dc = ds.grad_batch(torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda(),
                             torch.from_numpy(w["heights"]).cuda(),
                             layout=0 if w["layout"] == "heap" else 1, flags=flags)
    ds.sync()
    smse, dc = smse.cpu().numpy(), dc.cpu().numpy()
    ds.close()
    tally, fit_tally = PA.Tally(), PA.Tally()
    y64 = w["y"].astype(np.float64)
    var_y, mean_y2 = float(np.var(y64)), float(np.mean(y64 ** 2))
    for p in range(w["P"]):
        t, f64, f32, fit64, fit32, cond, bounds = PA.oracle_trial(w, p)
        before = fit_tally.excluded
        PA.check_fit(float(smse[p]), None, fit64, fit32, var_y, mean_y2, fit_tally,
                     tag=f"trial {p}", bounds=bounds)
        if fit_tally.excluded != before or not PA.intermediates_finite_f32(t, w["X"]):
            tally.excluded += 1
            continue
        g64, _, gabs = O.grad(t, w["X"], w["y"], mode, with_abs=True)
        if not fit64["finite"] or (mode == "smse" and fit64["b"] == 0.0):
            assert np.all(dc[p] == 0.0), p
            tally.checked += 1
            continue
        if not np.all(np.isfinite(g64)):
            tally.excluded += 1
            continue
        PA.check_grad(dc[p], g64, tally, tag=f"trial {p}", rabs=gabs)
    assert tally.failed == 0 and fit_tally.failed == 0, (repr(tally), repr(fit_tally))
    assert tally.checked >= w["P"] // 3, repr(tally)
