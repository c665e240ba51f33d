"""Size objective, NMSE, and the Experiment III ladder workloads on the GPU."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from fixtures import heap_template
import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def test_trial_sizes_match_active_sets(gg):
    w = synth.workload("c3", 2, n_rows=10, n_trials=300)
    size = gg.trial_sizes(torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda(),
                          w["F"], torch.from_numpy(w["heights"]).cuda()).cpu().numpy()
    want = [int(O.active_mask(PA.template(w, p)).sum()) for p in range(300)]
    np.testing.assert_array_equal(size, want)


@pytest.mark.parametrize("layout", ["heap", "prefix"])
def test_trial_sizes_and_changed_in_both_layouts(gg, layout):
    """Active-node counts and the active-part "changed" test in either
    template layout, against the oracle's active sets."""
    rng = np.random.default_rng(21)
    op, cv, hs = synth.random_templates(rng, 200, rng.integers(0, 8, 200), 7,
                                        synth.FULL_SET, 4, 0.6)
    op2, cv2 = op.copy(), cv.copy()
    flip = rng.random(op.shape) < 0.03  # mutate a few nodes (active or intron)
    op2[flip] = synth.FEAT0 + rng.integers(0, 4, flip.sum())
    if layout == "prefix":
        op, cv = synth.to_prefix(op, cv, hs.astype(np.int64))
        op2, cv2 = synth.to_prefix(op2, cv2, hs.astype(np.int64))
    lay = 0 if layout == "heap" else 1
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    h8 = hs.astype(np.int8)
    size = gg.trial_sizes(d(op), d(cv), 4, d(h8), layout=lay).cpu().numpy()
    ch = gg.gom_changed(d(op2), d(cv2), d(op), d(cv), 4, d(h8), layout=lay).cpu().numpy()
    torch.cuda.synchronize()
    for p in range(200):
        t = O.Template(op[p], cv[p], int(hs[p]), layout, 4)
        assert size[p] == int(O.active_mask(t).sum()), p
    want = O.gom.changed(op2, cv2, op, cv, hs, layout, 4)
    np.testing.assert_array_equal(ch, want)
    assert 0 < want.sum() < 200


def test_nmse_and_dataset_info(gg):
    w = PA.build("c2", 5000, 30)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    n, f, ym, yv = ds.info()
    y = w["y"].astype(np.float64)
    assert (n, f) == (5000, 8)
    np.testing.assert_allclose([ym, yv], [y.mean(), y.var()], rtol=1e-6)
    res = ds.evaluate(torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda(),
                      want=("smse", "mse", "nmse"))
    mse, nmse = res["mse"].cpu().numpy(), res["nmse"].cpu().numpy()
    ds.sync()
    ds.close()
    fin = np.isfinite(mse)
    np.testing.assert_allclose(nmse[fin], mse[fin] / yv, rtol=2e-7)
    checked = 0
    for p in range(30):
        t, f64, f32, fit64, fit32, cond, bounds = PA.oracle_trial(w, p)
        if not fit64["finite"] or not np.isfinite(nmse[p]) or bounds is None:
            continue
        if bounds[1] > 1e-6 * fit64["mse"]:
            continue
        checked += 1
        assert abs(nmse[p] - fit64["nmse"]) <= 2e-4 * fit64["nmse"] + 1e-8
    assert checked >= 10


@pytest.mark.parametrize("fold", [True, False])
def test_error_and_size_objectives_in_one_call(gg, fold):
    """evaluate() returns every objective of every trial from one launch
    sequence: scaled MSE, MSE and NMSE as eval_batch computes them, and the
    size objective (active nodes, the oracle's active set) with the nodes
    evaluated per row after folding (the host packer's count); an invalid
    trial gets size -1.  Device and pinned host batches agree."""
    w = PA.build("c3", 3001, 120)
    w["op"][7, 0] = 200  # an invalid root
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = torch.from_numpy(w["op"]).cuda(), torch.from_numpy(w["cval"]).cuda()
    hs = torch.from_numpy(w["heights"]).cuda()
    flags = 0 if fold else gg.F_NO_FOLD
    res = {k: v.cpu().numpy() for k, v in ds.evaluate(op, cv, hs, flags=flags).items()}
    ref = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=flags)]
    with pytest.raises(gg.GGEvalError):
        ds.sync()
    host = ds.evaluate(torch.from_numpy(w["op"]).pin_memory(),
                       torch.from_numpy(w["cval"]).pin_memory(),
                       torch.from_numpy(w["heights"]).pin_memory(), flags=flags)
    torch.cuda.synchronize()
    with pytest.raises(gg.GGEvalError):
        ds.sync()
    ds.close()
    for k, r in zip(("smse", "a", "b", "mse"), ref):
        np.testing.assert_array_equal(res[k], r)
    for k, v in host.items():
        assert not v.is_cuda
        np.testing.assert_array_equal(v.numpy(), res[k])
    st = gg.batch_stats(torch.from_numpy(w["op"]), torch.from_numpy(w["cval"]),
                        torch.from_numpy(w["heights"]), n_features=w["F"]).numpy()
    for p in range(w["P"]):
        if p == 7:
            assert res["size"][p] == -1 and res["size_evaluated"][p] == -1
            assert np.isnan(res["smse"][p])
            continue
        assert res["size"][p] == int(O.active_mask(PA.template(w, p)).sum()), p
        want_eval = st[p, 13] if fold else st[p, 0]
        assert res["size_evaluated"][p] == want_eval, p
    if fold:
        assert (res["size_evaluated"] < res["size"]).any()


@pytest.mark.parametrize("cfg", ["l_add", "l_squ", "l_sub", "l8_add", "l8_div", "l8_sub",
                                 "l8_mul", "l8_squ"])
def test_ladder_parity(gg, cfg):
    """The Experiment III ladder (Table 1 targets) with the depth-6 and
    depth-8 templates (127 and 511 nodes) of Table 2, on 4,000-row slices."""
    w = PA.build(cfg, 4000, 40)
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    smse, a, b, mse = (t.cpu().numpy() for t in
                       ds.eval_batch(torch.from_numpy(w["op"]).cuda(),
                                     torch.from_numpy(w["cval"]).cuda()))
    ds.sync()
    ds.close()
    tf = PA.Tally()
    var_y = float(np.var(w["y"].astype(np.float64)))
    mean_y2 = float(np.mean(w["y"].astype(np.float64) ** 2))
    for p in range(w["P"]):
        t, f64, f32, fit64, fit32, cond, bounds = PA.oracle_trial(w, p)
        PA.check_fit(float(smse[p]), float(mse[p]), fit64, fit32, var_y, mean_y2, tf,
                     tag=f"trial {p}", bounds=bounds)
    PA.report(f"ladder {w['name']} (4,000 rows, 40 trials)", "trials", tf)
    assert tf.failed == 0, repr(tf)
    assert tf.checked >= 20, repr(tf)


def test_feynman_squaring_expression_scores_zero(gg):
    """Table 1's Feynman I.9.18 expression, written as a template, scores a
    scaled MSE at the FP32 noise floor on its own dataset (Section 4.4:
    NMSE 1e-6 is the FP32 precision level)."""
    w = synth.workload("l_squ", 0, n_rows=20_000, n_trials=1)
    # (x0 x1 x2) / ((x4 - x3)^2 + (x6 - x5)^2 + (x8 - x7)^2), heap layout, height 5
    tree = {0: "/", 1: "*", 2: "+", 3: "*", 4: "x2", 7: "x0", 8: "x1",
            5: "+", 6: "sq", 11: "sq", 12: "sq", 23: "-", 24: None, 25: "-",
            13: "-", 27: "x8", 28: "x7", 47: "x4", 48: "x3", 51: "x6", 52: "x5"}
    op, cv = heap_template(tree, 5)
    t = O.Template(op, cv, 5, n_features=9)
    np.testing.assert_allclose(O.eval_tree(t, w["X"]), synth.LADDER["squaring"](
        w["X"].astype(np.float64)), rtol=1e-6)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    smse, a, b, mse = (x.item() for x in ds.eval_batch(torch.from_numpy(op[None]).cuda(),
                                                          torch.from_numpy(cv[None]).cuda()))
    ds.sync()
    var_y = float(np.var(w["y"].astype(np.float64)))
    assert smse <= 1e-6 * var_y and abs(b - 1) < 1e-3 and mse / var_y <= 1e-6
    ds.close()
