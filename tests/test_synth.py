"""Seeded workload generators: determinism, shapes and recipe (CPU only)."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("cfg", sorted(synth.CONFIGS))
def test_workload_small_is_deterministic(cfg):
    a = synth.workload(cfg, 0, n_rows=300, n_trials=40)
    b = synth.workload(cfg, 0, n_rows=300, n_trials=40)
    for k in ("X", "op", "cval", "heights", "z"):
        np.testing.assert_array_equal(a[k], b[k])
    c = synth.CONFIGS[cfg]
    assert a["X"].shape == (300, c["F"]) and a["X"].dtype == np.float32
    assert a["op"].shape == (40, synth.n_nodes(c["h"]))
    if a["y_cands"] is None:  # closed-form target (Experiment III ladder)
        np.testing.assert_array_equal(a["y"], b["y"])
        assert a["y"].shape == (300,) and np.all(np.isfinite(a["y"]))
    else:
        ga = next(a["y_cands"]())
        gb = next(b["y_cands"]())
        np.testing.assert_array_equal(ga[0], gb[0])


def test_heights_and_padding():
    w = synth.workload("c3", 1, n_rows=10, n_trials=200)
    hs = w["heights"].astype(int)
    assert hs.min() >= 3 and hs.max() <= 7 and len(set(hs)) == 5
    for p in range(200):
        n = synth.n_nodes(hs[p])
        assert np.all(w["op"][p, n:] == synth.PAD)
        assert np.all(w["op"][p, :n] != synth.PAD)
        assert w["op"][p, 0] in synth.FULL_SET  # root is a function


def test_erc_leaves_recipe():
    w = synth.workload("c4", 0, n_rows=10, n_trials=50)
    stride = w["op"].shape[1]
    leaves = np.arange(stride) >= (stride - 1) // 2
    assert np.all(w["op"][:, leaves] == synth.ERC)
    internal_terms = (~leaves)[None, :] & (w["op"] >= synth.ERC)
    assert np.all(w["op"][internal_terms] >= synth.FEAT0)
    ercs = w["cval"][:, leaves]
    assert ercs.min() >= -5 and ercs.max() <= 5


def test_prefix_permutation_is_preorder():
    perm = synth.heap_to_prefix_perm(2)
    assert perm.tolist() == [0, 1, 3, 4, 2, 5, 6]


def test_fos_step_changes_only_the_subset():
    rng = np.random.default_rng(0)
    op, cv, _ = synth.random_templates(rng, 32, 4, 4, synth.FULL_SET, 3, 0.5)
    order = np.argsort(rng.random((32, op.shape[1])), axis=1)
    op2, cv2 = synth.fos_step_trials(rng, op, cv, 3, order)
    mask = synth.fos_subset_mask(op.shape[1], order[:, 3])
    assert np.all((op2 == op) | mask)


def test_make_target_noise():
    f = np.linspace(-1, 1, 1000)
    z = np.random.default_rng(0).standard_normal(1000)
    y = synth.make_target(f, z, 0.01)
    assert y.dtype == np.float32
    np.testing.assert_allclose(np.std(y.astype(float) - f), 0.01 * np.std(f) * np.std(z), rtol=1e-3)


def test_ladder_targets_are_the_table_expressions():
    # hand-evaluated rows of the Table 1 expressions
    x = np.array([[1, 2, 3, 4, 5, 6, 7, 8, 9], [2, 1, 1, 3, 1, 2, 4, 5, 2]], np.float64)
    L = synth.LADDER
    np.testing.assert_allclose(L["addition"](x), [45, 21])
    np.testing.assert_allclose(L["division"](x), [6 / 39, 4 / 17])
    np.testing.assert_allclose(L["subtraction"](x), [6 / 3, 4 / (1 - 3 + 4 - 2 + 2 - 5)])
    np.testing.assert_allclose(L["multiplication"](x), [6 / 3, 2 / -3])
    np.testing.assert_allclose(L["squaring"](x), [6 / 3, 2 / (4 + 4 + 9)])
