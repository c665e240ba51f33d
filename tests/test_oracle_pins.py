"""Pins of the FP64 oracle to things other than itself: the paper's worked
example (Fig. 1), hand-computed values, closed forms, invariants, library
special cases (numpy corrcoef / polyfit / var) and finite differences.

CPU only.  The last test plants mistakes in the oracle and checks that the
pins catch each one.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from fixtures import (ADD, AQ, COS, DIV, ERC, EXP, FEAT0, LOG, LOG_ABS, MUL, PAD, POW,
                      SIN, SQRT, SQRT_ABS, SQUARE, SUB, fig1, heap_template)


def T(tokens, h, **kw):
    op, cv = heap_template(tokens, h)
    return O.Template(op, cv, h, **kw)


# ---------------------------------------------------------------- Fig. 1 ----
def fig1_rpn_tokens(t):
    names = {ADD: "+", SUB: "-", MUL: "*", DIV: "/", SIN: "sin"}
    out = []
    for _, o, c in O.rpn(t):
        if o >= FEAT0:
            out.append(f"x{o - FEAT0}")
        elif o == ERC:
            out.append(f"{c:g}")
        else:
            out.append(names[o])
    return out


def test_fig1_rpn_and_encoding():
    op, cv, rows = fig1()
    t = O.Template(op, cv, 3, n_features=6)
    assert fig1_rpn_tokens(t) == rows["rpn"]
    Tr, Vr = O.paper_encoding(t)
    assert Tr == [int(v) for v in rows["type"]]
    assert Vr == [float(v) for v in rows["value"]]
    assert O.active_mask(t).astype(int).tolist() == [int(v) for v in rows["active"]]


def test_fig1_value_is_printed_expression():
    op, cv, _ = fig1()
    t = O.Template(op, cv, 3, n_features=6)
    X = np.random.default_rng(1).uniform(1.0, 2.0, (64, 6))
    want = -2.0 / (4.0 * X[:, 0] + X[:, 1])  # the expression printed in Fig. 1
    np.testing.assert_allclose(O.eval_tree(t, X), want, rtol=1e-15)


def test_fig1_prefix_layout_same_rpn():
    op, cv, rows = fig1()
    pop, pcv = synth.to_prefix(op[None], cv[None], np.array([3]))
    t = O.Template(pop[0], pcv[0], 3, layout="prefix", n_features=6)
    assert fig1_rpn_tokens(t) == rows["rpn"]
    X = np.random.default_rng(2).uniform(1.0, 2.0, (16, 6))
    np.testing.assert_array_equal(O.eval_tree(t, X),
                                  O.eval_tree(O.Template(op, cv, 3), X))


# ---------------------------------------------------- hand-computed values ----
X2 = np.array([[2.0, 5.0], [3.0, 4.0], [6.0, 3.0], [-3.0, 0.0]])


@pytest.mark.parametrize("tok,want", [
    ("+", [7.0, 7.0, 9.0, -3.0]),
    ("-", [-3.0, -1.0, 3.0, -3.0]),
    ("*", [10.0, 12.0, 18.0, -0.0]),
    ("aq", [2 / math.sqrt(26), 3 / math.sqrt(17), 6 / math.sqrt(10), -3.0]),
    ("/", [0.4, 0.75, 2.0, -math.inf]),
    ("pow", [32.0, 81.0, 216.0, 1.0]),
])
def test_binary_hand_values(tok, want):
    t = T([tok, "x0", "x1"], 1)
    np.testing.assert_allclose(O.eval_tree(t, X2), want, rtol=1e-15)


@pytest.mark.parametrize("tok,x,want", [
    ("sin", math.pi / 6, 0.5), ("cos", math.pi / 3, 0.5), ("exp", 1.0, math.e),
    ("logabs", -math.e, 1.0), ("sqrtabs", -9.0, 3.0), ("sq", -3.0, 9.0),
    ("log", math.e ** 2, 2.0), ("sqrt", 16.0, 4.0),
])
def test_unary_hand_values_use_left_child(tok, x, want):
    # child 0 holds x0 = x; child 1 (an intron) holds x1 = 100
    t = T([tok, "x0", "x1"], 1)
    X = np.array([[x, 100.0]])
    np.testing.assert_allclose(O.eval_tree(t, X), [want], rtol=1e-14)


def test_unprotected_log_sqrt_nan_and_protected_zero():
    X = np.array([[-1.0, 0.0]])
    assert np.isnan(O.eval_tree(T(["log", "x0", "x1"], 1), X)[0])
    assert np.isnan(O.eval_tree(T(["sqrt", "x0", "x1"], 1), X)[0])
    assert O.eval_tree(T(["logabs", "x1", "x0"], 1), X)[0] == -math.inf
    assert O.eval_tree(T(["sqrtabs", "x1", "x0"], 1), X)[0] == 0.0


def test_pow_special_cases_and_reductions():
    """pow(a, b) follows C99 pow: a negative base with an integer exponent is
    defined, with a non-integer exponent it is NaN (so the fitness is +inf),
    0 to a negative power is inf; x^2 and x^0.5 reduce to the square and the
    square root."""
    t = T(["pow", "x0", "x1"], 1)
    got = O.eval_tree(t, np.array([[-2.0, 3.0], [-2.0, 0.5], [0.0, -1.0], [4.0, -0.5]]))
    assert got[0] == -8.0 and np.isnan(got[1]) and got[2] == math.inf and got[3] == 0.5
    assert not O.fitness(got, np.arange(4.0))["finite"]
    X = np.random.default_rng(4).uniform(0.1, 3.0, (64, 1))
    np.testing.assert_allclose(O.eval_tree(T(["pow", "x0", "2"], 1), X), X[:, 0] ** 2, rtol=1e-15)
    np.testing.assert_allclose(O.eval_tree(T(["pow", "x0", "0.5"], 1), X), np.sqrt(X[:, 0]),
                               rtol=1e-15)


def test_pow_exponent_derivative_at_negative_base():
    """READING: d a^b / db at a < 0 and integer b is the real part of the
    derivative of the principal complex power, a^b (ln|a| + i pi)."""
    a = np.array([-2.0, -0.5, -3.0])
    b = np.array([3.0, 2.0, -1.0])
    out = np.power(a, b)
    _, db = O.gp._dapply(POW, a, b, out)
    want = np.real(np.power(a.astype(complex), b) * np.log(a.astype(complex)))
    np.testing.assert_allclose(db, want, rtol=1e-14)


def test_pow_ambiguous_rows():
    """Rows where pow has a negative base and an exponent next to an integer
    (FP32 rounding decides between a number and NaN) are flagged; a positive
    base, or an exponent far from an integer, is not."""
    t = T(["pow", "x0", "x1"], 1)
    X = np.array([[-2.0, 3.0], [-2.0, 0.5], [2.0, 3.0], [-2.0, 3.0000001], [-2.0, 1e6 + 0.5],
                  [-2.0, 3.1]])
    np.testing.assert_array_equal(O.pow_ambiguous_rows(t, X),
                                  [True, False, False, True, True, False])
    # nested: the flag follows the active pow node wherever it sits
    t2 = T(["+", "x1", "pow", None, None, "x0", "x1"], 2)
    np.testing.assert_array_equal(O.pow_ambiguous_rows(t2, X[:3]), [True, False, False])


def test_height2_hand_value():
    # (x0 AQ x1) - (2 * x0) at x0 = 3, x1 = 4: 3/sqrt(17) - 6
    t = T(["-", "aq", "*", "x0", "x1", "2", "x0"], 2)
    np.testing.assert_allclose(O.eval_tree(t, np.array([[3.0, 4.0]])),
                               [-5.272393124891001], rtol=1e-15)


def test_aq_zero_denominator_is_identity():
    t = T(["aq", "x0", "0"], 1)
    X = np.array([[1.5], [-2.25]])
    np.testing.assert_array_equal(O.eval_tree(t, X), X[:, 0])


def test_height0_terminal_tree():
    assert O.eval_tree(T(["x1"], 0), X2).tolist() == X2[:, 1].tolist()
    assert O.eval_tree(T(["2.5"], 0), X2).tolist() == [2.5] * 4


# ------------------------------------------------------------- active set ----
def test_active_function_at_leaf_is_invalid():
    t = T(["+", "x0", "*"], 1)
    with pytest.raises(O.InvalidTemplate):
        O.eval_tree(t, X2)


def test_active_pad_and_bad_feature_are_invalid():
    with pytest.raises(O.InvalidTemplate):
        O.eval_tree(T(["+", "x0", None], 1), X2)
    with pytest.raises(O.InvalidTemplate):
        O.active_mask(T(["+", "x0", "x7"], 1, n_features=2))


def test_intron_invariance_random_trees():
    rng = np.random.default_rng(5)
    X = rng.uniform(-2, 2, (200, 4))
    op, cv, hs = synth.random_templates(rng, 60, 4, 4, synth.FULL_SET, 4, 0.6)
    for p in range(op.shape[0]):
        t = O.Template(op[p], cv[p], 4, n_features=4)
        mask = O.active_mask(t)
        f = O.eval_tree(t, X)
        op2 = op[p].copy()
        cv2 = cv[p].copy()
        op2[~mask] = rng.integers(0, 256, (~mask).sum())
        cv2[~mask] = rng.normal(0, 100, (~mask).sum())
        t2 = O.Template(op2, cv2, 4, n_features=4)
        np.testing.assert_array_equal(O.eval_tree(t2, X), f)
        assert [x[:2] for x in O.rpn(t2)] == [x[:2] for x in O.rpn(t)]


# --------------------------------------------------------------- fitness ----
def rand_xy(seed=0, n=500, f=3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-2, 2, (n, f))
    return rng, X


def test_generating_tree_scores_zero():
    rng, X = rand_xy(1)
    t = T(["+", "sin", "*", "x0", None, "x1", "x2"], 2)
    y = O.eval_tree(t, X)
    fit = O.fitness(O.eval_tree(t, X), y)
    assert fit["smse"] <= 1e-28 * np.var(y)
    assert fit["mse"] == 0.0
    assert abs(fit["b"] - 1.0) < 1e-13 and abs(fit["a"]) < 1e-13


def test_affine_wrapper_leaves_smse_unchanged():
    rng, X = rand_xy(2)
    y = np.sin(X[:, 0]) + 0.3 * X[:, 1] ** 2
    inner = ["aq", "x0", "cos", None, None, "x1", "x2"]
    t = T(inner, 2)
    # c1 + c2 * T: ADD(ERC 1.75, MUL(ERC -3.5, T)) with T re-rooted below MUL
    wrapped = {0: "+", 1: "1.75", 2: "*", 5: "-3.5", 6: "aq", 13: "x0", 14: "cos", 29: "x1"}
    tw = T(wrapped, 4)
    f = O.eval_tree(t, X)
    fw = O.eval_tree(tw, X)
    np.testing.assert_allclose(fw, 1.75 + np.float32(-3.5) * f, rtol=1e-14)
    a = O.fitness(f, y)
    b = O.fitness(fw, y)
    assert abs(a["smse"] - b["smse"]) <= 1e-10 * a["smse"]
    assert abs(b["b"] * -3.5 - a["b"]) <= 1e-10 * abs(a["b"])


def test_constant_tree_scores_var_y():
    rng, X = rand_xy(3)
    y = rng.normal(2.0, 3.0, X.shape[0])
    fit = O.fitness(O.eval_tree(T(["*", "2", "3"], 1), X), y)
    assert fit["b"] == 0.0
    np.testing.assert_allclose(fit["smse"], np.var(y), rtol=1e-13)
    np.testing.assert_allclose(fit["a"], np.mean(y), rtol=1e-13)


def test_single_feature_tree_is_one_minus_rho_squared():
    rng, X = rand_xy(4)
    y = np.exp(X[:, 0]) + rng.normal(0, 0.5, X.shape[0])
    rho = np.corrcoef(X[:, 0], y)[0, 1]
    fit = O.fitness(O.eval_tree(T(["x0"], 0), X), y)
    np.testing.assert_allclose(fit["smse"], np.var(y) * (1 - rho ** 2), rtol=1e-11)


def test_scaling_matches_polyfit_and_nmse():
    rng, X = rand_xy(5)
    t = T(["-", "sin", "x1", "x0"], 2)
    f = O.eval_tree(t, X)
    y = rng.normal(size=f.size) + 0.7 * f
    fit = O.fitness(f, y)
    b, a = np.polyfit(f, y, 1)
    np.testing.assert_allclose([fit["a"], fit["b"]], [a, b], rtol=1e-10)
    np.testing.assert_allclose(fit["mse"], np.mean((f - y) ** 2), rtol=1e-13)
    np.testing.assert_allclose(fit["nmse"], fit["mse"] / np.var(y), rtol=1e-13)
    assert fit["smse"] <= fit["mse"]


def test_infinite_fitness_rules():
    X = np.array([[0.0], [1.0], [2.0]])
    y = np.array([1.0, 2.0, 0.5])
    fit = O.fitness(O.eval_tree(T(["logabs", "x0"], 1), X), y)
    assert fit["smse"] == math.inf and fit["a"] == 0.0 and fit["b"] == 0.0
    big = T(["exp", "*", None, "40", "x0"], 2)  # exp(80) > 2**50 at x0 = 2
    assert O.fitness(O.eval_tree(big, X), y)["smse"] == math.inf
    ok = T(["exp", "*", None, "10", "x0"], 2)  # exp(20) < 2**50
    assert np.isfinite(O.fitness(O.eval_tree(ok, X), y)["smse"])


def test_constant_threshold():
    rng, X = rand_xy(6)
    y = rng.normal(size=X.shape[0])
    flat = 1.0 + 1e-8 * X[:, 0]
    assert O.fitness(flat, y)["b"] == 0.0
    assert O.fitness(1.0 + 1e-4 * X[:, 0], y)["b"] != 0.0


# -------------------------------------------------------------- gradient ----
def c4_like_trees(n=40, seed=7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((300, 3))
    op, cv, hs = synth.random_templates(rng, n, 3, 3, synth.FULL_SET, 3, 0.75,
                                        p_feature=0.5)
    y = np.sin(X[:, 0]) * X[:, 1] + 0.5 * X[:, 2]
    return X, y, op, cv


# one hand-built tree per function, each with an ERC below it (height 3)
OP_TREES = [
    ["+", "sin", "x1", "*", None, None, None, "0.7", "x0"],
    ["-", "cos", "x1", "+", None, None, None, "x0", "0.3"],
    ["*", "exp", "x1", "*", None, None, None, "x2", "-0.4"],
    ["+", "logabs", "x1", "+", None, None, None, "x0", "2.5"],
    ["+", "sqrtabs", "x1", "-", None, None, None, "x0", "-2.5"],
    ["aq", "x0", "*", None, None, "1.3", "x2"],
    ["aq", "*", "x2", "0.9", "x1"],
    ["/", "x1", "+", None, None, "x0", "3.5"],
    ["+", "sq", "x0", "-", None, None, None, "x1", "0.6"],
    ["+", "log", "x2", "+", None, None, None, "x0", "4.5"],
    ["+", "sqrt", "x2", "+", None, None, None, "x1", "4.5"],
    ["pow", "sqrtabs", "+", "x0", None, "x1", "0.5"],
    ["pow", "1.3", "sin", None, None, "x0"],
    ["pow", "sqrtabs", "0.8", "x2"],
    ["pow", "exp", "+", "*", None, "x1", "x2", "x0", "0.3"],
]


def fd_cases():
    X, y, op, cv = c4_like_trees()
    for p in range(op.shape[0]):
        yield O.Template(op[p], cv[p], 3, n_features=3)
    for toks in OP_TREES:
        yield T(toks, 3, n_features=3)


@pytest.mark.parametrize("mode", ["smse", "mse"])
def test_reverse_mode_matches_central_fd(mode):
    X, y, op, cv = c4_like_trees()
    checked = 0
    for t in fd_cases():
        g, fit = O.grad(t, X, y, mode)
        if not fit["finite"]:
            continue
        fd = O.fd_grad(t, X, y, mode)
        # FD rounding noise is about 1e-16 * smse / h, h >= 1e-6
        atol = 1e-6 * np.max(np.abs(fd)) + 1e-8 * max(fit[mode], 1e-300)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=atol)
        checked += np.count_nonzero(fd)
    assert checked > 10


def test_gradient_scale_and_shift_invariance():
    rng, X = rand_xy(8)
    y = np.cos(X[:, 0]) + X[:, 1]
    for toks in (["*", "1.5", "sin", None, None, "x0"], ["+", "-0.5", "sin", None, None, "x0"]):
        t = T(toks, 2)
        g, fit = O.grad(t, X, y)
        assert abs(g[1]) <= 1e-12 * abs(fit["b"]) + 1e-15


def test_gradient_perturbation_probe():
    """grad's perturb: a zero perturbation is the plain gradient; a
    perturbation of relative size rel moves a well-conditioned gradient by
    O(rel)."""
    rng, X = rand_xy(14)
    y = np.cos(X[:, 0]) + X[:, 1]
    t = T(["+", "*", "sin", "x0", "1.7", "x1", None], 2)
    g0, _ = O.grad(t, X, y)
    g1, _ = O.grad(t, X, y, perturb=(0.0, rng))
    np.testing.assert_array_equal(g0, g1)
    g2, _ = O.grad(t, X, y, perturb=(1e-7, rng))
    assert 0 < np.max(np.abs(g2 - g0)) <= 1e-4 * np.max(np.abs(g0))


def test_envelope_partials_vanish():
    rng, X = rand_xy(9)
    t = T(["aq", "x0", "sin", None, None, "x1"], 2)
    f = O.eval_tree(t, X)
    y = rng.normal(size=f.size) + f
    fit = O.fitness(f, y)
    loss = lambda a, b: np.mean((y - a - b * f) ** 2)
    h = 1e-6
    da = (loss(fit["a"] + h, fit["b"]) - loss(fit["a"] - h, fit["b"])) / (2 * h)
    db = (loss(fit["a"], fit["b"] + h) - loss(fit["a"], fit["b"] - h)) / (2 * h)
    assert abs(da) < 1e-8 and abs(db) < 1e-8
    np.testing.assert_allclose(loss(fit["a"], fit["b"]), fit["smse"], rtol=1e-12)


def test_fp32_emulation_close_on_benign_tree():
    rng, X = rand_xy(10)
    t = T(["+", "*", "aq", "x0", "1.25", "x1", "x2"], 2)
    f64 = O.eval_tree(t, X)
    f32 = O.eval_tree_f32(t, X.astype(np.float32))
    assert f32.dtype == np.float32
    np.testing.assert_allclose(f32, f64, rtol=1e-6, atol=1e-6)


def test_fp32_emulation_rounds_every_node():
    """Each node's value is rounded to FP32 before its parent uses it:
    (x0 + x1) - x0 is 0 in FP32 when x1 is below half a unit in the last
    place of x0 (1 + 2^-30 and 3 + 2^-23 round to 1 and 3), while FP64
    keeps x1; (x0 * x0) - x1 with x0 = 1 + 2^-12, x1 = 1 + 2^-11 is 0 in FP32
    (1 + 2^-11 + 2^-24 rounds to even, down to 1 + 2^-11) and 2^-24 in FP64."""
    X = np.array([[1.0, 2.0 ** -30], [3.0, 2.0 ** -23]], dtype=np.float32)
    t = T(["-", "+", "x0", "x0", "x1"], 2)
    np.testing.assert_array_equal(O.eval_tree_f32(t, X), [0.0, 0.0])
    np.testing.assert_array_equal(O.eval_tree(t, X), [2.0 ** -30, 2.0 ** -23])
    X2 = np.array([[1.0 + 2.0 ** -12, 1.0 + 2.0 ** -11]], dtype=np.float32)
    t2 = T(["-", "*", "x1", "x0", "x0"], 2)
    assert O.eval_tree_f32(t2, X2)[0] == 0.0
    assert O.eval_tree(t2, X2)[0] == 2.0 ** -24


def test_gradient_scale_terms_hand_values():
    """oracle.grad's with_abs scale G = sum_i s_i |d f_i / d c| by hand.
    X = (1, 2, 3), y = (1, 3, 2).  Tree c * x0 with c = 2: f = (2, 4, 6),
    b* = 1/4, a* = 1, smse = 1/2; the smse gradient is 0 (c only scales f)
    and G = (2/3)(1/4) sum (1 + f_i/4 + y_i) x_i = 13/3; for mse the gradient
    is (2/3) sum (f_i - y_i) x_i = 10 and G = (2/3) sum (f_i + y_i) x_i = 82/3.
    Tree x0 (x0 + c) with c = 1: f = (2, 6, 12), b* = 3/38, a* = 28/19,
    residuals (12, -20, 8)/19, gradient (1/19) sum r_i x_i = -4/361 and
    G = (1/19) sum (28/19 + 3 f_i/38 + y_i) x_i = 490/361."""
    X = np.array([[1.0], [2.0], [3.0]])
    y = np.array([1.0, 3.0, 2.0])
    t = T(["*", "2", "x0"], 1)
    g, fit, ga = O.grad(t, X, y, with_abs=True)
    assert math.isclose(fit["a"], 1.0, rel_tol=1e-14) and math.isclose(fit["b"], 0.25, rel_tol=1e-14)
    assert math.isclose(fit["smse"], 0.5, rel_tol=1e-14)
    assert abs(g[1]) < 1e-15 and math.isclose(ga[1], 13 / 3, rel_tol=1e-14)
    g, fit, ga = O.grad(t, X, y, "mse", with_abs=True)
    assert math.isclose(g[1], 10.0, rel_tol=1e-14) and math.isclose(ga[1], 82 / 3, rel_tol=1e-14)
    t = T(["*", "x0", "+", None, None, "x0", "1"], 2)
    g, fit, ga = O.grad(t, X, y, with_abs=True)
    assert math.isclose(fit["b"], 3 / 38, rel_tol=1e-14)
    assert math.isclose(fit["a"], 28 / 19, rel_tol=1e-14)
    assert math.isclose(g[6], -4 / 361, rel_tol=1e-12)
    assert math.isclose(ga[6], 490 / 361, rel_tol=1e-14)
    assert np.count_nonzero(ga) == 1 and np.count_nonzero(g) == 1


def test_perturbed_evaluation_bounds():
    rng, X = rand_xy(12)
    t = T(["*", "x0", "x1"], 1)
    f = O.eval_tree(t, X)
    np.testing.assert_array_equal(O.eval_tree_perturbed(t, X, 0.0, rng), f)
    fp = O.eval_tree_perturbed(t, X, 1e-3, rng)
    np.testing.assert_allclose(np.abs(fp / f - 1.0), 1e-3, rtol=1e-9)
    # sin of a large argument: a tiny relative change of the argument moves it a lot
    ts = T(["sin", "*", None, "1e6", "x0"], 2)
    spread = np.abs(O.eval_tree_perturbed(ts, X, 1e-7, rng) - O.eval_tree(ts, X))
    assert np.median(spread) > 1e-2


def test_condition_bound_closed_forms():
    rng, X = rand_xy(13)
    rel = 1e-6
    # one multiplication: the bound is rel * |x0 x1|
    t = T(["*", "x0", "x1"], 1)
    np.testing.assert_allclose(O.condition_bound(t, X, rel), rel * np.abs(X[:, 0] * X[:, 1]),
                               rtol=1e-12)
    # exp(x0 * x1): errors at the product are amplified by |x0 x1|
    t = T(["exp", "*", None, "x0", "x1"], 2)
    e = np.exp(X[:, 0] * X[:, 1])
    np.testing.assert_allclose(O.condition_bound(t, X, rel),
                               rel * (e + e * np.abs(X[:, 0] * X[:, 1])), rtol=1e-12)
    # sin(c x0): slope bound 1 at the sin node, so the product's size counts fully
    t = T(["sin", "*", None, "300", "x0"], 2)
    np.testing.assert_allclose(O.condition_bound(t, X, rel),
                               rel * (np.abs(np.sin(300 * X[:, 0])) + 300 * np.abs(X[:, 0])),
                               rtol=1e-12)


def test_condition_bound_per_operator_closed_form():
    """The per-operator form: each function node carries its own relative
    error, so exp(x0 * x1) gets rel_exp e + rel_mul e |x0 x1| (a mistake that
    swapped the two, or used one for both, moves the bound)."""
    rng, X = rand_xy(17)
    rel = {O.MUL: 1e-7, O.EXP: 6e-7}
    t = T(["exp", "*", None, "x0", "x1"], 2)
    e = np.exp(X[:, 0] * X[:, 1])
    np.testing.assert_allclose(O.condition_bound(t, X, rel),
                               6e-7 * e + 1e-7 * e * np.abs(X[:, 0] * X[:, 1]), rtol=1e-12)
    # a uniform number is the same as a table holding it for every operator
    u = {k: 3e-7 for k in (O.MUL, O.EXP)}
    np.testing.assert_allclose(O.condition_bound(t, X, u), O.condition_bound(t, X, 3e-7),
                               rtol=1e-12)


def test_eval_batch_matches_single():
    rng, X = rand_xy(11)
    y = X[:, 0] * 2
    op, cv, hs = synth.random_templates(rng, 5, 2, 3, synth.BASIC_SET, 3, 0.7)
    out = O.eval_batch(op, cv, hs, 3, X, y)
    for p in range(5):
        fit = O.fitness(O.eval_tree(O.Template(op[p], cv[p], int(hs[p])), X), y)
        assert out["smse"][p] == fit["smse"]


# ------------------------------------------------- planted-mistake check ----
PINS = [test_fig1_rpn_and_encoding, test_fig1_value_is_printed_expression,
        test_height2_hand_value, test_generating_tree_scores_zero,
        test_affine_wrapper_leaves_smse_unchanged, test_constant_tree_scores_var_y,
        test_single_feature_tree_is_one_minus_rho_squared, test_scaling_matches_polyfit_and_nmse,
        lambda: test_reverse_mode_matches_central_fd("smse"),
        lambda: [test_binary_hand_values(k, w) for k, w in [
            ("-", [-3.0, -1.0, 3.0, -3.0]), ("aq", [2 / math.sqrt(26), 3 / math.sqrt(17), 6 / math.sqrt(10), -3.0]),
            ("/", [0.4, 0.75, 2.0, -math.inf]), ("pow", [32.0, 81.0, 216.0, 1.0])]],
        lambda: test_unary_hand_values_use_left_child("sin", math.pi / 6, 0.5),
        test_intron_invariance_random_trees, test_fp32_emulation_rounds_every_node,
        test_gradient_scale_terms_hand_values]


def _pins_fail():
    for pin in PINS:
        try:
            pin()
        except (AssertionError, O.InvalidTemplate, ValueError, KeyError):
            return True
    return False


def test_pins_catch_planted_mistakes(monkeypatch):
    gp = O.gp
    real_apply, real_dapply, real_fitness = gp._apply, gp._dapply, gp.fitness
    real_children = gp.Template.children
    mistakes = {
        "sub operands swapped": lambda o, a, b=None, xp=np: (b - a) if o == SUB else real_apply(o, a, b),
        "aq drops the +1": lambda o, a, b=None, xp=np: (a / np.sqrt(b * b)) if o == AQ else real_apply(o, a, b),
        "div transposed": lambda o, a, b=None, xp=np: (b / a) if o == DIV else real_apply(o, a, b),
        "mul as add": lambda o, a, b=None, xp=np: (a + b) if o == MUL else real_apply(o, a, b),
        "pow operands swapped": lambda o, a, b=None, xp=np: (np.power(b, a)) if o == POW
        else real_apply(o, a, b),
    }
    for name, fn in mistakes.items():
        monkeypatch.setattr(gp, "_apply", fn)
        assert _pins_fail(), name
        monkeypatch.setattr(gp, "_apply", real_apply)

    def unary_right(self, pos, depth):
        l, r = real_children(self, pos, depth)
        return (r, l) if int(self.op[pos]) in gp.UNARY else (l, r)
    monkeypatch.setattr(gp.Template, "children", unary_right)
    assert _pins_fail(), "unary takes child 1"
    monkeypatch.setattr(gp.Template, "children", real_children)

    def uncentred(f, y):
        out = real_fitness(f, y)
        if out["finite"]:
            f = np.asarray(f, float); y = np.asarray(y, float)
            b = np.sum(f * y) / max(np.sum(f * f), 1e-300)
            out = dict(out, b=b, a=0.0, smse=float(np.mean((y - b * f) ** 2)))
        return out
    monkeypatch.setattr(gp, "fitness", uncentred)
    monkeypatch.setattr(O, "fitness", uncentred)
    assert _pins_fail(), "scaling without intercept"
    monkeypatch.setattr(gp, "fitness", real_fitness)
    monkeypatch.setattr(O, "fitness", real_fitness)

    def dsin_sign(o, a, b, out):
        if o == SIN:
            return -np.cos(a), None
        return real_dapply(o, a, b, out)
    monkeypatch.setattr(gp, "_dapply", dsin_sign)
    assert _pins_fail(), "wrong sign in d sin"
    monkeypatch.setattr(gp, "_dapply", real_dapply)

    real_f32, real_grad = gp.eval_tree_f32, gp.grad
    rounded_at_end = lambda t, X: gp.eval_tree(t, X).astype(np.float32)
    monkeypatch.setattr(gp, "eval_tree_f32", rounded_at_end)
    monkeypatch.setattr(O, "eval_tree_f32", rounded_at_end)
    assert _pins_fail(), "FP32 emulation rounds only the result"
    monkeypatch.setattr(gp, "eval_tree_f32", real_f32)
    monkeypatch.setattr(O, "eval_tree_f32", real_f32)

    def scale_without_y(t, X, y, mode="smse", with_abs=False):
        out = real_grad(t, X, y, mode, with_abs)
        if not with_abs:
            return out
        g, fit, ga = out
        # the |y_i| term of the scale dropped
        _, _, ga0 = real_grad(t, X, np.zeros_like(np.asarray(y, float)), mode, True)
        return g, fit, ga0
    monkeypatch.setattr(gp, "grad", scale_without_y)
    monkeypatch.setattr(O, "grad", scale_without_y)
    assert _pins_fail(), "gradient scale drops |y|"
    monkeypatch.setattr(gp, "grad", real_grad)
    monkeypatch.setattr(O, "grad", real_grad)
    assert not _pins_fail()
