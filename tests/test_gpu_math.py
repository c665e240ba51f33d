"""Accuracy of the interpreter's sin, cos, sqrt and log against FP64 (per-row
values through the C ABI), in FP32 units in the last place of the exact
result.  Arguments cover the reduction's range (|x| <= 2^17), the
neighbourhoods of multiples of pi/2, the library fallback beyond it, the
neighbourhoods of 1 and of sqrt(1/2) 2^k where log's reduction switches
exponent, and the special values."""
import math

import numpy as np
import pytest
import torch

from fixtures import heap_template

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()
    return pkg


def ulp32(v):
    v = np.abs(np.asarray(v, dtype=np.float64)).astype(np.float32)
    return np.spacing(np.maximum(v, np.float32(1.17549435e-38))).astype(np.float64)


def rows_of(gg, tok, x):
    X = torch.from_numpy(x.astype(np.float32)[:, None])
    ds = gg.Dataset(X, torch.zeros(x.size))
    op, cv = heap_template([tok, "x0", "x0"], 1)
    f = ds.eval_rows(torch.from_numpy(op[None]).cuda(), torch.from_numpy(cv[None]).cuda())
    ds.sync()
    ds.close()
    return f[0].cpu().numpy()


def trig_args():
    rng = np.random.default_rng(0)
    k = np.arange(-80000, 80001, 37)
    near = (k * (np.pi / 2)).astype(np.float32)
    near = np.concatenate([near, np.nextafter(near, np.float32(np.inf)),
                           np.nextafter(near, np.float32(-np.inf))])
    return np.concatenate([rng.uniform(-4, 4, 20000), rng.uniform(-2 ** 17, 2 ** 17, 20000),
                           10.0 ** rng.uniform(-30, 5, 5000), near]).astype(np.float32)


@pytest.mark.parametrize("tok,fn", [("sin", np.sin), ("cos", np.cos)])
def test_trig_within_two_ulp_in_range(gg, tok, fn):
    x = trig_args()
    x = x[np.abs(x) <= 2 ** 17]
    got = rows_of(gg, tok, x).astype(np.float64)
    want = fn(x.astype(np.float64))
    err = np.abs(got - want) / ulp32(want)
    assert err.max() <= 2.0, (x[np.argmax(err)], got[np.argmax(err)], want[np.argmax(err)])


@pytest.mark.parametrize("tok,fn", [("sin", np.sin), ("cos", np.cos)])
def test_trig_large_and_special_arguments(gg, tok, fn):
    x = np.array([2.0 ** 17 + 1, 3e5, -7.5e6, 1e30, -3.4e38, np.inf, -np.inf, np.nan, 0.0, -0.0],
                 dtype=np.float32)
    got = rows_of(gg, tok, x).astype(np.float64)
    want = fn(x.astype(np.float64))
    fin = np.isfinite(x)
    assert np.all(np.isnan(got[~fin]))
    assert np.all(np.abs(got[fin] - want[fin]) <= 2.0 * ulp32(want[fin]))


@pytest.mark.parametrize("tok", ["sqrtabs", "sqrt"])
def test_sqrt_within_one_ulp(gg, tok):
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-45, 38, 30000), rng.uniform(0, 10, 10000),
                        [0.0, 1e-45, 1e-40, 1.17549435e-38, 3.4e38, np.inf]]).astype(np.float32)
    if tok == "sqrtabs":
        x = np.concatenate([x, -x])
    got = rows_of(gg, tok, x).astype(np.float64)
    want = np.sqrt(np.abs(x.astype(np.float64)))
    fin = np.isfinite(want)
    err = np.abs(got[fin] - want[fin]) / ulp32(want[fin])
    assert err.max() <= 1.0
    assert np.all(np.isinf(got[~fin]))
    if tok == "sqrt":
        assert np.isnan(rows_of(gg, "sqrt", np.array([-1.0, -1e-30], np.float32))).all()


@pytest.mark.parametrize("tok", ["logabs", "log"])
def test_log_within_one_and_a_half_ulp(gg, tok):
    rng = np.random.default_rng(2)
    k = np.arange(-126, 128)
    edge = (np.sqrt(0.5) * 2.0 ** k).astype(np.float32)
    one = np.float32(1.0) + np.arange(-3000, 3001, dtype=np.float32) * np.float32(2.0 ** -20)
    x = np.concatenate([10.0 ** rng.uniform(-37.9, 38.5, 30000), rng.uniform(0, 4, 10000),
                        edge, np.nextafter(edge, np.float32(0)), np.nextafter(edge, np.float32(np.inf)),
                        one]).astype(np.float32)
    x = x[(x >= np.float32(1.17549435e-38)) & np.isfinite(x)]
    if tok == "logabs":
        x = np.concatenate([x, -x])
    got = rows_of(gg, tok, x).astype(np.float64)
    want = np.log(np.abs(x.astype(np.float64)))
    err = np.abs(got - want) / ulp32(want)
    i = np.argmax(err)
    assert err.max() <= 1.5, (x[i], got[i], want[i])


@pytest.mark.parametrize("tok", ["logabs", "log"])
def test_log_special_arguments(gg, tok):
    x = np.array([0.0, -0.0, 1e-45, 1e-40, np.inf, np.nan, 1.0, 3.4028235e38, 1.17549435e-38],
                 dtype=np.float32)
    got = rows_of(gg, tok, x).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        want = np.log(np.abs(x.astype(np.float64)))
    assert np.all(got[:2] == -np.inf) and got[4] == np.inf and np.isnan(got[5])
    assert got[6] == 0.0
    fin = np.isfinite(want)
    assert np.all(np.abs(got[fin] - want[fin]) <= 1.5 * ulp32(want[fin]))
    neg = rows_of(gg, tok, np.array([-1.0, -2.5, -1e-30], np.float32))
    if tok == "log":
        assert np.isnan(neg).all()
    else:
        np.testing.assert_allclose(neg, np.log([1.0, 2.5, 1e-30]), rtol=2e-7)


def test_exp_within_three_ulp(gg):
    """exp as the own form (the SFU base-2 exponential with the rounding of
    x log2 e recovered exactly) on |x| <= 87, the library beyond."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-87, 87, 30000), rng.uniform(-1, 1, 10000),
                        10.0 ** rng.uniform(-30, 1.9, 5000), -10.0 ** rng.uniform(-30, 1.9, 5000),
                        np.arange(-87, 88, dtype=np.float64)]).astype(np.float32)
    got = rows_of(gg, "exp", x).astype(np.float64)
    want = np.exp(x.astype(np.float64))
    err = np.abs(got - want) / ulp32(want)
    i = np.argmax(err)
    assert err.max() <= 3.0, (x[i], got[i], want[i])


def test_exp_large_and_special_arguments(gg):
    """Beyond |x| = 87 exp squares 2^(hi/2): about 6 units in the last place
    up to the overflow threshold, IEEE-rounded subnormals below."""
    x = np.array([87.5, 88.5, 88.7, 89.0, 100.0, -87.5, -95.0, -104.0, -120.0, np.inf, -np.inf,
                  np.nan, 0.0, -0.0], dtype=np.float32)
    got = rows_of(gg, "exp", x).astype(np.float64)
    with np.errstate(over="ignore"):
        want = np.exp(x.astype(np.float64))
    assert np.isinf(got[3]) and np.isinf(got[4]) and got[3] > 0  # beyond FP32's range
    assert got[9] == np.inf and got[10] == 0.0 and np.isnan(got[11])
    assert got[12] == 1.0 and got[13] == 1.0
    for i in (0, 1, 2, 5):  # normal results
        assert abs(got[i] - want[i]) <= 6.0 * ulp32(want[i]), (x[i], got[i], want[i])
    for i in (6, 7):  # subnormal results
        assert abs(got[i] - want[i]) <= 2.0 * 2.0 ** -149, (x[i], got[i], want[i])
    assert got[8] == 0.0


@pytest.mark.parametrize("n_uniform,reps", [(4000, 40), (36000, 200)])  # 4 and 8 rows per lane
@pytest.mark.parametrize("tok", ["sin", "cos", "exp", "logabs", "log", "sqrtabs", "sqrt"])
def test_unary_row_depends_only_on_its_argument(gg, tok, n_uniform, reps):
    """A row's value never depends on the other rows evaluated with it:
    arguments inside and outside each operator's common domain (zeros,
    subnormals, negatives, large magnitudes, infinities, NaN) are mixed,
    then permuted so that every row meets other neighbours; the values must
    be bit-identical row for row (both NaN counts as equal)."""
    rng = np.random.default_rng(4)
    special = np.array([0.0, -0.0, 1e-40, -1e-40, 3e-45, -2.5, -1e-30, 88.0, -90.0, 200.0,
                        -1e5, 3e5, -7e8, 1e30, np.inf, -np.inf, np.nan], dtype=np.float32)
    x = np.concatenate([rng.uniform(-4, 4, n_uniform).astype(np.float32),
                        np.tile(special, reps)])
    rng.shuffle(x)
    perm = rng.permutation(x.size)
    a = rows_of(gg, tok, x)
    b = rows_of(gg, tok, x[perm])
    back = np.empty_like(b)
    back[perm] = b
    same = (a.view(np.uint32) == back.view(np.uint32)) | (np.isnan(a) & np.isnan(back))
    i = int(np.argmin(same))
    assert same.all(), (x[i], a[i], back[i])
