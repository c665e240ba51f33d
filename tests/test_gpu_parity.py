"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Small cases span several row tiles and a ragged
tail; the full-size cases run every configuration at its benchmark size and
compare a sample of trials the oracle computes one by one."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from fixtures import fig1, heap_template
import parity as PA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_30954_gb300 as pkg
    pkg.lib()  # raises ImportError if the library is not built
    return pkg


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def run_case(gg, w, sample=None, flags=0, check_rows=True, layout=0, tuned=False):
    """tuned: the launch configuration the benchmark times (autotuned tile
    shape, CUDA graph replay on a side stream)."""
    X = torch.from_numpy(w["X"])
    y = torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    hs = dev(w["heights"]) if len(set(w["heights"].tolist())) > 1 else None
    if w.get("uses_pow"):
        flags |= gg.F_POW
    if tuned:
        ds.autotune(op, cv, hs, layout=layout, flags=flags)
        st = torch.cuda.Stream()
        outs = [torch.full((w["P"],), -7.0, device="cuda") for _ in range(4)]
        for _ in range(2):  # the second call replays the captured graph
            ds.eval_batch(op, cv, hs, layout=layout, flags=flags | gg.F_GRAPH, stream=st, out=outs)
        st.synchronize()
        smse, a, b, mse = outs
    else:
        smse, a, b, mse = ds.eval_batch(op, cv, hs, layout=layout, flags=flags)
    idx = range(w["P"]) if sample is None else sample
    rows = None
    if check_rows:
        rows = ds.eval_rows(op, cv, hs, layout=layout, flags=flags & ~gg.F_GRAPH).cpu().numpy()
    ds.sync()
    smse, a, b, mse = (t.cpu().numpy() for t in (smse, a, b, mse))
    tr, tf = PA.Tally(), PA.Tally()
    var_y = float(np.var(w["y"].astype(np.float64)))
    mean_y2 = float(np.mean(w["y"].astype(np.float64) ** 2))
    for p in idx:
        t, f64, f32, fit64, fit32, cond, bounds = PA.oracle_trial(w, p)
        if rows is not None:
            PA.check_rows(rows[p], f64, f32, tr, tag=f"trial {p}", cond=cond)
        PA.check_fit(float(smse[p]), float(mse[p]), fit64, fit32, var_y, mean_y2, tf,
                     tag=f"trial {p}", bounds=bounds)
    ds.close()
    return tr, tf, (smse, a, b, mse)


def assert_tally(t, min_checked=1, max_excl=0.08, name=None, what=None):
    if name:
        PA.report(name, what, t)
    assert t.failed == 0, repr(t)
    assert t.checked >= min_checked, repr(t)
    assert t.excluded <= max_excl * (t.checked + t.excluded) + 2, repr(t)


# ------------------------------------------------------------------ basics --
def test_fig1_on_gpu(gg):
    op, cv, _ = fig1()
    X = np.random.default_rng(0).uniform(1, 2, (777, 6)).astype(np.float32)
    y = (np.sin(X[:, 0]) + X[:, 1]).astype(np.float32)
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(y))
    f = ds.eval_rows(dev(op[None]), dev(cv[None])).cpu().numpy()[0]
    want = -2.0 / (4.0 * X[:, 0].astype(np.float64) + X[:, 1])
    np.testing.assert_allclose(f, want, rtol=2e-7)
    smse, a, b, mse = ds.eval_batch(dev(op[None]), dev(cv[None]))
    fit = O.fitness(want, y)
    assert abs(smse.item() - fit["smse"]) <= 1e-4 * fit["smse"]
    ds.sync()
    ds.close()


@pytest.mark.parametrize("cfg,n_rows,n_trials", [
    ("c1", 1000, 256), ("c1", 3001, 97), ("c2", 5003, 64), ("c3", 4099, 48),
    ("c4", 2500, 40), ("c5", 3000, 32), ("t2", 5003, 64),
])
def test_small_configs_rows_and_fitness(gg, cfg, n_rows, n_trials):
    w = PA.build(cfg, n_rows, n_trials)
    tr, tf, _ = run_case(gg, w)
    assert_tally(tr, min_checked=n_rows * n_trials // 3)
    assert_tally(tf, min_checked=n_trials // 3, max_excl=0.2)


@pytest.mark.parametrize("cfg", ["c1", "c3"])
def test_prefix_layout_matches_heap(gg, cfg):
    wh = PA.build(cfg, 2000, 40, layout="heap")
    wp = PA.build(cfg, 2000, 40, layout="prefix")
    _, tf, outs_p = run_case(gg, wp, layout=1, check_rows=False)
    assert_tally(tf)
    _, _, outs_h = run_case(gg, wh, layout=0, check_rows=False)
    np.testing.assert_array_equal(outs_p[0], outs_h[0])


def test_grouped_sums_large_n(gg):
    # N >= 32768 selects the 8-rows-per-lane kernel with grouped sums
    w = PA.build("c2", 40_000, 48)
    tr, tf, _ = run_case(gg, w, check_rows=True)
    assert_tally(tr, min_checked=40_000 * 10)
    assert_tally(tf, min_checked=16)


def test_exact_flag_and_plain_form_agree(gg):
    w = PA.build("c2", 9000, 40)
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    s0 = ds.eval_batch(op, cv)[0]
    s1 = ds.eval_batch(op, cv, flags=gg.F_EXACT)[0]
    s2 = ds.eval_plain(op, cv)[0]
    ds.sync()
    for s in (s1, s2):
        a, b = s0.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
        fin = np.isfinite(a)
        assert np.array_equal(fin, np.isfinite(b))
        np.testing.assert_allclose(b[fin], a[fin], rtol=2e-4, atol=1e-8 * np.var(w["y"]))
    ds.close()


def test_graph_replay_and_host_batches(gg):
    w = PA.build("c1", 1000, 256)
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    ref = [t.clone() for t in ds.eval_batch(op, cv)]
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    outs = [torch.empty(256, device="cuda") for _ in range(4)]
    for _ in range(3):
        with torch.cuda.stream(st):
            ds.eval_batch(op, cv, flags=gg.F_GRAPH, out=outs, stream=st)
        st.synchronize()
        for r, o in zip(ref, outs):
            assert torch.equal(r, o)
    hop = torch.from_numpy(w["op"]).pin_memory()
    hcv = torch.from_numpy(w["cval"]).pin_memory()
    hout = ds.eval_batch(hop, hcv)
    torch.cuda.synchronize()
    for r, o in zip(ref, hout):
        assert not o.is_cuda
        assert torch.equal(r.cpu(), o)
    ds.sync()
    ds.close()


def test_autotune_keeps_results(gg):
    w = PA.build("c2", 50_000, 300)
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    a = ds.eval_batch(op, cv)[0].cpu().numpy()
    ds.autotune(op, cv)
    b = ds.eval_batch(op, cv)[0].cpu().numpy()
    ds.sync()
    fin = np.isfinite(a)
    np.testing.assert_array_equal(fin, np.isfinite(b))
    np.testing.assert_allclose(b[fin], a[fin], rtol=2e-4, atol=1e-8 * np.var(w["y"]))
    ds.close()


# -------------------------------------------------------------- edge cases --
def test_empty_batch_and_single_row(gg):
    X = torch.tensor([[0.5, -1.0]], dtype=torch.float32)
    y = torch.tensor([2.0])
    ds = gg.Dataset(X, y)
    op, cv = heap_template(["+", "x0", "sin", None, None, "x1"], 2)
    empty = torch.zeros((0, 7), dtype=torch.uint8, device="cuda")
    assert ds.eval_batch(empty, torch.zeros((0, 7), device="cuda"))[0].numel() == 0
    smse, a, b, mse = ds.eval_batch(dev(op[None]), dev(cv[None]))
    ds.sync()
    assert smse.item() == 0.0 and b.item() == 0.0
    assert abs(a.item() - 2.0) < 1e-6
    f = 0.5 + math.sin(-1.0)
    assert abs(mse.item() - (f - 2.0) ** 2) < 1e-5
    ds.close()


def test_degenerate_trees(gg):
    rng = np.random.default_rng(1)
    N = 3333
    X = rng.uniform(-1, 1, (N, 3)).astype(np.float32)
    X[17, 0] = 0.0
    y = (X[:, 0] * 2 + 1).astype(np.float32)
    trees = [
        (["2.5"], 0),                                  # constant, height 0
        (["x1"], 0),                                   # single feature
        (["*", "3", "-4"], 1),                         # constant tree
        (["logabs", "x0", "x1"], 1),                   # log|0| at row 17 -> +inf
        (["+", "x0", "1"], 1),                         # exact affine fit of y
        (["exp", "*", None, "60", "x1"], 2),           # > 2^50 somewhere -> +inf
        (["aq", "x0", "*", None, None, "1e10", "x1"], 2),  # huge denominator
    ]
    ops, cvs = [], []
    for toks, h in trees:
        o, c = heap_template(toks, h)
        oo = np.full(7, 255, np.uint8)
        cc = np.zeros(7, np.float32)
        # re-embed a height-h template into a height-2 row with its own height
        oo[:o.size], cc[:c.size] = o, c
        ops.append(oo)
        cvs.append(cc)
    hs = np.array([h for _, h in trees], dtype=np.int8)
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(y))
    smse, a, b, mse = (t.cpu().numpy() for t in ds.eval_batch(dev(np.stack(ops)), dev(np.stack(cvs)),
                                                               dev(hs)))
    ds.sync()
    vy = np.var(y.astype(np.float64))
    np.testing.assert_allclose(smse[0], vy, rtol=1e-5)
    assert b[0] == 0.0 and b[2] == 0.0
    rho = np.corrcoef(X[:, 1], y)[0, 1]
    np.testing.assert_allclose(smse[1], vy * (1 - rho ** 2), rtol=1e-4)
    np.testing.assert_allclose(smse[2], vy, rtol=1e-5)
    assert math.isinf(smse[3]) and math.isinf(mse[3]) and a[3] == 0 and b[3] == 0
    assert smse[4] <= 1e-8 * vy and abs(b[4] - 2) < 1e-5 and abs(a[4] + 1) < 1e-5
    assert math.isinf(smse[5])
    for p in (6,):
        t = O.Template(ops[p], cvs[p], int(hs[p]), n_features=3)
        fit = O.fitness(O.eval_tree(t, X), y)
        assert abs(smse[p] - fit["smse"]) <= 1e-4 * fit["smse"] + 1e-8 * vy
    ds.close()


def test_invalid_trial_reports_and_isolates(gg):
    w = PA.build("c1", 1000, 8)
    op = w["op"].copy()
    op[3, 0] = 200  # unknown opcode at the root
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    smse = ds.eval_batch(dev(op), dev(w["cval"]))[0]
    with pytest.raises(gg.GGEvalError) as e:
        ds.sync()
    assert e.value.status == -2
    s = smse.cpu().numpy()
    assert math.isnan(s[3]) and np.isfinite(s[np.arange(8) != 3]).sum() >= 5
    ds.sync()  # status was cleared
    ds.close()


def test_pow_needs_its_flag(gg):
    """An active pow node is an invalid template unless GGEVAL_F_POW selects
    the kernels that implement pow; with the flag it evaluates to the
    oracle's value, the plain and masked forms included."""
    w = PA.build("c1", 2000, 8)
    op, cv = w["op"].copy(), w["cval"].copy()
    rows = {0: "pow", 1: "x0", 2: "+", 5: "x1", 6: "0.75"}  # x0 ^ (x1 + 0.75)
    op[2], cv[2] = heap_template(rows, 3)
    X = np.abs(w["X"]) + 0.25
    ds = gg.Dataset(torch.from_numpy(X), torch.from_numpy(w["y"]))
    smse = ds.eval_batch(dev(op), dev(cv))[0]
    with pytest.raises(gg.GGEvalError) as e:
        ds.sync()
    assert e.value.status == -2
    s0 = smse.cpu().numpy()
    assert math.isnan(s0[2]) and np.all(np.isfinite(s0[np.arange(8) != 2]))
    for call in (ds.eval_batch, ds.eval_plain):
        s1 = call(dev(op), dev(cv), flags=gg.F_POW)[0].cpu().numpy()
        ds.sync()
        np.testing.assert_allclose(s1[np.arange(8) != 2], s0[np.arange(8) != 2], rtol=1e-5)
        fit = O.fitness(O.eval_tree(O.Template(op[2], cv[2], 3, n_features=5), X), w["y"])
        assert abs(s1[2] - fit["smse"]) <= 1e-4 * fit["smse"] + 1e-8 * np.var(w["y"])
    ds.close()


@pytest.mark.parametrize("cfg", ["c2", "c3", "t2", "l_squ"])
def test_constant_folding_is_bit_identical(gg, cfg):
    """Folding constant subtrees (the default) must not change a single bit
    of the outputs: the folded constants are computed with the
    interpreter's own FP32 operator functions."""
    w = PA.build(cfg, 3001, 96)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = dev(w["op"]), dev(w["cval"])
    hs = dev(w["heights"]) if len(set(w["heights"].tolist())) > 1 else None
    pf = gg.F_POW if w.get("uses_pow") else 0
    st = gg.batch_stats(torch.from_numpy(w["op"]), torch.from_numpy(w["cval"]),
                        torch.from_numpy(w["heights"]), n_features=w["F"]).numpy()
    assert st[st[:, 0] >= 0, 13].sum() < st[st[:, 0] >= 0, 0].sum()  # something folds
    for flags in (pf, pf | gg.F_EXACT):
        a = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=flags)]
        b = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=flags | gg.F_NO_FOLD)]
        for x, z in zip(a, b):
            np.testing.assert_array_equal(x, z)
    p1 = [t.cpu().numpy() for t in ds.eval_plain(op, cv, hs, flags=pf)]
    p2 = [t.cpu().numpy() for t in ds.eval_plain(op, cv, hs, flags=pf | gg.F_NO_FOLD)]
    for x, z in zip(p1, p2):
        np.testing.assert_array_equal(x, z)
    ds.sync()
    ds.close()


@pytest.mark.parametrize("cfg", ["t2", "l_squ"])
def test_early_exit_matches_plain_form(gg, cfg):
    """The batched form stops evaluating a trial once a tile of it is
    non-finite (its fitness is +inf); the plain form evaluates every row.
    Both give the same +inf trials and the same finite fitness."""
    w = PA.build(cfg, 40000, 128)
    ds = gg.Dataset(torch.from_numpy(w["X"]), torch.from_numpy(w["y"]))
    op, cv = dev(w["op"]), dev(w["cval"])
    hs = dev(w["heights"]) if len(set(w["heights"].tolist())) > 1 else None
    pf = gg.F_POW if w.get("uses_pow") else 0
    bat = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=pf)]
    pla = [t.cpu().numpy() for t in ds.eval_plain(op, cv, hs, flags=pf)]
    ds.sync()
    ds.close()
    inf_b, inf_p = np.isinf(bat[0]), np.isinf(pla[0])
    np.testing.assert_array_equal(inf_b, inf_p)
    assert 10 <= inf_b.sum() <= 118  # the workload has both kinds
    np.testing.assert_array_equal(bat[1][inf_b], 0.0)
    np.testing.assert_array_equal(bat[2][inf_b], 0.0)
    assert np.all(np.isinf(bat[3][inf_b]))
    for x, z in zip(bat, pla):
        np.testing.assert_allclose(x[~inf_b], z[~inf_b], rtol=2e-5, atol=1e-30)


def test_bad_arguments_rejected(gg):
    X = torch.zeros((10, 2))
    y = torch.arange(10, dtype=torch.float32)
    with pytest.raises(gg.GGEvalError):
        gg.Dataset(X, y * float("nan"))
    ds = gg.Dataset(X, y)
    op = torch.zeros((2, 1023), dtype=torch.uint8, device="cuda")  # height 9
    with pytest.raises(gg.GGEvalError) as e:
        ds.eval_batch(op, torch.zeros((2, 1023), device="cuda"))
    assert e.value.status == -7
    ds.close()


@pytest.mark.parametrize("h,nf", [(8, 1), (8, 40), (0, 3)])
def test_max_height_and_feature_counts(gg, h, nf):
    rng = np.random.default_rng(h * 100 + nf)
    N = 2100
    X = rng.uniform(-1, 1, (N, nf)).astype(np.float32)
    y = (np.cos(X[:, 0]) + 0.1 * rng.standard_normal(N)).astype(np.float32)
    op, cv, hs = synth.random_templates(rng, 24, h, h, synth.BASIC_SET, nf, 0.9)
    w = dict(X=X, y=y, op=op, cval=cv, heights=hs, layout="heap", F=nf, P=24)
    tr, tf, _ = run_case(gg, w)
    # deep single-feature trees are often ill-conditioned in FP32
    assert_tally(tr, min_checked=N * 8, max_excl=0.5 if h == 8 else 0.2)
    assert_tally(tf, min_checked=8, max_excl=0.5)


# -------------------------------------------------------- full-size configs --
#: trials compared with the oracle at each workload's full size (None: all)
FULL = {"c1": None, "c2": None, "c3": 512, "c4": None, "c5": 512, "t2": None}
#: exclusion limits on the benchmark workloads: ill-conditioned trials and rows
MAX_TRIAL_EXCL, MAX_ROW_EXCL = 0.02, 0.05
#: workloads with more ill-conditioned trials: the Table 2 set's unprotected
#: operators (plain division, log, sqrt, pow; 6.6 % of trials), and the
#: gradient workload's ERC-dense trees of cancelling constants, where the
#: worst-case error bound (each function node's rounding, summed over some 30
#: nodes) exceeds half the tolerance on 2.4 % of trials (the FP32 emulation
#: itself stays within it); excluded trials are still held to the loose bound
MAX_TRIAL_EXCL_BY_CFG = {"t2": 0.08, "c4": 0.03}
#: the largest workload's height-6 trees (exp and sin chains, cancelling
#: sums) leave about 11 % of their rows ill-conditioned in FP32 (more than
#: half of them because the FP32 emulation itself is beyond half the
#: tolerance); those rows are still held to the loose bound
MAX_ROW_EXCL_BY_CFG = {"c5": 0.13}


def bench_config_eval(gg, ds, op, cv, hs, flags, P):
    """The launch configuration the benchmark times: autotuned tile shape,
    the call replayed as a CUDA graph on a side stream."""
    ds.autotune(op, cv, hs, flags=flags)
    st = torch.cuda.Stream()
    outs = [torch.full((P,), -7.0, device="cuda") for _ in range(4)]
    for _ in range(2):  # the second call replays the captured graph
        ds.eval_batch(op, cv, hs, flags=flags | gg.F_GRAPH, stream=st, out=outs)
    st.synchronize()
    return [t.cpu().numpy() for t in outs]


@pytest.mark.parametrize("cfg", list(FULL))
def test_full_size_config(gg, cfg):
    """Every configuration at its benchmark size: the fitness of every trial
    (C1, C2, C4, Table 2 set) or of 512 sampled trials (C3, C5) against the
    oracle, in the default launch configuration and in the benchmark's
    (autotuned, graph replay), with at most 2 % of trials excluded as
    ill-conditioned in FP32 (8 % for the Table 2 set, 3 % for the gradient
    workload)."""
    w = PA.build(cfg)
    P = w["P"]
    trials = list(range(P)) if FULL[cfg] is None else sorted(
        np.random.default_rng(7).choice(P, FULL[cfg], replace=False).tolist())
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    hs = dev(w["heights"]) if len(set(w["heights"].tolist())) > 1 else None
    flags = gg.F_POW if w.get("uses_pow") else 0
    default = [t.cpu().numpy() for t in ds.eval_batch(op, cv, hs, flags=flags)]
    tuned = bench_config_eval(gg, ds, op, cv, hs, flags, P)
    cfg_used = ds.tile_config(op, cv, hs, flags=flags)
    ds.sync()
    ds.close()
    for outs in (default, tuned):
        assert np.sum(np.isnan(outs[0])) == 0
    t_def, t_tun = PA.check_fitness(w, trials, [default[0], tuned[0]], [default[3], tuned[3]])
    lim = MAX_TRIAL_EXCL_BY_CFG.get(cfg, MAX_TRIAL_EXCL)
    assert_tally(t_def, min_checked=len(trials) // 2, max_excl=lim,
                 name=f"full-size {w['name']}", what="trials")
    assert_tally(t_tun, min_checked=len(trials) // 2, max_excl=lim,
                 name=f"full-size {w['name']} {tuple(cfg_used)}", what="trials")


@pytest.mark.parametrize("cfg,n_trials", [("c2", 48), ("c5", 24)])
def test_rows_in_benchmark_configuration(gg, cfg, n_trials):
    """Per-row values from the kernel the benchmark times: the configuration
    the autotuner picks for the full batch (8 rows per lane on these
    workloads) is forced on a sample of its trials, at the full row count,
    and eval_rows runs that configuration's kernel in its per-row build.
    Every other fitness variant must give bit-identical rows."""
    w = PA.build(cfg)
    P = w["P"]
    X, y = torch.from_numpy(w["X"]), torch.from_numpy(w["y"])
    ds = gg.Dataset(X, y)
    op, cv = dev(w["op"]), dev(w["cval"])
    ds.autotune(op, cv)
    variant, tile, group, warps = ds.tile_config(op, cv)
    trials = sorted(np.random.default_rng(11).choice(P, n_trials, replace=False).tolist())
    sop, scv = dev(w["op"][trials]), dev(w["cval"][trials])
    ds.tile_config(sop, scv, set=(variant, tile, min(group, n_trials), warps))
    rows = ds.eval_rows(sop, scv)
    ref = rows.cpu().numpy()
    for v in (0, 1, 2, 4, 5, 6, 8, 9):
        if v == variant:
            continue
        r = 32 * (8 if v in (0, 4, 8) else 4)
        ds.tile_config(sop, scv, set=(v, max(r, (tile // r) * r), min(group, n_trials), 8))
        other = ds.eval_rows(sop, scv).cpu().numpy()
        np.testing.assert_array_equal(other.view(np.uint32), ref.view(np.uint32), err_msg=f"variant {v}")
    ds.sync()
    ds.close()
    t = PA.check_rows_many(w, trials, ref)
    assert_tally(t, min_checked=n_trials * w["N"] // 2,
                 max_excl=MAX_ROW_EXCL_BY_CFG.get(cfg, MAX_ROW_EXCL),
                 name=f"rows {w['name']} variant {variant}", what="rows")
