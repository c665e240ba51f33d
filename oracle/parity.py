"""Parity checks: build a seeded workload with its target from the oracle,
and compare library outputs with the oracle under the stated tolerances.

Test infrastructure, like the rest of this package: the GPU tests and the
benchmark's oracle leg use it; the library never does.

Tolerances (from the accuracy targets of this evaluator):
  per row   |g - r| <= 1e-5 (|r| + rms(r))      rms over the trial's rows
  smse      |g - r| <= 1e-4 r + 1e-8 Var(y)
  mse       |g - r| <= 1e-4 r + 1e-8 (mean y^2 + mean f^2)
  gradient  |g - r| <= 1e-3 (|r| + 1e-3 max_k |r_k|) + 1e-6 G_k, G_k the
            oracle's scale of the FP32 row terms (oracle.grad with_abs)
A row is ill-conditioned in FP32, and excluded, when its FP32-emulated
oracle value or the first-order bound on the effect of relative errors of
4 FP32 units in the last place at every function node
(oracle.condition_bound) exceeds half of its tolerance, or when FP32
rounding may turn it NaN (oracle.pow_ambiguous_rows: a negative base to an
exponent next to an integer; its trial is excluded too).  A trial is
excluded when the same bound, carried to its smse (or mse), exceeds half
of that tolerance, or when its FP64 and FP32-emulated fitness
disagree on being infinite (ambiguous).  Both counts are reported.
"""
import math

import numpy as np

import synth

from . import gp as O

ROW_TOL = 1e-5
SMSE_RTOL, SMSE_FLOOR = 1e-4, 1e-8
GRAD_TOL = 1e-3
COND_MARGIN = 0.5


def target_from_oracle(w):
    """First candidate generator tree with finite values, nonzero variance
    and |f| <= 1e6 (the oracle evaluates it), plus the workload's noise."""
    for gop, gcv, gh in w["y_cands"]():
        f = O.eval_tree(O.Template(gop, gcv, gh, "heap", w["F"]), w["X"])
        with np.errstate(all="ignore"):
            if np.all(np.isfinite(f)) and np.var(f) > 0 and np.max(np.abs(f)) <= 1e6:
                return synth.make_target(f, w["z"], w["noise"]), (gop, gcv, gh)
    raise RuntimeError("no usable generator tree")


def build(cfg, n_rows=None, n_trials=None, rep=0, layout="heap"):
    w = synth.workload(cfg, rep, n_rows, n_trials, layout)
    if "y" not in w:
        w["y"], w["gen"] = target_from_oracle(w)
    return w


def template(w, p):
    h = int(w["heights"][p])
    return O.Template(w["op"][p], w["cval"][p], h, w["layout"], w["F"])


#: An excluded (ill-conditioned) row or trial is still compared with the
#: oracle, against LOOSE times its first-order error bound (or the FP32
#: emulation's distance from FP64, if larger) plus the tolerance, so that a
#: gross error cannot hide among the excluded values.
LOOSE = 16.0


class Tally:
    def __init__(self):
        self.checked = self.excluded = self.failed = 0
        self.loose = 0  # excluded values compared against the loose bound
        self.strict = 0  # excluded values within the strict tolerance all the same
        self.worst = 0.0
        self.msgs = []

    def __repr__(self):
        return (f"checked={self.checked} excluded={self.excluded} failed={self.failed} "
                f"worst={self.worst:.3g} {self.msgs[:5]}")

    def merge(self, other):
        self.checked += other.checked
        self.excluded += other.excluded
        self.failed += other.failed
        self.loose += other.loose
        self.strict += other.strict
        self.worst = max(self.worst, other.worst)
        self.msgs.extend(other.msgs)
        return self

    def excluded_frac(self):
        n = self.checked + self.excluded
        return self.excluded / n if n else 0.0

    def as_dict(self):
        return {"checked": self.checked, "excluded": self.excluded, "failed": self.failed,
                "excluded_but_within_loose_bound": self.loose,
                "excluded_but_within_tolerance": self.strict,
                "worst_err_over_tol": self.worst}


def value_class(v):
    """0 finite, 1 NaN, 2 +inf, 3 -inf."""
    v = np.asarray(v, dtype=np.float64)
    return np.where(np.isnan(v), 1, np.where(v == np.inf, 2, np.where(v == -np.inf, 3, 0)))


def check_rows(g, f64, f32, tally, tag="", cond=None):
    """Per-row values of one trial.  ``cond``: per-row error bound
    (oracle.condition_bound) used with f32 to flag ill-conditioned rows.
    A row that is non-finite in the oracle's FP64 and FP32 passes alike
    (both NaN, or the same infinity) must be that on the GPU too; a row on
    which the two passes disagree is excluded."""
    with np.errstate(all="ignore"):
        fin = np.isfinite(f64)
        rms = math.sqrt(np.mean(f64[fin] ** 2)) if fin.any() else 0.0
        tol = ROW_TOL * (np.abs(f64) + rms)
        err32 = np.abs(f32.astype(np.float64) - f64)
        c64, c32, cg = value_class(f64), value_class(f32), value_class(g)
        amb = np.isnan(cond) if cond is not None else np.zeros(f64.shape, dtype=bool)
        special = (c64 != 0) & (c64 == c32) & ~amb
        ill = ~special & (~fin | (c32 != 0) | (err32 > COND_MARGIN * tol))
        if cond is not None:
            ill |= amb | (fin & ~(cond <= COND_MARGIN * tol))
        err = np.where(special, 0.0, np.abs(g.astype(np.float64) - f64))
        bad = ~ill & np.where(special, cg != c64, ~(err <= tol))
        # excluded rows with a finite bound: the loose comparison
        bound = np.maximum(np.where(np.isnan(cond), np.inf, cond) if cond is not None
                           else 0.0, err32)
        loose = ill & fin & (c32 == 0) & np.isfinite(bound)
        loose_bad = loose & ~(err <= LOOSE * bound + tol)
    tally.checked += int((~ill).sum())
    tally.excluded += int(ill.sum())
    tally.loose += int((loose & ~loose_bad).sum())
    tally.strict += int((ill & fin & (err <= tol)).sum())
    if loose_bad.any():
        tally.failed += int(loose_bad.sum())
        i = int(np.argmax(np.where(loose_bad, err / np.maximum(bound, 1e-300), 0)))
        tally.msgs.append(f"{tag} row {i} (ill-conditioned, bound {bound[i]:.3g}): "
                          f"gpu {g[i]!r} oracle {f64[i]!r}")
    if bad.any():
        tally.failed += int(bad.sum())
        where = np.flatnonzero(bad)
        i = int(where[np.argmax(err[where] / np.maximum(tol[where], 1e-300))])
        tally.msgs.append(f"{tag} row {i}: gpu {g[i]!r} oracle {f64[i]!r} "
                          f"({int(bad.sum())} rows)")
    ok = ~ill
    if ok.any():
        tally.worst = max(tally.worst, float(np.max(err[ok] / np.maximum(tol[ok], 1e-300))))


def fit_bounds(f64, y, fit64, cond):
    """Bounds on the change of smse and mse when every row value moves by at
    most cond_i: (1/N) sum (2 |r_i| e_i + e_i^2) with r_i the residual of
    the scaled (b e_i) or plain fit."""
    y = np.asarray(y, dtype=np.float64)
    with np.errstate(all="ignore"):
        r = y - fit64["a"] - fit64["b"] * f64
        e = np.abs(fit64["b"]) * cond
        ds = float(np.mean(2 * np.abs(r) * e + e * e))
        rm = f64 - y
        dm = float(np.mean(2 * np.abs(rm) * cond + cond * cond))
    return ds, dm


def check_fit(g_smse, g_mse, fit64, fit32, var_y, mean_y2, tally, tag="", bounds=None):
    """smse (and mse) of one trial.  ``bounds``: (smse, mse) change bounds
    from fit_bounds, used with fit32 to flag ill-conditioned trials."""
    inf64 = not fit64["finite"]
    inf32 = not fit32["finite"]
    if bounds is not None and np.isnan(bounds[0]):  # a row FP32 rounding may turn NaN
        tally.excluded += 1
        return
    if inf64 != inf32 or (bounds is not None and not inf64 and not np.isfinite(bounds[0])):
        tally.excluded += 1
        return
    if inf64:
        tally.checked += 1
        if not (math.isinf(g_smse) and g_smse > 0):
            tally.failed += 1
            tally.msgs.append(f"{tag}: oracle +inf, gpu {g_smse}")
        return
    r = fit64["smse"]
    tol = SMSE_RTOL * r + SMSE_FLOOR * var_y
    if (abs(fit32["smse"] - r) > COND_MARGIN * tol or (fit64["b"] == 0.0) != (fit32["b"] == 0.0)
            or (bounds is not None and not bounds[0] <= COND_MARGIN * tol)):
        tally.excluded += 1
        # the loose comparison, when the bound is finite and both are finite
        bound = max(abs(fit32["smse"] - r), bounds[0] if bounds is not None else 0.0)
        if fit32["finite"] and math.isfinite(bound) and (fit64["b"] == 0.0) == (fit32["b"] == 0.0):
            if abs(g_smse - r) <= LOOSE * bound + tol:
                tally.loose += 1
                tally.strict += int(abs(g_smse - r) <= tol)
            else:
                tally.failed += 1
                tally.msgs.append(f"{tag}: smse (ill-conditioned, bound {bound:.3g}) gpu "
                                  f"{g_smse!r} oracle {r!r}")
        return
    tally.checked += 1
    err = abs(g_smse - r)
    # a zero tolerance (one row, or a constant target) asks for the exact value
    tally.worst = max(tally.worst, err / tol if tol > 0 else (0.0 if err == 0 else math.inf))
    if not err <= tol:
        tally.failed += 1
        tally.msgs.append(f"{tag}: smse gpu {g_smse!r} oracle {r!r} tol {tol:.3g}")
    if g_mse is not None:
        rm = fit64["mse"]
        tm = SMSE_RTOL * rm + SMSE_FLOOR * mean_y2
        well = abs(fit32["mse"] - rm) <= COND_MARGIN * tm and (
            bounds is None or bounds[1] <= COND_MARGIN * tm)
        if well and not abs(g_mse - rm) <= tm:
            tally.failed += 1
            tally.msgs.append(f"{tag}: mse gpu {g_mse!r} oracle {rm!r}")


#: relative error assumed at every function node: 4 FP32 units of roundoff
#: (the gradient's perturbation probes)
COND_REL = 4 * 2.0 ** -24
_U = 2.0 ** -24
#: relative error of each operator's FP32 evaluation (reading 12), in units
#: of roundoff u = 2^-24: +, -, x, / and x^2 are correctly rounded (u); the
#: interpreter's sqrt, log, sin / cos and exp are within 1, 1.5, 2 and 3 FP32
#: units in the last place of their FP64 values (2u, 3u, 4u, 6u; the GPU
#: math tests hold them to those bounds); AQ = a rsqrt(1 + b^2) with the
#: approximate reciprocal square root, 6u; pow, the library function, 8u
COND_REL_BY_OP = {O.ADD: _U, O.SUB: _U, O.MUL: _U, O.DIV: _U, O.SQUARE: _U,
                  O.SQRT: 2 * _U, O.SQRT_ABS: 2 * _U, O.LOG: 3 * _U, O.LOG_ABS: 3 * _U,
                  O.SIN: 4 * _U, O.COS: 4 * _U, O.EXP: 6 * _U, O.AQ: 6 * _U,
                  O.POW: 8 * _U}


def oracle_trial(w, p, X=None, y=None):
    """Oracle data of trial p: template, FP64 rows, FP32-emulated rows,
    their fitness, the per-row condition bound and the fitness bounds."""
    X = w["X"] if X is None else X
    y = w["y"] if y is None else y
    t = template(w, p)
    f64 = O.eval_tree(t, X)
    f32 = O.eval_tree_f32(t, X)
    fit64 = O.fitness(f64, y)
    cond = O.condition_bound(t, X, COND_REL_BY_OP)
    bounds = fit_bounds(f64, y, fit64, cond) if fit64["finite"] else None
    if np.any(t.op[O.active_mask(t)] == O.POW):
        amb = O.pow_ambiguous_rows(t, X)
        if amb.any():  # NaN marks rows (and the trial) whose finiteness FP32 decides
            cond = np.where(amb, np.nan, cond)
            bounds = (math.nan, math.nan)
    return t, f64, f32, fit64, O.fitness(f32.astype(np.float64), y), cond, bounds


def intermediates_finite_f32(t, X):
    """True if every active node of the FP32-emulated evaluation is finite."""
    store = {}
    O._eval(t, np.asarray(X, dtype=np.float32), np.float32, store=store)
    with np.errstate(all="ignore"):
        return all(np.all(np.isfinite(v)) for v in store.values())


#: FP32 floor of the gradient test, relative to the size of the terms the
#: FP32 residual a + b f - y is made of: a gradient that is 0 (or small) by
#: an invariance is a cancelling FP32 sum of such terms
GRAD_FLOOR = 1e-6


def floor_only_entries(g, r, rabs):
    """Gradient entries inside the tolerance only because of its FP32 floor
    term GRAD_FLOOR * G_k (outside 1e-3 (|r| + 1e-3 max|r|))."""
    scale = 1e-3 * float(np.max(np.abs(r))) if r.size else 0.0
    base = GRAD_TOL * (np.abs(r) + scale)
    err = np.abs(np.asarray(g, dtype=np.float64) - r)
    return int(np.sum((err > base) & (err <= base + GRAD_FLOOR * rabs)))


def grad_tolerance(r, rabs=None):
    scale = 1e-3 * float(np.max(np.abs(r))) if r.size else 0.0
    tol = GRAD_TOL * (np.abs(r) + scale)
    if rabs is not None:
        tol = tol + GRAD_FLOOR * rabs
    return tol


#: perturbed reverse sweeps that probe a gradient's FP32 conditioning
GRAD_PROBES = 3


def grad_ill_conditioned(t, X, y, mode, r, tol, seed):
    """Gradient entries whose FP32 value is ill-conditioned: the FP64
    gradient with every function node's value moved by +-4 FP32 units in the
    last place (random signs per row, GRAD_PROBES draws, oracle.grad's
    perturb) moves by more than a quarter of the entry's tolerance.
    Section 5 of the paper: FP32 and FP64 results differ where expressions
    amplify rounding errors; for a gradient, a cancelling sum of residuals
    does (a weak fit, b* near 0)."""
    rng = np.random.default_rng(seed)
    spread = np.zeros_like(r)
    for _ in range(GRAD_PROBES):
        rp, _ = O.grad(t, X, y, mode, perturb=(COND_REL, rng))
        with np.errstate(invalid="ignore"):
            spread = np.maximum(spread, np.where(np.isfinite(rp), np.abs(rp - r), np.inf))
    return spread > 0.25 * tol


def check_grad(g, r, tally, tag="", rabs=None, skip=None):
    """Gradient entries of one trial; entries marked in ``skip`` (the
    ill-conditioned ones) are left out of the comparison."""
    tol = grad_tolerance(r, rabs)
    if skip is not None:
        r = np.where(skip, 0.0, r)
        g = np.where(skip, 0.0, g)
    err = np.abs(g.astype(np.float64) - r)
    tally.checked += 1
    with np.errstate(all="ignore"):
        ratio = np.where(tol > 0, err / np.maximum(tol, 1e-300), np.where(err > 0, np.inf, 0.0))
    tally.worst = max(tally.worst, float(np.max(ratio)) if ratio.size else 0.0)
    if not np.all(err <= tol):
        tally.failed += 1
        k = int(np.argmax(ratio))
        tally.msgs.append(f"{tag} pos {k}: gpu {g[k]!r} oracle {r[k]!r}")


# --------------------------------------------- checks over a process pool --
# The oracle is slow on purpose; checking thousands of trials at the full row
# count runs it on every host core.  The pool is started with "spawn" so
# that it is safe after CUDA work in the calling process.

#: arrays a worker needs (the workload's generator closure is not sent)
_SHIP = ("X", "y", "op", "cval", "heights", "layout", "F")
_W = None


def _init_worker(w):
    global _W
    _W = w


def _fit_task(items):
    w = _W
    y = w["y"].astype(np.float64)
    var_y, mean_y2 = float(np.var(y)), float(np.mean(y * y))
    tallies = None
    for p, results in items:
        _, _, _, fit64, fit32, _, bounds = oracle_trial(w, p)
        if tallies is None:
            tallies = [Tally() for _ in results]
        for t, (g_smse, g_mse) in zip(tallies, results):
            check_fit(g_smse, g_mse, fit64, fit32, var_y, mean_y2, t, tag=f"trial {p}",
                      bounds=bounds)
    return tallies or []


def _rows_task(items):
    w = _W
    t = Tally()
    for p, g in items:
        _, f64, f32, _, _, cond, _ = oracle_trial(w, p)
        check_rows(g, f64, f32, t, tag=f"trial {p}", cond=cond)
    return t


def _grad_task(items):
    """Worker: the gradient of each (trial, mode, GPU gradient row, GPU smse)
    against the oracle's reverse mode.  A trial whose fitness is excluded as
    ill-conditioned, whose FP32 evaluation overflows at an intermediate node,
    or whose FP64 gradient is not finite is excluded; one with infinite
    fitness (or b* = 0 for smse) must have a zero gradient."""
    w = _W
    y = w["y"].astype(np.float64)
    var_y, mean_y2 = float(np.var(y)), float(np.mean(y * y))
    t, tf, n_floor, n_ill = Tally(), Tally(), 0, 0
    for p, mode, g, g_smse in items:
        tt, f64, f32, fit64, fit32, cond, bounds = oracle_trial(w, p)
        before = tf.excluded
        check_fit(g_smse, None, fit64, fit32, var_y, mean_y2, tf, tag=f"trial {p}",
                  bounds=bounds)
        if tf.excluded != before or not intermediates_finite_f32(tt, w["X"]):
            t.excluded += 1
            continue
        r, fit, rabs = O.grad(tt, w["X"], w["y"], mode, with_abs=True)
        if not fit64["finite"] or (mode == "smse" and fit64["b"] == 0.0):
            t.checked += 1
            if not np.all(g == 0.0):
                t.failed += 1
                t.msgs.append(f"trial {p}: gradient should be 0")
            continue
        if not np.all(np.isfinite(r)):  # a derivative is infinite at some row
            t.excluded += 1
            continue
        ill = grad_ill_conditioned(tt, w["X"], w["y"], mode, r, grad_tolerance(r, rabs), p)
        n_ill += int(ill.sum())
        n_floor += floor_only_entries(np.where(ill, r, g), r, rabs)
        check_grad(g, r, t, tag=f"trial {p}", rabs=rabs, skip=ill)
    return t, tf, n_floor, n_ill


def _pool_map(w, fn, items, processes, chunk):
    """fn over chunks of items on a spawn-started process pool.  A worker
    that dies raises BrokenProcessPool here instead of leaving the pool
    waiting for it."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    tasks = [items[i:i + chunk] for i in range(0, len(items), chunk)]
    if not tasks:
        return []
    n = min(processes or os.cpu_count() or 1, len(tasks))
    ship = {k: w[k] for k in _SHIP}
    if n <= 1:
        _init_worker(ship)
        return [fn(tk) for tk in tasks]
    with cf.ProcessPoolExecutor(n, mp_context=mp.get_context("spawn"),
                                initializer=_init_worker, initargs=(ship,)) as ex:
        return list(ex.map(fn, tasks))


def check_fitness(w, trials, smse, mse=None, processes=None, chunk=2):
    """Check GPU smse (and mse) of the listed trials against the oracle at the
    workload's full row count, on a spawn-started process pool.  ``smse``
    (and ``mse``) may be one array or a list of arrays (several GPU runs
    checked against one oracle pass); returns a Tally, or a list of them."""
    many = isinstance(smse, (list, tuple))
    smses = list(smse) if many else [smse]
    mses = list(mse) if many and mse is not None else [mse] * len(smses)
    items = [(int(p), [(float(s[p]), None if m is None else float(m[p]))
                       for s, m in zip(smses, mses)]) for p in trials]
    out = [Tally() for _ in smses]
    for ts in _pool_map(w, _fit_task, items, processes, chunk):
        for o, t in zip(out, ts):
            o.merge(t)
    return out if many else out[0]


def check_rows_many(w, trials, rows, processes=None, chunk=1):
    """Per-row values of the listed trials (``rows[i]`` belongs to
    ``trials[i]``) against the oracle, on the process pool."""
    items = [(int(p), np.asarray(r)) for p, r in zip(trials, rows)]
    out = Tally()
    for t in _pool_map(w, _rows_task, items, processes, chunk):
        out.merge(t)
    return out


def check_gradients(w, trials, dcval, smse, mode="smse", processes=None, chunk=1):
    """Check GPU gradients (rows of dcval) of the listed trials against the
    oracle's reverse mode on the process pool; returns (gradient Tally,
    fitness Tally, gradient entries that pass only through the FP32 floor
    term GRAD_FLOOR * G_k of the tolerance, entries left out as
    ill-conditioned in FP32)."""
    items = [(int(p), mode, np.asarray(dcval[p], dtype=np.float64), float(smse[p]))
             for p in trials]
    out, fout, floor, ill = Tally(), Tally(), 0, 0
    for t, tf, nf, ni in _pool_map(w, _grad_task, items, processes, chunk):
        out.merge(t)
        fout.merge(tf)
        floor += nf
        ill += ni
    return out, fout, floor, ill
