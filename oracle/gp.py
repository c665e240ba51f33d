"""Plain recursive FP64 evaluator, scaled MSE and gradients (the oracle).

Test infrastructure only (see the package docstring).  Every function cites
the passage of the paper it follows; readings of points the paper leaves
open are marked READING.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "ADD", "SUB", "MUL", "AQ", "SIN", "COS", "EXP", "LOG_ABS", "SQRT_ABS", "DIV",
    "SQUARE", "LOG", "SQRT", "POW", "ERC", "FEAT0", "PAD", "BINARY", "UNARY", "BIG",
    "VAR_TOL", "InvalidTemplate", "Template", "active_mask", "rpn", "paper_encoding",
    "eval_tree", "eval_tree_f32", "eval_tree_perturbed", "condition_bound", "pow_ambiguous_rows",
    "fitness", "grad",
    "fd_grad", "eval_batch",
]

# Template opcodes: the library's documented interface values.
ADD, SUB, MUL, AQ = 0, 1, 2, 3
SIN, COS, EXP, LOG_ABS, SQRT_ABS = 4, 5, 6, 7, 8
DIV, SQUARE, LOG, SQRT, POW = 9, 10, 11, 12, 13
ERC = 31
FEAT0 = 32
PAD = 255
BINARY = (ADD, SUB, MUL, AQ, DIV, POW)
UNARY = (SIN, COS, EXP, LOG_ABS, SQRT_ABS, SQUARE, LOG, SQRT)

#: READING: a trial whose output exceeds this magnitude at any row (or is
#: non-finite there) has fitness +inf.  2**50 keeps every FP32 square and
#: product of the fitness sums finite.
BIG = 2.0 ** 50
#: READING: a population variance of f at or below VAR_TOL * mean(f)^2 is
#: treated as zero (a constant tree): b* = 0, a* = mean(y).
VAR_TOL = 1e-12


class InvalidTemplate(ValueError):
    pass


class Template:
    """One trial: a fixed-shape arity-2 template of height ``h``.

    Section 3.1: an individual is a fixed-length string mapped onto a tree
    template; nodes not reached from the root are introns.  ``layout`` is
    "heap" (children 2i+1, 2i+2) or "prefix" (pre-order of the full
    template; children p+1 and p+2**s for a node whose subtree has height s).
    """

    def __init__(self, op, cval, h: int, layout: str = "heap", n_features: int | None = None):
        self.op = np.asarray(op).astype(np.int64)
        self.cval = np.asarray(cval, dtype=np.float32)
        self.h = int(h)
        self.layout = layout
        self.n_features = n_features
        if layout not in ("heap", "prefix"):
            raise ValueError(layout)
        if self.op.size < (1 << (self.h + 1)) - 1:
            raise InvalidTemplate("template row shorter than 2**(h+1)-1")

    def children(self, pos: int, depth: int):
        if self.layout == "heap":
            return 2 * pos + 1, 2 * pos + 2
        return pos + 1, pos + (1 << (self.h - depth))

    def check(self, pos: int, depth: int) -> int:
        """Validate one ACTIVE node and return its opcode.  READING: an intron
        may hold anything; an active node must be a known opcode, a function
        must not sit at a leaf position, a feature index must be < F."""
        o = int(self.op[pos])
        if o in BINARY or o in UNARY:
            if depth >= self.h:
                raise InvalidTemplate(f"function {o} at leaf position {pos}")
            return o
        if o == ERC:
            return o
        if FEAT0 <= o < PAD:
            if self.n_features is not None and o - FEAT0 >= self.n_features:
                raise InvalidTemplate(f"feature {o - FEAT0} >= {self.n_features}")
            return o
        raise InvalidTemplate(f"opcode {o} active at position {pos}")


def active_mask(t: Template) -> np.ndarray:
    """Active nodes (Section 3.1, Fig. 1): the root is active; both children
    of an active binary function are active; only child 0 (the left child)
    of an active unary function is active (READING: Fig. 1 draws sin with
    two children and fixes no operand); a terminal has no active children
    (Fig. 1: the subtrees under the terminals -2 and x1 are introns)."""
    mask = np.zeros(t.op.size, dtype=bool)

    def visit(pos, depth):
        o = t.check(pos, depth)
        mask[pos] = True
        if o in BINARY:
            l, r = t.children(pos, depth)
            visit(l, depth + 1)
            visit(r, depth + 1)
        elif o in UNARY:
            l, _ = t.children(pos, depth)
            visit(l, depth + 1)

    visit(0, 0)
    return mask


def rpn(t: Template) -> list:
    """Post-order traversal of the active nodes, left operand first
    (Section 3.2: RPN, operators after their operands, introns ignored).
    Returns a list of (position, opcode, constant)."""
    out = []

    def visit(pos, depth):
        o = t.check(pos, depth)
        if o in BINARY:
            l, r = t.children(pos, depth)
            visit(l, depth + 1)
            visit(r, depth + 1)
        elif o in UNARY:
            l, _ = t.children(pos, depth)
            visit(l, depth + 1)
        out.append((pos, o, float(t.cval[pos])))

    visit(0, 0)
    return out


#: the paper's operator indices in Fig. 1 (+ = 0, - = 1, x = 2, / = 3, sin = 4)
PAPER_OP_INDEX = {ADD: 0, SUB: 1, MUL: 2, DIV: 3, SIN: 4}


def paper_encoding(t: Template):
    """(T, V) rows of Fig. 1: type 0 = variable, 1 = constant, 2 = operator;
    value = variable index, constant value or operator index."""
    T, V = [], []
    for _, o, c in rpn(t):
        if o >= FEAT0:
            T.append(0)
            V.append(float(o - FEAT0))
        elif o == ERC:
            T.append(1)
            V.append(c)
        else:
            T.append(2)
            V.append(float(PAPER_OP_INDEX[o]))
    return T, V


def _apply(o, a, b=None, xp=np):
    """One function node.  AQ(a, b) = a / sqrt(1 + b^2) (analytic quotient,
    Ni, Drieberg and Rockett 2013); log|x| and sqrt|x| are the protected
    forms of the function set; DIV, SQUARE, LOG, SQRT and POW are the paper's
    Table 2 operators (plain division, square, unprotected log and sqrt,
    power).  READING: pow(a, b) = a^b with the IEEE 754 / C99 pow special
    cases (Table 2 names pow without a definition): a negative base with a
    non-integer exponent gives NaN, 0 to a negative power gives inf, and
    x^0 = 1 for every x.  Binary operands in template order: op(left,
    right), so the left child is the base."""
    if o == ADD:
        return a + b
    if o == SUB:
        return a - b
    if o == MUL:
        return a * b
    if o == AQ:
        one = a.dtype.type(1)
        return a / np.sqrt(one + b * b)
    if o == DIV:
        return a / b
    if o == POW:
        return np.power(a, b)
    if o == SIN:
        return np.sin(a)
    if o == COS:
        return np.cos(a)
    if o == EXP:
        return np.exp(a)
    if o == LOG_ABS:
        return np.log(np.abs(a))
    if o == SQRT_ABS:
        return np.sqrt(np.abs(a))
    if o == SQUARE:
        return a * a
    if o == LOG:
        return np.log(a)
    if o == SQRT:
        return np.sqrt(a)
    raise InvalidTemplate(o)


def _eval(t: Template, X: np.ndarray, dtype, store=None, perturb=None) -> np.ndarray:
    n = X.shape[0]

    def visit(pos, depth):
        o = t.check(pos, depth)
        if o >= FEAT0:
            v = X[:, o - FEAT0].astype(dtype)
        elif o == ERC:
            v = np.full(n, dtype(t.cval[pos]), dtype=dtype)
        elif o in BINARY:
            l, r = t.children(pos, depth)
            v = _apply(o, visit(l, depth + 1), visit(r, depth + 1))
        else:
            l, _ = t.children(pos, depth)
            v = _apply(o, visit(l, depth + 1))
        if perturb is not None and o < ERC:
            rel, rng = perturb
            v = v * (1.0 + rel * rng.choice(np.array([-1.0, 1.0]), n))
        if store is not None:
            store[pos] = v
        return v

    with np.errstate(all="ignore"):
        return visit(0, 0)


def eval_tree(t: Template, X: np.ndarray) -> np.ndarray:
    """f(x_i) for every row i, recursively from the root in FP64
    (Section 3.2: each subexpression is evaluated before its parent)."""
    return _eval(t, np.asarray(X), np.float64)


def eval_tree_f32(t: Template, X: np.ndarray) -> np.ndarray:
    """The same recursion with every node value rounded to float32 and
    float32 library functions.  Used only to flag ill-conditioned rows."""
    return _eval(t, np.asarray(X, dtype=np.float32), np.float32)


def eval_tree_perturbed(t: Template, X: np.ndarray, rel: float, rng) -> np.ndarray:
    """FP64 evaluation with the value of every function node multiplied by
    (1 + rel * s), s = +1 or -1 at random per row: a first-order probe of
    how far rounding errors of relative size ``rel`` at each node can move
    the result.  Tests use it (with rel a few FP32 units in the last place)
    to tell rows and trials whose FP32 value is ill-conditioned, the effect
    Section 5 of the paper notes for redundant subexpressions."""
    return _eval(t, np.asarray(X), np.float64, perturb=(rel, rng))


def condition_bound(t: Template, X: np.ndarray, rel) -> np.ndarray:
    """First-order bound, per row, on how far the tree's value moves when the
    value of every function node carries a relative error of at most
    ``rel`` (a number, or a mapping from opcode to that operator's relative
    error): sum over function nodes n of rel_n * |d f / d v_n| * |v_n|, with
    the sensitivities d f / d v_n from an FP64 reverse sweep and |cos|, |sin|
    replaced by their bound 1 at sin and cos nodes (so a large argument is
    never hidden by a small local slope).  This is the forward error
    analysis of an expression DAG (Higham, "Accuracy and Stability of
    Numerical Algorithms", ch. 3) applied to the tree; tests compare it with
    a quarter of the tolerance to tell rows whose FP32 value is
    ill-conditioned (Section 5 of the paper notes FP32 error growth on such
    expressions).  Non-finite where any node value is non-finite."""
    X = np.asarray(X)
    per_op = isinstance(rel, dict)
    vals = {}
    f = _eval(t, X, np.float64, store=vals)
    n = f.size
    bound = np.zeros(n)

    def back(pos, depth, adj):
        nonlocal bound
        o = int(t.op[pos])
        if o >= ERC:
            return
        bound = bound + (rel[o] if per_op else 1.0) * np.abs(adj * vals[pos])
        l, r = t.children(pos, depth)
        if o in BINARY:
            da, db = _dapply(o, vals[l], vals[r], vals[pos])
            back(l, depth + 1, adj * da)
            back(r, depth + 1, adj * db)
        else:
            if o in (SIN, COS):
                da = np.ones(n)
            else:
                da, _ = _dapply(o, vals[l], None, vals[pos])
            back(l, depth + 1, adj * da)

    with np.errstate(all="ignore"):
        back(0, 0, np.ones(n))
        bound = np.where(np.isfinite(f), bound if per_op else rel * bound, np.inf)
        return np.where(np.isnan(bound), np.inf, bound)


def pow_ambiguous_rows(t: Template, X: np.ndarray, ulps: float = 64.0) -> np.ndarray:
    """Rows whose value FP32 rounding may flip between a number and NaN.

    A negative base raised to a non-integer exponent is NaN, to an integer
    exponent a number, so pow is discontinuous in its exponent at a negative
    base.  READING: a row where an active pow node has a negative base and an
    exponent within `ulps` FP32 units in the last place (of max(1, |b|)) of
    an integer has a value that FP32 evaluation does not determine (rounding
    the exponent decides); tests exclude such rows, and the finiteness of
    their trials, from parity and count them.  Exponents of 2^18 and beyond
    are always within the window (FP32 spacing there is at least 1/64)."""
    X = np.asarray(X)
    vals = {}
    _eval(t, X, np.float64, store=vals)
    amb = np.zeros(X.shape[0], dtype=bool)

    def visit(pos, depth):
        nonlocal amb
        o = int(t.op[pos])
        if o >= ERC:
            return
        l, r = t.children(pos, depth)
        visit(l, depth + 1)
        if o in BINARY:
            visit(r, depth + 1)
        if o == POW:
            a, b = vals[l], vals[r]
            with np.errstate(all="ignore"):
                near = np.abs(b - np.rint(b)) <= ulps * 2.0 ** -24 * np.maximum(1.0, np.abs(b))
            amb = amb | ((a < 0) & near)

    visit(0, 0)
    return amb


def _overflowed(f: np.ndarray) -> bool:
    with np.errstate(all="ignore"):
        return (not np.all(np.isfinite(f))) or bool(np.any(np.abs(f) > BIG))


def fitness(f: np.ndarray, y: np.ndarray) -> dict:
    """MSE (Eq. 1), NMSE (Eq. 2) and linearly scaled MSE of one trial.

    smse = min_{a,b} (1/N) sum_i (y_i - a - b f_i)^2, reached at
    b* = cov(f, y) / var(f), a* = mean(y) - b* mean(f) (ordinary least
    squares of y on f).  Two centred FP64 passes give the means and the
    centred sums; smse is then a third, direct pass over the residuals.
    Variances use 1/N (READING: Eq. 2 does not say; 1/N matches Eq. 1)."""
    f = np.asarray(f, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = f.size
    if n == 0 or _overflowed(f):
        return dict(smse=math.inf, mse=math.inf, a=0.0, b=0.0, nmse=math.inf,
                    var_f=math.nan, finite=False)
    fbar = float(np.sum(f) / n)
    ybar = float(np.sum(y) / n)
    fc = f - fbar
    yc = y - ybar
    var_f = float(np.sum(fc * fc) / n)
    cov = float(np.sum(fc * yc) / n)
    var_y = float(np.sum(yc * yc) / n)
    if var_f <= VAR_TOL * fbar * fbar:
        b = 0.0
    else:
        b = cov / var_f
    a = ybar - b * fbar
    smse = float(np.sum((y - a - b * f) ** 2) / n)
    mse = float(np.sum((f - y) ** 2) / n)
    return dict(smse=smse, mse=mse, a=a, b=b, nmse=mse / var_y if var_y > 0 else math.inf,
                var_f=var_f, finite=True)


def _dapply(o, a, b, out):
    """Local partial derivatives of one function node at its inputs (a, b)
    and its output ``out``.  READING at kinks: d sqrt|x| / dx = 0 at x = 0.
    READING for pow: d a^b / da = b a^(b-1); d a^b / db = a^b ln|a|, which
    for a < 0 (integer b) is the real part of the derivative of the
    principal complex power, and 0 where a^b = 0."""
    one = 1.0
    if o == ADD:
        return np.ones_like(a), np.ones_like(b)
    if o == SUB:
        return np.ones_like(a), -np.ones_like(b)
    if o == MUL:
        return b, a
    if o == AQ:
        q = one / np.sqrt(one + b * b)
        return q, -a * b * q * q * q
    if o == DIV:
        return one / b, -a / (b * b)
    if o == POW:
        return b * np.power(a, b - one), np.where(out == 0, 0.0, out * np.log(np.abs(a)))
    if o == SIN:
        return np.cos(a), None
    if o == COS:
        return -np.sin(a), None
    if o == EXP:
        return out, None
    if o == LOG_ABS or o == LOG:
        return one / a, None
    if o == SQRT_ABS:
        s = np.sqrt(np.abs(a))
        return np.where(a == 0, 0.0, np.sign(a) / (2.0 * np.where(s == 0, 1.0, s))), None
    if o == SQRT:
        return 0.5 / out, None
    if o == SQUARE:
        return 2.0 * a, None
    raise InvalidTemplate(o)


def grad(t: Template, X: np.ndarray, y: np.ndarray, mode: str = "smse", with_abs: bool = False,
         perturb=None):
    """Reverse-mode FP64 gradient of smse (or mse) with respect to the
    constant of every active ERC node; 0 at every other template position.

    For smse, a* and b* are the least-squares optimum, so their own
    partials vanish (envelope theorem) and
        d smse / d c_k = (2 b*/N) sum_i (a* + b* f_i - y_i) d f_i / d c_k.
    For mse: (2/N) sum_i (f_i - y_i) d f_i / d c_k.  READING: the gradient
    is 0 for trials with infinite fitness and (smse) for b* = 0.
    Returns (gradient float64 [stride], fitness dict); with ``with_abs``
    also, per entry, sum_i s_i |d f_i / d c| with s_i = (2/N)|b*|(|a*| +
    |b* f_i| + |y_i|) (smse) or (2/N)(|f_i| + |y_i|) (mse): the size of the
    terms whose rounding in FP32 an FP32 gradient cannot avoid (the residual
    a + b f - y is a difference of such terms).  ``perturb`` = (rel, rng)
    multiplies every function node's value by (1 +- rel) as
    eval_tree_perturbed does (a probe of the gradient's FP32 conditioning;
    a* and b* then belong to the perturbed values)."""
    X = np.asarray(X)
    y = np.asarray(y, dtype=np.float64)
    vals = {}
    f = _eval(t, X, np.float64, store=vals, perturb=perturb)
    fit = fitness(f, y)
    g = np.zeros(t.op.size, dtype=np.float64)
    gabs = np.zeros(t.op.size, dtype=np.float64)
    n = f.size
    out = (lambda: (g, fit, gabs)) if with_abs else (lambda: (g, fit))
    if not fit["finite"]:
        return out()
    if mode == "smse":
        if fit["b"] == 0.0:
            return out()
        seed = (2.0 / n) * fit["b"] * (fit["a"] + fit["b"] * f - y)
        scale = (2.0 / n) * abs(fit["b"]) * (abs(fit["a"]) + np.abs(fit["b"] * f) + np.abs(y))
    elif mode == "mse":
        seed = (2.0 / n) * (f - y)
        scale = (2.0 / n) * (np.abs(f) + np.abs(y))
    else:
        raise ValueError(mode)

    def back(pos, depth, adj, aabs):
        o = int(t.op[pos])
        if o == ERC:
            g[pos] += float(np.sum(adj))
            gabs[pos] += float(np.sum(aabs))
            return
        if o >= FEAT0:
            return
        l, r = t.children(pos, depth)
        if o in BINARY:
            da, db = _dapply(o, vals[l], vals[r], vals[pos])
            back(l, depth + 1, adj * da, aabs * np.abs(da))
            back(r, depth + 1, adj * db, aabs * np.abs(db))
        else:
            da, _ = _dapply(o, vals[l], None, vals[pos])
            back(l, depth + 1, adj * da, aabs * np.abs(da))

    with np.errstate(all="ignore"):
        back(0, 0, seed, scale)
    return out()


def fd_grad(t: Template, X: np.ndarray, y: np.ndarray, mode: str = "smse",
            rel_step: float = 1e-6) -> np.ndarray:
    """Central finite differences of smse (or mse) in every active ERC
    constant, step h = rel_step * max(1, |c|), constants held in FP64."""
    mask = active_mask(t)
    g = np.zeros(t.op.size, dtype=np.float64)
    X = np.asarray(X)

    def value(pos, c):
        tt = Template(t.op, t.cval, t.h, t.layout, t.n_features)
        # evaluate with an FP64 constant at ``pos`` (not rounded to float32)
        vals = {}
        saved = tt.cval
        tt.cval = saved.astype(np.float64)
        tt.cval[pos] = c
        f = _eval(tt, X, np.float64, store=vals)
        return fitness(f, y)[mode]

    for pos in np.nonzero(mask & (t.op == ERC))[0]:
        c = float(t.cval[pos])
        h = rel_step * max(1.0, abs(c))
        g[pos] = (value(pos, c + h) - value(pos, c - h)) / (2.0 * h)
    return g


def eval_batch(op, cval, heights, h_max, X, y, layout="heap", n_features=None):
    """Fitness of every trial of a batch: arrays smse, a, b, mse (float64)."""
    op = np.asarray(op)
    P = op.shape[0]
    out = {k: np.zeros(P) for k in ("smse", "a", "b", "mse")}
    for p in range(P):
        h = int(heights[p]) if heights is not None else int(h_max)
        t = Template(op[p], cval[p], h, layout, n_features)
        fit = fitness(eval_tree(t, X), y)
        for k in out:
            out[k][p] = fit[k]
    return out
