"""Seeded synthetic workloads for batched GP-GOMEA trial evaluation.

This module is the one place that both the CUDA path (through ``bench.py``
and the GPU tests) and the FP64 oracle take their inputs from.  It draws
random numbers and lays them out; it holds none of the method's arithmetic:
it never evaluates a tree and never computes a fitness.  The target ``y`` of
every workload comes from evaluating a seeded generator tree, and that
evaluation is done by the consumer of the workload (the oracle, in the
tests and in the benchmark's oracle leg), then passed to
:func:`make_target`.

Template format (the library's input format, Section 3.1 of the paper: a
fixed-shape template tree whose inactive nodes are introns):

* a trial of height ``h`` has ``2**(h+1) - 1`` nodes, arity 2;
* ``heap`` layout: node ``i`` has children ``2i+1`` and ``2i+2``;
* ``prefix`` layout: pre-order of the full template, so a node at position
  ``p`` whose subtree has height ``s`` has children ``p+1`` and ``p+2**s``;
* one row per trial with stride ``2**(h_max+1) - 1``; positions beyond the
  trial's own node count hold ``PAD``.

Opcodes are the library's documented interface values (written out here by
hand, as they are in the C header and in the oracle):
"""
from __future__ import annotations

import numpy as np

# ---- template opcodes (interface values) ---------------------------------
ADD, SUB, MUL, AQ = 0, 1, 2, 3
SIN, COS, EXP, LOG_ABS, SQRT_ABS = 4, 5, 6, 7, 8
DIV, SQUARE, LOG, SQRT, POW = 9, 10, 11, 12, 13
ERC = 31
FEAT0 = 32
PAD = 255

BINARY = (ADD, SUB, MUL, AQ, DIV, POW)
UNARY = (SIN, COS, EXP, LOG_ABS, SQRT_ABS, SQUARE, LOG, SQRT)

#: function set of the small plain-evaluation workload
BASIC_SET = (ADD, SUB, MUL, AQ)
#: the full function set {+, -, *, AQ, sin, cos, exp, log|x|, sqrt|x|}
FULL_SET = (ADD, SUB, MUL, AQ, SIN, COS, EXP, LOG_ABS, SQRT_ABS)
#: the paper's Table 2 operator set for Experiments I/II
PAPER_SET = (ADD, SUB, MUL, DIV, SIN, COS, SQUARE, SQRT, EXP, LOG, POW)
#: the paper's Table 2 operator set for Experiment III
EXP3_SET = (ADD, SUB, MUL, DIV, SQUARE, SQRT)


def _ladder_targets():
    """Ground-truth expressions of the Experiment III datasets (Table 1), as
    functions of X [N, 9]: the workload's target function, not a tree."""
    def s(x, *k):
        return sum(x[:, i] for i in k)
    return {
        "addition": lambda x: s(x, *range(9)),
        "division": lambda x: s(x, 0, 1, 2) / s(x, 3, 4, 5, 6, 7, 8),
        "subtraction": lambda x: s(x, 0, 1, 2) / (x[:, 4] - x[:, 3] + x[:, 6] - x[:, 5]
                                                 + x[:, 8] - x[:, 7]),
        "multiplication": lambda x: x[:, 0] * x[:, 1] * x[:, 2] / (
            x[:, 4] - x[:, 3] + x[:, 6] - x[:, 5] + x[:, 8] - x[:, 7]),
        "squaring": lambda x: x[:, 0] * x[:, 1] * x[:, 2] / (
            (x[:, 4] - x[:, 3]) ** 2 + (x[:, 6] - x[:, 5]) ** 2 + (x[:, 8] - x[:, 7]) ** 2),
    }


LADDER = _ladder_targets()


def n_nodes(h: int) -> int:
    return (1 << (h + 1)) - 1


def heap_depth(n: int) -> np.ndarray:
    """Depth of every heap position 0..n-1 (root depth 0)."""
    i = np.arange(n, dtype=np.int64)
    return np.floor(np.log2(i + 1) + 1e-9).astype(np.int64)


def heap_to_prefix_perm(h: int) -> np.ndarray:
    """perm[k] = heap index of the node at prefix position k (height h)."""
    out = []
    stack = [0]
    n = n_nodes(h)
    while stack:
        i = stack.pop()
        if i >= n:
            continue
        out.append(i)
        stack.append(2 * i + 2)
        stack.append(2 * i + 1)
    return np.asarray(out, dtype=np.int64)


def to_prefix(op: np.ndarray, cval: np.ndarray, heights: np.ndarray) -> tuple:
    """Re-order heap-layout template rows into prefix layout (pure permutation)."""
    op2 = np.full_like(op, PAD)
    cv2 = np.zeros_like(cval)
    for h in np.unique(heights):
        rows = np.nonzero(heights == h)[0]
        perm = heap_to_prefix_perm(int(h))
        op2[np.ix_(rows, np.arange(perm.size))] = op[np.ix_(rows, perm)]
        cv2[np.ix_(rows, np.arange(perm.size))] = cval[np.ix_(rows, perm)]
    return op2, cv2


def random_templates(rng: np.random.Generator, n: int, heights, h_max: int,
                     funcs=FULL_SET, n_features: int = 1, p_func=0.5,
                     p_feature: float = 0.5, erc_range=(-5.0, 5.0),
                     erc_leaves: bool = False):
    """Draw ``n`` random heap-layout templates (introns included).

    Every node of the template gets a value, as in GP-GOMEA's fixed-length
    strings: the root is a function; every other non-leaf position is a
    function with probability ``p_func`` (per trial, scalar or array), else a
    terminal; leaf positions are terminals.  A terminal is a feature with
    probability ``p_feature`` (uniform index) else an ERC ~ U[erc_range].
    With ``erc_leaves`` every leaf position holds an ERC and every non-leaf
    terminal is a feature.  Positions beyond a trial's own height are PAD.
    Returns (op uint8 [n, stride], cval float32 [n, stride], heights int8 [n]).
    """
    stride = n_nodes(h_max)
    heights = np.broadcast_to(np.asarray(heights, dtype=np.int64), (n,)).copy()
    p_func = np.broadcast_to(np.asarray(p_func, dtype=np.float64), (n,))
    depth = heap_depth(stride)[None, :]
    used = np.arange(stride)[None, :] < ((1 << (heights + 1)) - 1)[:, None]
    leaf = depth == heights[:, None]
    u_func = rng.random((n, stride))
    is_func = (~leaf) & ((np.arange(stride)[None, :] == 0) | (u_func < p_func[:, None]))
    fsel = np.asarray(funcs, dtype=np.int64)[rng.integers(0, len(funcs), (n, stride))]
    is_feat = rng.random((n, stride)) < p_feature
    feat = FEAT0 + rng.integers(0, n_features, (n, stride))
    erc = rng.uniform(erc_range[0], erc_range[1], (n, stride)).astype(np.float32)
    if erc_leaves:
        is_feat = ~leaf
    op = np.where(is_func, fsel, np.where(is_feat, feat, ERC))
    op = np.where(used, op, PAD).astype(np.uint8)
    cval = np.where(used & ~is_func & ~is_feat, erc, np.float32(0)).astype(np.float32)
    return op, cval, heights.astype(np.int8)


def fos_subset_mask(stride: int, node: np.ndarray) -> np.ndarray:
    """Mask of the FOS subset {node, its two children} for each trial (heap)."""
    idx = np.arange(stride)[None, :]
    node = np.asarray(node)[:, None]
    return (idx == node) | (idx == 2 * node + 1) | (idx == 2 * node + 2)


def fos_step_trials(rng: np.random.Generator, pop_op, pop_cval, step: int,
                    order: np.ndarray):
    """Trials of one GOM step over the FOS (Algorithm 1): every offspring j is
    a clone of individual j whose subset FOS[order[j, step]] is copied from a
    randomly drawn donor.  The FOS holds one subset per template node: the
    node and its children (a node-proximity style FOS; the paper does not
    define its FOS further).  Heap layout only."""
    n, stride = pop_op.shape
    donors = rng.integers(0, n, n)
    node = order[:, step]
    mask = fos_subset_mask(stride, node)
    op = np.where(mask, pop_op[donors], pop_op).astype(np.uint8)
    cv = np.where(mask, pop_cval[donors], pop_cval).astype(np.float32)
    return op, cv


def _x(rng, n, f, dist):
    kind = dist[0]
    if kind == "uniform":
        return rng.uniform(dist[1], dist[2], (n, f)).astype(np.float32)
    if kind == "normal":
        return rng.standard_normal((n, f)).astype(np.float32)
    raise ValueError(dist)


#: The five workloads.  Sizes follow the benchmark configurations; half the
#: trials are "full" trees (every non-leaf position a function) and half
#: "grow" trees (a function with probability 1/2), unless stated.
CONFIGS = {
    "c1": dict(index=0, name="plain-256xh3-1000x5", P=256, h=3, funcs=BASIC_SET,
               N=1_000, F=5, x=("uniform", -1.0, 1.0), y_h=3, y_funcs=BASIC_SET,
               noise=0.0, fos=False),
    "c2": dict(index=1, name="fos-step-4096xh4-100000x8", P=4_096, h=4, funcs=FULL_SET,
               N=100_000, F=8, x=("uniform", -3.0, 3.0), y_h=4, y_funcs=FULL_SET,
               noise=0.01, fos=True),
    "c3": dict(index=2, name="uneven-8192xh3to7-200000x10", P=8_192, h=7, h_min=3,
               funcs=FULL_SET, N=200_000, F=10, x=("uniform", -2.0, 2.0), y_h=5,
               y_funcs=FULL_SET, noise=0.0, fos=False, p_func_range=(0.2, 1.0)),
    "c4": dict(index=3, name="diff-1024xh5-50000x6", P=1_024, h=5, funcs=BASIC_SET,
               N=50_000, F=6, x=("normal",), y_h=5, y_funcs=FULL_SET, noise=0.0,
               fos=False, erc_leaves=True, p_func=0.9),
    "c5": dict(index=4, name="large-16384xh6-1000000x10", P=16_384, h=6, funcs=FULL_SET,
               N=1_000_000, F=10, x=("uniform", -1.0, 1.0), y_h=6, y_funcs=FULL_SET,
               noise=0.01, fos=True),
}
# The FOS-step shape over the paper's Experiments I/II operator set
# (Table 2, with pow); positive features so that log, sqrt and pow of a
# feature are defined
CONFIGS["t2"] = dict(index=10, name="table2-ops-4096xh4-100000x8", P=4_096, h=4,
                     funcs=PAPER_SET, N=100_000, F=8, x=("uniform", 0.5, 3.0), y_h=4,
                     y_funcs=PAPER_SET, noise=0.01, fos=True)
# Experiment III ladder (Table 1): 100,000 x 9, depth-6 templates over the
# Experiment III operators, the starting population of 2,000; X ~ U[1, 5]
# (the paper does not state the sampling distribution)
for _i, _name in enumerate(("addition", "division", "subtraction", "multiplication",
                            "squaring")):
    CONFIGS["l_" + _name[:3]] = dict(
        index=5 + _i, name=f"ladder-{_name}-2000xh6-100000x9", P=2_000, h=6, funcs=EXP3_SET,
        N=100_000, F=9, x=("uniform", 1.0, 5.0), target=_name, noise=0.0, fos=False)
    # the same ladder with the depth-8 templates (511 nodes) of Table 2
    CONFIGS["l8_" + _name[:3]] = dict(
        index=11 + _i, name=f"ladder-{_name}-2000xh8-100000x9", P=2_000, h=8, funcs=EXP3_SET,
        N=100_000, F=9, x=("uniform", 1.0, 5.0), target=_name, noise=0.0, fos=False)


def seed_of(cfg: str, rep: int = 0) -> int:
    return 1000 * CONFIGS[cfg]["index"] + rep


def workload(cfg: str, rep: int = 0, n_rows: int | None = None,
             n_trials: int | None = None, layout: str = "heap",
             fos_step: int = 0) -> dict:
    """Build one seeded workload.  ``n_rows`` / ``n_trials`` shrink it for
    tests (same recipe, fewer draws).  Returns a dict with

    X        float32 [N, F] row-major
    op, cval trial templates [P, stride] (uint8 / float32), in ``layout``
    heights  int8 [P]; h_max
    y_cands  generator: candidate y-generating trees (op, cval, h) in heap
             layout; the consumer evaluates them and keeps the first whose
             values are finite with nonzero variance
    z        float64 [N] standard-normal draws for the target noise
    noise    noise fraction (sigma = noise * std(f_gen))
    uses_pow whether the trials' function set has pow
    """
    c = CONFIGS[cfg]
    ss = np.random.SeedSequence(seed_of(cfg, rep))
    r_x, r_y, r_t, r_z, r_f = [np.random.default_rng(s) for s in ss.spawn(5)]
    N = int(n_rows if n_rows is not None else c["N"])
    P = int(n_trials if n_trials is not None else c["P"])
    F = c["F"]
    h_max = c["h"]
    X = _x(r_x, N, F, c["x"])
    if "h_min" in c:
        heights = r_t.integers(c["h_min"], h_max + 1, P)
    else:
        heights = np.full(P, h_max)
    if "p_func_range" in c:
        p_func = r_t.uniform(c["p_func_range"][0], c["p_func_range"][1], P)
    elif "p_func" in c:
        p_func = np.full(P, c["p_func"])
    else:  # half "full" trees, half "grow" trees
        p_func = np.where(r_t.random(P) < 0.5, 1.0, 0.5)
    op, cval, heights = random_templates(
        r_t, P, heights, h_max, c["funcs"], F, p_func,
        erc_leaves=c.get("erc_leaves", False))
    if c["fos"]:
        stride = op.shape[1]
        order = np.argsort(r_f.random((P, stride)), axis=1)
        op, cval = fos_step_trials(r_f, op, cval, fos_step % stride, order)
    if layout == "prefix":
        op, cval = to_prefix(op, cval, heights.astype(np.int64))
    elif layout != "heap":
        raise ValueError(layout)
    z = r_z.standard_normal(N)

    def y_cands(max_tries: int = 200):
        for _ in range(max_tries):
            pf = 1.0 if r_y.random() < 0.5 else 0.5
            gop, gcv, _ = random_templates(r_y, 1, c["y_h"], c["y_h"], c["y_funcs"], F, pf)
            yield gop[0], gcv[0], c["y_h"]

    out = dict(cfg=cfg, name=c["name"], X=X, op=op, cval=cval, heights=heights,
               h_max=h_max, layout=layout, y_cands=y_cands if "target" not in c else None,
               z=z, noise=float(c["noise"]), N=N, P=P, F=F, uses_pow=POW in c["funcs"])
    if "target" in c:  # a closed-form target (Table 1), given directly
        out["y"] = LADDER[c["target"]](X.astype(np.float64)).astype(np.float32)
    return out


def make_target(f_gen: np.ndarray, z: np.ndarray, noise: float) -> np.ndarray:
    """y = f_gen + noise * std(f_gen) * z, stored as float32."""
    f = np.asarray(f_gen, dtype=np.float64)
    y = f + noise * float(np.std(f)) * np.asarray(z, dtype=np.float64)
    return y.astype(np.float32)
