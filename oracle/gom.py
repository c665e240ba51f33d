"""One GOM step over a FOS index (Algorithm 1's inner loop), plain NumPy.

Test infrastructure only (see the package docstring).  Definitions:

* donate: offspring j takes the nodes of FOS subset s_j from population
  member d_j: O_j[FOS[s_j]] <- P_{d_j}[FOS[s_j]] (Algorithm 1).
* changed: O_j differs from its backup B_j at a node active in either
  (opcode, or the constant of an ERC) - the paper evaluates an offspring
  only if an actively used part of the template changed (Section 3.1).
* accept: keep O_j when unchanged or when f(O_j) is not worse than f(B_j)
  (Section 3.1, Algorithm 1; READING: a NaN never replaces a number, a
  number always replaces a NaN), then B_j <- O_j; otherwise O_j <- B_j.
"""
import numpy as np

from .gp import BINARY, ERC, UNARY, InvalidTemplate, Template


def donate(op, cval, pop_op, pop_cval, donor, subset, fos):
    """Return new (op, cval) after the donor copy; fos is a list of lists of
    template positions."""
    op = op.copy()
    cval = cval.copy()
    for j in range(op.shape[0]):
        s, d = int(subset[j]), int(donor[j])
        if not (0 <= s < len(fos) and 0 <= d < pop_op.shape[0]):
            continue
        for node in fos[s]:
            if 0 <= node < op.shape[1]:
                op[j, node] = pop_op[d, node]
                cval[j, node] = pop_cval[d, node]
    return op, cval


def _active_loose(op_row, h, layout, n_features):
    """Active mask; an invalid active node stops the walk below it but is
    itself marked (a changed test does not need a valid tree)."""
    t = Template(op_row, np.zeros(op_row.size, np.float32), h, layout, n_features)
    mask = np.zeros(op_row.size, dtype=bool)

    def visit(pos, depth):
        mask[pos] = True
        try:
            o = t.check(pos, depth)
        except InvalidTemplate:
            return
        l, r = t.children(pos, depth)
        if o in BINARY:
            visit(l, depth + 1)
            visit(r, depth + 1)
        elif o in UNARY:
            visit(l, depth + 1)

    visit(0, 0)
    return mask


def changed(op, cval, bop, bcval, heights, layout, n_features):
    out = np.zeros(op.shape[0], dtype=np.uint8)
    for j in range(op.shape[0]):
        h = int(heights[j])
        n = (1 << (h + 1)) - 1
        act = _active_loose(op[j], h, layout, n_features)[:n] | \
            _active_loose(bop[j], h, layout, n_features)[:n]
        diff = (op[j, :n] != bop[j, :n]) | ((op[j, :n] == ERC) & (cval[j, :n] != bcval[j, :n]))
        out[j] = np.uint8(bool(np.any(act & diff)))
    return out


def accept(op, cval, bop, bcval, ch, f_new, f_old):
    """Return (op, cval, bop, bcval, f_old, accepted) after accept/revert."""
    op, cval, bop, bcval, f_old = op.copy(), cval.copy(), bop.copy(), bcval.copy(), f_old.copy()
    acc = np.zeros(op.shape[0], dtype=np.uint8)
    for j in range(op.shape[0]):
        c = True if ch is None else bool(ch[j])
        fn, fo = float(f_new[j]), float(f_old[j])
        a = (not c) or fn <= fo or (np.isnan(fo) and not np.isnan(fn))
        if a:
            bop[j], bcval[j] = op[j], cval[j]
            if c:
                f_old[j] = f_new[j]
        else:
            op[j], cval[j] = bop[j], bcval[j]
        acc[j] = a
    return op, cval, bop, bcval, f_old, acc
