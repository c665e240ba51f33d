"""Pins of the GOM-step oracle (Algorithm 1) on hand-written cases."""
import math

import numpy as np

from oracle import gom
from fixtures import ERC, heap_template


def test_donate_copies_the_subset_from_the_donor():
    pop_op = np.array([[0, 32, 33], [2, 31, 34]], np.uint8)
    pop_cv = np.array([[0, 0, 0], [0, 1.5, 0]], np.float32)
    op = pop_op.copy()
    cv = pop_cv.copy()
    fos = [[0], [1, 2], [0, 1, 2]]
    # offspring 0 takes subset 1 from member 1; offspring 1 subset 0 from member 0
    o, c = gom.donate(op, cv, pop_op, pop_cv, donor=[1, 0], subset=[1, 0], fos=fos)
    assert o.tolist() == [[0, 31, 34], [0, 31, 34]]
    assert c.tolist() == [[0, 1.5, 0], [0, 1.5, 0]]
    # out-of-range donor or subset: unchanged
    o, c = gom.donate(op, cv, pop_op, pop_cv, donor=[5, 0], subset=[1, 9], fos=fos)
    assert o.tolist() == op.tolist()


def rows(*trees, h=2):
    ops, cvs = zip(*(heap_template(t, h) for t in trees))
    return np.stack(ops), np.stack(cvs)


def test_changed_only_for_active_parts():
    b_op, b_cv = rows(["+", "x0", "2.5", "x1", "x2", None, None])
    cases = {
        0: ["+", "x0", "2.5", "x3", "x2", None, None],       # intron under x0 changed
        1: ["-", "x0", "2.5", "x1", "x2", None, None],       # active function changed
        1.5: ["+", "x0", "3.5", "x1", "x2", None, None],     # active ERC constant changed
        2: ["+", "sin", "2.5", "x1", "x2", None, None],      # terminal -> function
    }
    for want, tree in [(0, cases[0]), (1, cases[1]), (1, cases[1.5]), (1, cases[2])]:
        o, c = rows(tree)
        got = gom.changed(o, c, b_op, b_cv, heights=[2], layout="heap", n_features=4)
        assert got.tolist() == [want], tree
    # a unary function's right child is an intron
    bo, bc = rows(["sin", "x0", "x1", None, None, None, None])
    o, c = rows(["sin", "x0", "x2", None, None, None, None])
    assert gom.changed(o, c, bo, bc, [2], "heap", 4).tolist() == [0]
    # an intron ERC whose constant changes: not changed
    bo, bc = rows(["+", "x0", "x1", "2.5", None, None, None])
    o, c = rows(["+", "x0", "x1", "-7", None, None, None])
    assert gom.changed(o, c, bo, bc, [2], "heap", 4).tolist() == [0]


def test_accept_rules():
    op = np.array([[0], [1], [2], [3], [4], [5]], np.uint8)
    bop = np.array([[9]] * 6, np.uint8)
    cv = np.zeros((6, 1), np.float32)
    bcv = np.ones((6, 1), np.float32)
    f_new = np.array([1.0, 3.0, 2.0, math.nan, 1.0, 5.0], np.float32)
    f_old = np.array([2.0, 2.0, 2.0, 2.0, math.nan, 1.0], np.float32)
    ch = np.array([1, 1, 1, 1, 1, 0], np.uint8)
    o, c, b, bc, fo, acc = gom.accept(op, cv, bop, bcv, ch, f_new, f_old)
    # better, worse, equal, NaN over number, number over NaN, unchanged
    assert acc.tolist() == [1, 0, 1, 0, 1, 1]
    assert o[:, 0].tolist() == [0, 9, 2, 9, 4, 5]
    assert b[:, 0].tolist() == [0, 9, 2, 9, 4, 5]
    assert fo[:3].tolist() == [1.0, 2.0, 2.0] and fo[3] == 2.0 and fo[4] == 1.0
    assert fo[5] == 1.0  # unchanged keeps its backup fitness
