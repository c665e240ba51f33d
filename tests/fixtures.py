"""Shared test helpers: golden-file parsing and small tree builders.

Builds templates from hand-written token lists; holds no evaluation code.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# interface opcodes, written out as in the header
ADD, SUB, MUL, AQ = 0, 1, 2, 3
SIN, COS, EXP, LOG_ABS, SQRT_ABS = 4, 5, 6, 7, 8
DIV, SQUARE, LOG, SQRT, POW = 9, 10, 11, 12, 13
ERC, FEAT0, PAD = 31, 32, 255

TOKENS = {"+": ADD, "-": SUB, "*": MUL, "aq": AQ, "sin": SIN, "cos": COS,
          "exp": EXP, "logabs": LOG_ABS, "sqrtabs": SQRT_ABS, "/": DIV,
          "sq": SQUARE, "log": LOG, "sqrt": SQRT, "pow": POW}


def token_to_node(tok):
    """'x3' -> (FEAT0+3, 0); '-2' -> (ERC, -2.0); '/' -> (DIV, 0)."""
    if tok in TOKENS:
        return TOKENS[tok], 0.0
    if tok[0] == "x" and tok[1:].isdigit():
        return FEAT0 + int(tok[1:]), 0.0
    return ERC, float(tok)


def read_golden(name):
    rows = {}
    tree = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            if key == "tree":
                tree[int(rest[0])] = rest[1]
            else:
                rows[key] = rest
    return tree, rows


def heap_template(tokens, h):
    """Template row (op uint8, cval float32) of height h from a dict or list
    of heap-ordered tokens; unspecified positions are PAD."""
    n = (1 << (h + 1)) - 1
    op = np.full(n, PAD, dtype=np.uint8)
    cv = np.zeros(n, dtype=np.float32)
    items = tokens.items() if isinstance(tokens, dict) else enumerate(tokens)
    for i, tok in items:
        if tok is None:
            continue
        o, c = token_to_node(tok)
        op[i] = o
        cv[i] = c
    return op, cv


def fig1():
    tree, rows = read_golden("fig1_tree.txt")
    op, cv = heap_template(tree, 3)
    return op, cv, rows
