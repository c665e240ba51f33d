"""A slow FP64 emulator of the interpreter's instruction set, for CPU tests
of the packer.  The instruction forms are the ones documented at the top of
the library's ``csrc/isa.h``; the numbering is written out here by hand.
"""
import math

import numpy as np

I_LDF0, I_LDC0, I_PSF, I_PSC, I_UN, I_BF, I_BC, I_LF, I_LC, I_BS, I_RS, I_NOP = \
    0, 1, 2, 3, 4, 12, 17, 22, 27, 32, 37, 42
I_PW, I_PWS, I_PWR, I_END = 43, 47, 48, 49  # pow: fused groups, then the stack forms
KINDS = ["+", "-", "*", "aq", "/", "pow"]
UNARY = ["sin", "cos", "exp", "logabs", "sqrtabs", "sq", "log", "sqrt"]


def binop(k, a, b):
    with np.errstate(all="ignore"):
        if k == 0:
            return a + b
        if k == 1:
            return a - b
        if k == 2:
            return a * b
        if k == 3:
            return a / np.sqrt(1.0 + b * b)
        if k == 5:
            return np.power(a, b)
        return a / b


def unop(u, a):
    with np.errstate(all="ignore"):
        return [np.sin, np.cos, np.exp, lambda x: np.log(np.abs(x)), lambda x: np.sqrt(np.abs(x)),
                lambda x: x * x, np.log, np.sqrt][u](a)


def decode(word):
    """(form, arg, feature) of one instruction word; form is ldf / ldc (with
    arg True when the load pushes A first), un, bf, bc, lf, lc, bs or rs."""
    opc = int(word) & 0xFF
    feat = int(word) >> 8
    if opc in (I_LDF0, I_PSF):
        return ("ldf", opc == I_PSF, feat)
    if opc in (I_LDC0, I_PSC):
        return ("ldc", opc == I_PSC, None)
    if I_UN <= opc < I_BF:
        return ("un", opc - I_UN, None)
    if I_BF <= opc < I_BS:
        grp, k = divmod(opc - I_BF, 5)
        return (["bf", "bc", "lf", "lc"][grp], k, feat)
    if I_BS <= opc < I_RS:
        return ("bs", opc - I_BS, None)
    if I_RS <= opc < I_NOP:
        return ("rs", opc - I_RS, None)
    if I_PW <= opc < I_PWS:
        return (["bf", "bc", "lf", "lc"][opc - I_PW], 5, feat)
    if opc == I_PWS:
        return ("bs", 5, None)
    if opc == I_PWR:
        return ("rs", 5, None)
    raise ValueError(opc)


def run(words, consts, X):
    """Evaluate a packed program over all rows of X (FP64); returns the
    values and the deepest stack (slots) the program used."""
    n = X.shape[0]
    A = np.zeros(n)
    stack = []
    used = 0
    for w, c in zip(words, consts):
        form, arg, feat = decode(w)
        c = float(c)
        if form in ("ldf", "ldc"):
            if arg:
                stack.append(A.copy())
                used = max(used, len(stack))
            A = X[:, feat].astype(np.float64) if form == "ldf" else np.full(n, c)
        elif form == "un":
            A = unop(arg, A)
        elif form == "bf":
            A = binop(arg, A, X[:, feat].astype(np.float64))
        elif form == "bc":
            A = binop(arg, A, np.full(n, c))
        elif form == "lf":
            A = binop(arg, X[:, feat].astype(np.float64), A)
        elif form == "lc":
            A = binop(arg, np.full(n, c), A)
        elif form == "bs":
            A = binop(arg, stack.pop(), A)
        elif form == "rs":
            A = binop(arg, A, stack.pop())
    assert not stack, "program left values on the stack"
    return A, used


def tokens(words, consts):
    """Human-readable form of a program, e.g. ['ldc 4', 'bf * x0', ...]."""
    out = []
    for w, c in zip(words, consts):
        form, arg, feat = decode(w)
        if form == "ldf":
            out.append(f"ldf x{feat}")
        elif form == "ldc":
            out.append(f"ldc {float(c):g}")
        elif form == "un":
            out.append(f"un {UNARY[arg]}")
        elif form in ("bf", "lf"):
            out.append(f"{form} {KINDS[arg]} x{feat}")
        elif form in ("bc", "lc"):
            out.append(f"{form} {KINDS[arg]} {float(c):g}")
        else:
            out.append(f"{form} {KINDS[arg]}")
    return out
