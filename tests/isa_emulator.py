"""A slow FP64 emulator of the interpreter's instruction set, for CPU tests
of the packer.  The instruction forms are the ones documented at the top of
the library's ``csrc/isa.h``; the numbering is written out here by hand.
"""
import math

import numpy as np

I_LDF0, I_LDC0, I_UN, I_BF, I_BC, I_LF, I_LC, I_BS, I_RS, I_LDF, I_LDC, I_NOP = \
    0, 1, 2, 10, 15, 20, 25, 30, 70, 110, 118, 126
I_PW, I_PWS, I_PWR, I_END = 127, 131, 139, 147  # pow: fused groups, then slot forms
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
    opc = int(word) & 0xFF
    feat = int(word) >> 8
    if opc == I_LDF0:
        return ("ldf", None, feat)
    if opc == I_LDC0:
        return ("ldc", None, None)
    if I_UN <= opc < I_BF:
        return ("un", opc - I_UN, None)
    if I_BF <= opc < I_BS:
        grp, k = divmod(opc - I_BF, 5)
        return (["bf", "bc", "lf", "lc"][grp], k, feat)
    if I_BS <= opc < I_RS:
        k, j = divmod(opc - I_BS, 8)
        return ("bs", (k, j), None)
    if I_RS <= opc < I_LDF:
        k, j = divmod(opc - I_RS, 8)
        return ("rs", (k, j), None)
    if I_LDF <= opc < I_LDC:
        return ("ldf", opc - I_LDF, feat)
    if I_LDC <= opc < I_NOP:
        return ("ldc", opc - I_LDC, None)
    if I_PW <= opc < I_PWS:
        return (["bf", "bc", "lf", "lc"][opc - I_PW], 5, feat)
    if I_PWS <= opc < I_PWR:
        return ("bs", (5, opc - I_PWS), None)
    if I_PWR <= opc < I_END:
        return ("rs", (5, opc - I_PWR), None)
    raise ValueError(opc)


def run(words, consts, X, max_slots=8):
    """Evaluate a packed program over all rows of X (FP64)."""
    n = X.shape[0]
    A = np.zeros(n)
    S = [np.zeros(n) for _ in range(max_slots)]
    used = -1
    for w, c in zip(words, consts):
        form, arg, feat = decode(w)
        c = float(c)
        if form in ("ldf", "ldc"):
            if arg is not None:
                S[arg] = A.copy()
                used = max(used, arg)
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
            k, j = arg
            A = binop(k, S[j], A)
        elif form == "rs":
            k, j = arg
            A = binop(k, A, S[j])
    return A, used + 1


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
            out.append(f"{form} {KINDS[arg[0]]} s{arg[1]}")
    return out
