"""Derive the sin and cos polynomial coefficients of gmath.cuh.

sin r = r + r^3 p(r^2) with p of degree 2 and cos r = 1 - r^2/2 + r^4 q(r^2)
with q of degree 2, on |r| <= pi/4 (the range the Cody-Waite reduction
leaves).  p and q minimise the largest relative error of sin and cos: the
Remez exchange algorithm (E. Ya. Remez, 1934) on the weighted error
w(s) (p(s) - g(s)), s = r^2, g the exact quotient, w the factor that turns
it into the relative error of the function.  The coefficients are then
rounded to FP32 and each is moved by up to two FP32 steps to minimise the
largest error of the FP32 evaluation itself (Horner's rule with fused
multiply-adds, emulated in FP64 and rounded to FP32 after every operation),
measured in FP32 units in the last place against the FP64 function.

Run: python trig_minimax.py (needs mpmath and numpy; not part of the build).
"""
from __future__ import annotations

import itertools

import mpmath as mp
import numpy as np

mp.mp.dps = 40
R = mp.pi / 4


def g_sin(s):
    x = mp.sqrt(s)
    return (mp.sin(x) - x) / x ** 3


def w_sin(s):
    x = mp.sqrt(s)
    return x ** 3 / mp.sin(x)


def g_cos(s):
    x = mp.sqrt(s)
    return (mp.cos(x) - 1 + s / 2) / s ** 2


def w_cos(s):
    return s ** 2 / mp.cos(mp.sqrt(s))


def remez(g, w, deg, hi, iters=30, grid_n=4000):
    """Coefficients c_0..c_deg of the minimax p (lowest power first) on
    (0, hi] and the largest weighted error."""
    n = deg + 2
    ref = [hi * (1 - mp.cos(mp.pi * (i + mp.mpf(1) / 2) / n)) / 2 for i in range(n)]
    grid = [hi * mp.mpf(k) / grid_n for k in range(1, grid_n + 1)]
    for _ in range(iters):
        A = mp.matrix(n, n)
        b = mp.matrix(n, 1)
        for i, s in enumerate(ref):
            ws = w(s)
            for j in range(deg + 1):
                A[i, j] = ws * s ** j
            A[i, deg + 1] = (-1) ** i
            b[i] = ws * g(s)
        sol = mp.lu_solve(A, b)
        c = [sol[j] for j in range(deg + 1)]
        err = [w(s) * (sum(c[j] * s ** j for j in range(deg + 1)) - g(s)) for s in grid]
        ext, best = [], None
        for s, e in zip(grid, err):  # the largest point of every run of one sign
            if best is not None and mp.sign(e) != mp.sign(best[1]):
                ext.append(best)
                best = None
            if best is None or abs(e) > abs(best[1]):
                best = (s, e)
        ext.append(best)
        while len(ext) > n:  # drop the smaller end until n alternations remain
            ext.pop(0 if abs(ext[0][1]) < abs(ext[-1][1]) else -1)
        if len(ext) == n:
            ref = [s for s, _ in ext]
    return [float(x) for x in c], float(max(abs(e) for e in err))


def fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(np.float32)


def ulp32(v):
    v = np.abs(np.asarray(v, np.float64)).astype(np.float32)
    return np.spacing(np.maximum(v, np.float32(1.17549435e-38))).astype(np.float64)


def horner_sin(r, c):  # c highest power first
    s = (r * r).astype(np.float32)
    p = fma32(s, c[0], c[1])
    for k in c[2:]:
        p = fma32(s, p, k)
    return fma32((r * s).astype(np.float32), p, r)


def horner_cos(r, c):
    s = (r * r).astype(np.float32)
    p = fma32(s, c[0], c[1])
    for k in c[2:]:
        p = fma32(s, p, k)
    return fma32(s, p, np.float32(1.0))


def refine(ev, fn, c, r, free):
    """Move each of the first `free` coefficients by up to two FP32 steps;
    keep the combination with the smallest largest error in ulps."""
    want = fn(r.astype(np.float64))
    c = [np.float32(x) for x in c]
    best = None
    for d in itertools.product(range(-2, 3), repeat=free):
        t = list(c)
        for i, k in enumerate(d):
            for _ in range(abs(k)):
                t[i] = np.nextafter(t[i], np.float32(np.inf if k > 0 else -np.inf))
        e = float(np.max(np.abs(ev(r, t).astype(np.float64) - want) / ulp32(want)))
        if best is None or e < best[0]:
            best = (e, t)
    return best


def main():
    r = np.concatenate([np.linspace(0, float(R), 200001), np.linspace(0.99 * float(R), float(R), 20001)])
    r = r[r > 0].astype(np.float32)
    cs, es = remez(g_sin, w_sin, 2, R * R)
    cc, ec = remez(g_cos, w_cos, 2, R * R)
    print(f"sin: Remez relative error {es:.3g}")
    print(f"cos: Remez relative error {ec:.3g}")
    e_s, sin_c = refine(horner_sin, np.sin, cs[::-1], r, 3)
    e_c, cos_c = refine(horner_cos, np.cos, cc[::-1] + [-0.5], r, 3)
    print(f"sin coefficients (r^7, r^5, r^3): {[str(x) for x in sin_c]}, "
          f"FP32 evaluation {e_s:.3f} ulp")
    print(f"cos coefficients (r^8, r^6, r^4, r^2): {[str(x) for x in cos_c]}, "
          f"FP32 evaluation {e_c:.3f} ulp")


if __name__ == "__main__":
    main()
