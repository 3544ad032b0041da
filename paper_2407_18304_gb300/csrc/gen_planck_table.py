#!/usr/bin/env python3
"""Write planck_table.h: piecewise polynomials for the group Planck integrals.

With I(x) = int_0^x t^3/(e^t - 1) dt (so P(x) = 15/pi^4 I(x)) the CUDA
library evaluates
    g(x) = I(x) / x^3                      for x < 2  (P = 15/pi^4 x^3 g),
    h(x) = e^x (pi^4/15 - I(x)) / x^3      for x >= 2 (Q = 15/pi^4 x^3 e^-x h),
both smooth and slowly varying, as polynomials in u = (x - c_s) / w_s on
segments s.  Segments: [0, 2^-8) (centre 0, Taylor-like), then every octave
[2^e, 2^(e+1)) for e = -8 .. 9 split into four equal parts; beyond 2^10
Q underflows in FP64 and is taken as 0.  The segment of an x is read off its
binary exponent and two leading mantissa bits, so the device code evaluates
every edge with the same instructions (no branch on x).

The values come from mpmath at 50 digits: g from the Bernoulli series of
t/(e^t - 1) (convergent for x < 2 pi), h from the exponential tail series
sum_n e^(-n x) (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4); each segment polynomial
interpolates at Chebyshev points and
is converted to the monomial basis in u.  The script checks every segment
against mpmath at 400 points and fails above 4e-16 relative.

    python paper_2407_18304_gb300/csrc/gen_planck_table.py   (needs mpmath)
"""
from __future__ import annotations

import os
import sys

import mpmath as mp

mp.mp.dps = 50
DEG = 13                  # polynomial degree (DEG + 1 coefficients)
E_MIN, E_MAX = -8, 9      # octaves [2^e, 2^(e+1)) covered by four segments each
SUB = 4
N_SEG = 1 + SUB * (E_MAX - E_MIN + 1)
X_SPLIT = 2
TOL = 4e-16  # about two units in the last place

def g(x):
    """I(x)/x^3 from t^3/(e^t-1) = sum_k B_k t^(k+2)/k! (|x| < 2 pi)."""
    if x == 0:
        return mp.mpf(1) / 3
    s = mp.mpf(0)
    for k in range(0, 140):
        s += mp.bernoulli(k) * x ** k / (mp.factorial(k) * (k + 3))
    return s


def h(x):
    """e^x (pi^4/15 - I(x))/x^3 from the tail sum_n e^(-n x) (x^3/n + 3x^2/n^2
    + 6x/n^3 + 6/n^4) (x > 0; used from x = 2)."""
    s = mp.mpf(0)
    for n in range(1, 400):
        t = mp.e ** (-(n - 1) * x) * (x ** 3 / n + 3 * x ** 2 / n ** 2 + 6 * x / n ** 3
                                      + mp.mpf(6) / n ** 4)
        s += t
        if t < mp.mpf(10) ** (-60) * s:
            break
    return s / x ** 3


def segment(s):
    """(lo, hi) of segment s."""
    if s == 0:
        return mp.mpf(0), mp.mpf(2) ** E_MIN
    k = s - 1
    e, q = E_MIN + k // SUB, k % SUB
    base = mp.mpf(2) ** e
    return base * (1 + mp.mpf(q) / SUB), base * (1 + mp.mpf(q + 1) / SUB)


def fit(f, lo, hi):
    """Monomial coefficients in u = (x - c)/w of the Chebyshev interpolant."""
    c, w = (lo + hi) / 2, (hi - lo) / 2
    n = DEG + 1
    nodes = [mp.cos(mp.pi * (2 * j + 1) / (2 * n)) for j in range(n)]
    vals = [f(c + w * u) for u in nodes]
    # Chebyshev coefficients
    cheb = []
    for k in range(n):
        s = sum(vals[j] * mp.cos(mp.pi * k * (2 * j + 1) / (2 * n)) for j in range(n))
        cheb.append(s * (1 if k == 0 else 2) / n)
    # to monomials: T_k(u) expanded
    T = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for k in range(2, n):
        a = [mp.mpf(0)] + [2 * t for t in T[k - 1]]
        b = T[k - 2] + [mp.mpf(0)] * (len(a) - len(T[k - 2]))
        T.append([x - y for x, y in zip(a, b)])
    mono = [mp.mpf(0)] * n
    for k in range(n):
        for i, t in enumerate(T[k]):
            mono[i] += cheb[k] * t
    return c, w, mono


def check(f, lo, hi, c, w, coef):
    worst = 0.0
    for j in range(401):
        x = lo + (hi - lo) * mp.mpf(j) / 400
        if x == 0:
            continue
        # evaluate in binary64 the way the device does (Horner in u)
        xf = float(x)
        u = (xf - float(c)) * float(1 / w)
        p = float(coef[DEG])
        for k in range(DEG - 1, -1, -1):
            p = p * u + float(coef[k])
        ref = f(mp.mpf(xf))
        worst = max(worst, float(abs((p - ref) / ref)))
    return worst


def main(out):
    rows, worst = [], 0.0
    for s in range(N_SEG):
        lo, hi = segment(s)
        f = g if hi <= X_SPLIT else h
        c, w, coef = fit(f, lo, hi)
        err = check(f, lo, hi, c, w, coef)
        worst = max(worst, err)
        if err > TOL:
            sys.exit(f"segment {s} [{lo}, {hi}): relative error {err:.3e} > {TOL}")
        rows.append((float(c), float(1 / w), [float(a) for a in coef]))
    with open(out, "w") as fh:
        fh.write("// planck_table.h -- written by gen_planck_table.py (do not edit).\n")
        fh.write("// Piecewise polynomials of g(x) = I(x)/x^3 (x < 2) and\n")
        fh.write("// h(x) = e^x (pi^4/15 - I(x))/x^3 (x >= 2), I(x) = int_0^x t^3/(e^t-1) dt,\n")
        fh.write(f"// in u = (x - centre) * inv_halfwidth; degree {DEG}; {N_SEG} segments;\n")
        fh.write(f"// worst relative error in binary64 Horner evaluation: {worst:.2e}.\n")
        fh.write("#pragma once\n\nnamespace rhd {\nnamespace planck_table {\n\n")
        fh.write(f"constexpr int kDeg = {DEG};\nconstexpr int kSeg = {N_SEG};\n")
        fh.write(f"constexpr int kEMin = {E_MIN};\nconstexpr int kEMax = {E_MAX};\n")
        fh.write(f"constexpr int kSub = {SUB};\n\n")
        fh.write("// centre, 1 / half-width of each segment\n")
        fh.write("constexpr double kCentre[kSeg] = {\n")
        fh.write(",\n".join(f"    {r[0].hex()}" for r in rows) + "};\n")
        fh.write("constexpr double kInvHalf[kSeg] = {\n")
        fh.write(",\n".join(f"    {r[1].hex()}" for r in rows) + "};\n")
        fh.write("// coefficient k of segment s at kCoef[k][s]\n")
        fh.write("constexpr double kCoef[kDeg + 1][kSeg] = {\n")
        for k in range(DEG + 1):
            fh.write("    {" + ", ".join(r[2][k].hex() for r in rows) + "},\n")
        fh.write("};\n\n}  // namespace planck_table\n}  // namespace rhd\n")
    print(f"wrote {out}: {N_SEG} segments, worst relative error {worst:.2e}")


if __name__ == "__main__":
    main(os.path.join(os.path.dirname(os.path.abspath(__file__)), "planck_table.h"))
