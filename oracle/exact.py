"""Exact rational solution of a tridiagonal Toeplitz system.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every FP64 input (coefficients and right-hand side) is converted to a Fraction without
rounding, and the Thomas elimination is carried out in exact rational arithmetic, so the
result is the exact solution of the system the FP64 numbers describe.  Used for the small
golden fixtures under tests/golden/ and as brute force on tiny inputs.
"""
from __future__ import annotations

from fractions import Fraction


def solve_exact(t, F):
    """x = T^-1 F exactly (list of Fractions).  Raises ZeroDivisionError if a pivot vanishes."""
    tm1, t0, tp1 = (Fraction(float(v)) for v in t)
    f = [Fraction(float(v)) for v in F]
    n = len(f)
    if n == 0:
        return []
    cp = [Fraction(0)] * n
    dp = [Fraction(0)] * n
    m = t0
    cp[0] = tp1 / m
    dp[0] = f[0] / m
    for i in range(1, n):
        m = t0 - tm1 * cp[i - 1]
        cp[i] = tp1 / m
        dp[i] = (f[i] - tm1 * dp[i - 1]) / m
    x = [Fraction(0)] * n
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def residual_exact(t, x, F):
    """F - T x in exact arithmetic (x given as Fractions)."""
    tm1, t0, tp1 = (Fraction(float(v)) for v in t)
    n = len(x)
    r = []
    for i in range(n):
        v = t0 * x[i]
        if i > 0:
            v += tm1 * x[i - 1]
        if i + 1 < n:
            v += tp1 * x[i + 1]
        r.append(Fraction(float(F[i])) - v)
    return r
