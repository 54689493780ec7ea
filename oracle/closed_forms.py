"""Closed forms from the paper and from textbook linear algebra, used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``theorem1_inverse``  -- T^-1 entry by entry from Theorem 1 (eq. 20, Sec. 3.1).
  As printed, the formula carries a factor 1/t_1; reproducing T^-1 needs -1/t_1
  (the overall sign is flipped; the roots q_1, q_2 and the factor (q_1 q_2)^{n-k}
  stay as printed).  ``sign`` selects the reading; -1 is the one adopted.
* ``cheb_U``            -- Chebyshev polynomials of the second kind U_n(x) (eq. 23).
* ``laplace_prelim``    -- the preliminary vectors for tridiag{-1, 2x, -1} of order
  N-1 (N intervals, unknowns 1..N-1, eq. 22) by eq. 24 (Z^{L,R}) and eq. 25 (G^{L,R}).
* ``eigenpair``         -- lambda_k, v_k of a Toeplitz tridiagonal with t_1 t_-1 > 0:
  v_k(j) = (t_-1/t_1)^{j/2} sin(j k pi/(N+1)),
  lambda_k = t_0 + 2 sgn(t_1) sqrt(t_1 t_-1) cos(k pi/(N+1))   (j, k = 1..N).
"""
from __future__ import annotations

import math

import numpy as np


def theorem1_inverse(N: int, t, sign: float = -1.0) -> np.ndarray:
    """Dense T^-1 from eq. 20 with 1-based indices n (row) and k (column)."""
    tm1, t0, tp1 = (float(v) for v in t)
    disc = t0 * t0 - 4.0 * tm1 * tp1
    sq = math.sqrt(disc)
    q1 = (-t0 + sq) / (2.0 * tp1)
    q2 = (-t0 - sq) / (2.0 * tp1)
    den = (q2 - q1) * (q2 ** (N + 1) - q1 ** (N + 1))
    A = np.zeros((N, N))
    for n in range(1, N + 1):
        for k in range(1, N + 1):
            if k < n:
                num = (q1 * q2) ** (n - k) * (q2 ** (N + 1 - n) - q1 ** (N + 1 - n)) * (q2 ** k - q1 ** k)
            else:
                num = (q2 ** (N + 1 - k) - q1 ** (N + 1 - k)) * (q2 ** n - q1 ** n)
            A[n - 1, k - 1] = sign * num / den / tp1
    return A


def cheb_U(n: int, x: float) -> float:
    """U_n(x) by the three-term recurrence; U_{-1} = 0, U_0 = 1."""
    if n < 0:
        return 0.0
    u0, u1 = 1.0, 2.0 * x
    if n == 0:
        return u0
    for _ in range(n - 1):
        u0, u1 = u1, 2.0 * x * u1 - u0
    return u1


def laplace_prelim(N: int, x: float, mL: int, mR: int):
    """eq. 24-25 for the block [mL, mR] (1-based) of tridiag{-1, 2x, -1}, unknowns 1..N-1.

    Returns (ZL, ZR, GL, GR) as length N-1 arrays indexed by unknown-1; entries outside
    the ranges stated in eq. 24-25 are 0.
    """
    M = N - 1
    ZL, ZR, GL, GR = (np.zeros(M) for _ in range(4))
    UN1 = cheb_U(N - 1, x)
    for i in range(1, M + 1):
        if i <= mL:
            ZL[i - 1] = cheb_U(i - 1, x) / cheb_U(mL - 1, x)
        if i >= mR:
            ZR[i - 1] = cheb_U(N - i - 1, x) / cheb_U(N - mR - 1, x)
        if mL <= i <= mR:
            GL[i - 1] = cheb_U(N - i - 1, x) / UN1 * cheb_U(mL - 1, x)
            GR[i - 1] = cheb_U(i - 1, x) / UN1 * cheb_U(N - mR - 1, x)
    return ZL, ZR, GL, GR


def eigenpair(N: int, t, k: int):
    """(lambda_k, v_k) for t_1 t_-1 > 0, k = 1..N."""
    tm1, t0, tp1 = (float(v) for v in t)
    if tm1 * tp1 <= 0:
        raise ValueError("closed form needs t_1 t_-1 > 0")
    j = np.arange(1, N + 1, dtype=np.int64)
    rho = math.sqrt(tm1 / tp1)
    # reduce j*k modulo 2(N+1) in integers so the sine argument is accurate for large N
    r = (j * k) % (2 * (N + 1))
    v = rho ** j.astype(np.float64) * np.sin(r * math.pi / (N + 1))
    lam = t0 + 2.0 * math.copysign(1.0, tp1) * math.sqrt(tm1 * tp1) * math.cos(k * math.pi / (N + 1))
    return lam, v
