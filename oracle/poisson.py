"""Oracle for the 2-D Dirichlet Poisson problem by separation of variables (Sec. 3.2, Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).  -Laplace(u) = f on the unit square,
u = 0 on the boundary, five-point stencil, (M + 1) x (M + 1) intervals, h = 1 / (M + 1),
u and f as [M, M] arrays indexed [i, j] = (x_i, y_j).  Steps, each a plain library call or the
oracle's Thomas solve:
  fhat = orthonormal DST-I of f along x (scipy.fft.dst, type 1),
  for every mode k: Thomas on tridiag{-1, 2 + 4 sin^2(k pi / (2 (M + 1))), -1} v_k = h^2 fhat_k,
  u = orthonormal DST-I of v along x (the transform is its own inverse).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft

from . import thomas


def laplacian5(u: np.ndarray) -> np.ndarray:
    """-Laplace_h(u) with the five-point stencil and zero boundary values (u: [M, M])."""
    M = u.shape[0]
    h = 1.0 / (M + 1)
    p = np.zeros((M + 2, M + 2))
    p[1:-1, 1:-1] = u
    return (4.0 * p[1:-1, 1:-1] - p[:-2, 1:-1] - p[2:, 1:-1] - p[1:-1, :-2] - p[1:-1, 2:]) / (h * h)


def poisson2d(f: np.ndarray) -> np.ndarray:
    """u with -Laplace_h(u) = f (five-point stencil, Dirichlet zero), by separation of variables."""
    f = np.asarray(f, dtype=np.float64)
    M = f.shape[0]
    h = 1.0 / (M + 1)
    fhat = scipy.fft.dst(f, type=1, norm="ortho", axis=0)
    v = np.empty_like(fhat)
    for k in range(1, M + 1):
        t0 = 2.0 + 4.0 * math.sin(k * math.pi / (2.0 * (M + 1))) ** 2
        v[k - 1] = thomas((-1.0, t0, -1.0), h * h * fhat[k - 1])
    return scipy.fft.dst(v, type=1, norm="ortho", axis=0)
