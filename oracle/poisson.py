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

from . import thomas, thomas_quasi


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


def laplacian5_neumann_y(u: np.ndarray) -> np.ndarray:
    """-Laplace_h(u) on [M, My] values: five-point stencil, x nodes at i / (M + 1) with zero
    Dirichlet values beyond them, y cell centres at (j + 1/2) / My with du/dy = 0 at y = 0, 1
    (ghost cells equal to their neighbours)."""
    M, My = u.shape
    hx, hy = 1.0 / (M + 1), 1.0 / My
    p = np.zeros((M + 2, My + 2))
    p[1:-1, 1:-1] = u
    p[1:-1, 0] = u[:, 0]
    p[1:-1, -1] = u[:, -1]
    c = p[1:-1, 1:-1]
    return (2.0 * c - p[:-2, 1:-1] - p[2:, 1:-1]) / (hx * hx) + (2.0 * c - p[1:-1, :-2] - p[1:-1, 2:]) / (hy * hy)


def poisson2d_neumann_y(f: np.ndarray) -> np.ndarray:
    """u with laplacian5_neumann_y(u) = f by separation of variables: orthonormal DST-I along x;
    mode k leaves the quasi-Toeplitz system of eq. 21 along y, tridiag{-1, t_0(k), -1} with
    t_0(k) = 2 + (hy / hx)^2 4 sin^2(k pi / (2 (M + 1))) and psi = chi = -1 (the Neumann rows),
    right-hand side hy^2 fhat_k; inverse DST-I."""
    f = np.asarray(f, dtype=np.float64)
    M, My = f.shape
    hx, hy = 1.0 / (M + 1), 1.0 / My
    fhat = scipy.fft.dst(f, type=1, norm="ortho", axis=0)
    v = np.empty_like(fhat)
    for k in range(1, M + 1):
        t0 = 2.0 + (hy / hx) ** 2 * 4.0 * math.sin(k * math.pi / (2.0 * (M + 1))) ** 2
        v[k - 1] = thomas_quasi((-1.0, t0, -1.0), -1.0, -1.0, hy * hy * fhat[k - 1])
    return scipy.fft.dst(v, type=1, norm="ortho", axis=0)
