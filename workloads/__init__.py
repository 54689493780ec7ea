"""Seeded synthetic inputs for the Toeplitz tridiagonal workloads (both sides use these).

This module draws random numbers and lays out inputs; it contains none of the solver's
arithmetic and imports neither the oracle nor the CUDA package.  The paper's experiments
(Sec. 4) are synthetic Poisson problems on uniform grids, so every workload here is
synthetic; there is no dataset to stand in for.

Seeds (numpy ``default_rng`` / torch Philox): 0 right-hand sides and manufactured
solutions, 1 coefficients, 2 system sizes, 3 adjoint weights w.

Workloads
  C1 ``single_c1``   tridiag{-1, 4, -1}, N = 65536, F ~ U[-1, 1]; variant x* ~ U[-1, 1]
  C2 ``single_c2``   tridiag{-1.2, 2.5, -0.8}, N = 2^26, F ~ N(0, 1); variant {-1, 2.001, -1}
  C3 ``poisson_c3``  4096 modes of the 2-D Dirichlet Poisson problem on a 4097 x 4097-interval
                     grid (separation of variables, Sec. 3.2 and Sec. 4): mode k has
                     t = (-1, 2 + 4 sin^2(k pi / (2 * 4097)), -1), N = 4096, right-hand side
                     -h^2 * (orthonormal DST-I along x of a seeded smooth source)(k, y_j)
  C4 ``uneven_c4``   10000 systems, N = round(exp(U[ln 256, ln 2^20])), t_0 ~ U[2.05, 4],
                     t_-1, t_1 ~ U[-1, -0.5] independently, F ~ U[-1, 1]
  C5 ``adjoint_c5``  1024 systems of N = 65536, coefficients as C4, F, w ~ U[-1, 1]
"""
from __future__ import annotations

import math

import numpy as np

SEED_RHS, SEED_COEF, SEED_SIZE, SEED_W = 0, 1, 2, 3

T_C1 = (-1.0, 4.0, -1.0)
T_C2 = (-1.2, 2.5, -0.8)
T_C2_WEAK = (-1.0, 2.001, -1.0)


# ------------------------------------------------------------------ single systems
def single_c1(N: int = 65536, seed: int = SEED_RHS) -> tuple[tuple, np.ndarray]:
    """C1: t = {-1, 4, -1}, F ~ U[-1, 1]."""
    return T_C1, np.random.default_rng(seed).uniform(-1.0, 1.0, N)


def manufactured_x(N: int, seed: int = SEED_RHS) -> np.ndarray:
    """x* ~ U[-1, 1] for manufactured-solution variants (F = T x* is formed by the caller)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, N)


def single_c2(N: int = 1 << 26, weak: bool = False, seed: int = SEED_RHS) -> tuple[tuple, np.ndarray]:
    """C2: t = {-1.2, 2.5, -0.8} (or the weakly dominant {-1, 2.001, -1}), F ~ N(0, 1)."""
    return (T_C2_WEAK if weak else T_C2), np.random.default_rng(seed).standard_normal(N)


# ------------------------------------------------------------------ 2-D Poisson modes (C3)
def poisson_t0(M: int = 4096) -> np.ndarray:
    """t_0 of mode k = 1..M: 2 + 4 sin^2(k pi / (2 (M + 1)))."""
    k = np.arange(1, M + 1, dtype=np.float64)
    return 2.0 + 4.0 * np.sin(k * math.pi / (2.0 * (M + 1))) ** 2


def poisson_source(M: int = 4096, seed: int = SEED_RHS, n_bumps: int = 8) -> np.ndarray:
    """Smooth source on the interior grid points x_i = i h, y_j = j h (i, j = 1..M, h = 1/(M+1)):
    f = x(1-x) y(1-y) sum_b a_b exp(-|(x, y) - c_b|^2 / (2 * 0.1^2)), a_b ~ N(0,1), c_b ~ U[0.2, 0.8]^2.
    Returned as f[i-1, j-1] (x index first)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_bumps)
    c = rng.uniform(0.2, 0.8, size=(n_bumps, 2))
    h = 1.0 / (M + 1)
    g = np.arange(1, M + 1, dtype=np.float64) * h
    X = g[:, None]
    Y = g[None, :]
    f = np.zeros((M, M))
    for b in range(n_bumps):
        f += a[b] * np.exp(-((X - c[b, 0]) ** 2 + (Y - c[b, 1]) ** 2) / (2 * 0.1 ** 2))
    return f * (X * (1 - X)) * (Y * (1 - Y))


def dst1_ortho_x(f: np.ndarray) -> np.ndarray:
    """Orthonormal DST-I along the first (x) axis (scipy.fft.dst type 1, norm='ortho')."""
    from scipy.fft import dst
    return dst(f, type=1, axis=0, norm="ortho")


def poisson_c3(M: int = 4096, seed: int = SEED_RHS):
    """C3 as (t_m1[M], t_0[M], t_1[M], N[M], rhs [M, M] system-major: rhs[k-1, j-1])."""
    h = 1.0 / (M + 1)
    fhat = dst1_ortho_x(poisson_source(M, seed))
    rhs = np.ascontiguousarray(-(h * h) * fhat)
    t0 = poisson_t0(M)
    return -np.ones(M), t0, -np.ones(M), np.full(M, M, dtype=np.int64), rhs


# ------------------------------------------------------------------ uneven series (C4) / adjoint (C5)
def uneven_sizes(nsys: int = 10000, seed: int = SEED_SIZE, lo: int = 256, hi: int = 1 << 20) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), nsys))).astype(np.int64)


def dominant_coeffs(nsys: int, seed: int = SEED_COEF):
    """t_0 ~ U[2.05, 4], t_-1 ~ U[-1, -0.5], t_1 ~ U[-1, -0.5] (diagonally dominant)."""
    rng = np.random.default_rng(seed)
    t0 = rng.uniform(2.05, 4.0, nsys)
    tm1 = rng.uniform(-1.0, -0.5, nsys)
    tp1 = rng.uniform(-1.0, -0.5, nsys)
    return tm1, t0, tp1


def offsets(N: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(N)[:-1]]).astype(np.int64) if len(N) else np.zeros(0, np.int64)


def uneven_c4(nsys: int = 10000, with_rhs: bool = True, lo: int = 256, hi: int = 1 << 20):
    """C4 as (N, offsets, t_m1, t_0, t_1, F or None)."""
    N = uneven_sizes(nsys, lo=lo, hi=hi)
    tm1, t0, tp1 = dominant_coeffs(nsys)
    F = np.random.default_rng(SEED_RHS).uniform(-1.0, 1.0, int(N.sum())) if with_rhs else None
    return N, offsets(N), tm1, t0, tp1, F


def adjoint_c5(nsys: int = 1024, N: int = 65536, with_data: bool = True):
    """C5 as (N[], offsets, t_m1, t_0, t_1, F or None, w or None)."""
    Ns = np.full(nsys, N, dtype=np.int64)
    tm1, t0, tp1 = dominant_coeffs(nsys)
    F = w = None
    if with_data:
        F = np.random.default_rng(SEED_RHS).uniform(-1.0, 1.0, nsys * N)
        w = np.random.default_rng(SEED_W).uniform(-1.0, 1.0, nsys * N)
    return Ns, offsets(Ns), tm1, t0, tp1, F, w


# ------------------------------------------------------------------ device-side uniform draws
def device_uniform(n: int, seed: int, device, lo: float = -1.0, hi: float = 1.0):
    """U[lo, hi) float64 drawn on a CUDA device with torch's seeded Philox generator (for the
    multi-gigabyte benchmark inputs); the same seed always gives the same bytes."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty(n, dtype=torch.float64, device=device)
    out.uniform_(lo, hi, generator=g)
    return out


def device_normal(n: int, seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty(n, dtype=torch.float64, device=device)
    out.normal_(0.0, 1.0, generator=g)
    return out
