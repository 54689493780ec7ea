"""The 2-D Dirichlet Poisson problem by separation of variables (Sec. 3.2 and Sec. 4).

-Laplace(u) = f on the unit square, u = 0 on the boundary, five-point stencil on a grid of
(M + 1) x (M + 1) intervals (h = 1 / (M + 1)), unknowns u[i, j] = u(x_i, y_j), i, j = 1..M, stored
as an [M, M] tensor (row i = x_i).  The orthonormal DST-I along x diagonalises the x part of the
operator; mode k = 1..M leaves one tridiagonal Toeplitz system along y,

    -v[k, j-1] + (2 + 4 sin^2(k pi / (2 (M + 1)))) v[k, j] - v[k, j+1] = h^2 fhat[k, j],

the series of Sec. 3.2 with one t_0 per mode.  All M systems are solved as one batch by the
Dichotomy kernels (the library's batched entry point); the inverse DST-I (the same transform)
returns u.  The transforms use torch's FFT (cuFFT): DST-I of length M through a real FFT of
length 2 (M + 1).

Neumann conditions in y (bc_y="neumann"): My cell-centred unknowns y_j = (j + 1/2) / My with
du/dy = 0 at y = 0 and y = 1 (ghost cells equal to their neighbours).  Mode k then leaves the
quasi-Toeplitz system of eq. 21 (Sec. 3.1), tridiag{-1, t_0(k), -1} with
t_0(k) = 2 + (hy / hx)^2 4 sin^2(k pi / (2 (M + 1))) and psi = chi = -1 in its first and last
rows, right-hand side hy^2 fhat_k; the batch's corner step handles the two rows.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import dichotomy as _d

__all__ = ["dst1", "mode_t0", "Poisson2D"]


def dst1(a: torch.Tensor, dim: int = 0) -> torch.Tensor:
    """Orthonormal DST-I along `dim`: X_k = sqrt(2 / (M + 1)) sum_j a_j sin(pi j k / (M + 1)),
    j, k = 1..M.  It is its own inverse.  One real FFT of length N = M + 1 (half the padded
    length): with a_0 = a_N = 0, y_j = sin(pi j / N) (a_j + a_{N-j}) + (a_j - a_{N-j}) / 2 has
    C_k - i S_k = sum_j y_j exp(-2 pi i j k / N) with S_k = X_{2k} (the antisymmetric part) and
    C_k = X_{2k+1} - X_{2k-1} (the symmetric part, by the product-to-sum identity), so the odd
    outputs are the running sums X_{2k+1} = C_0 / 2 + C_1 + ... + C_k."""
    x = a.movedim(dim, -1)
    M = x.shape[-1]
    N = M + 1
    z = torch.zeros(x.shape[:-1] + (1,), dtype=x.dtype, device=x.device)
    xp = torch.cat([z, x], dim=-1)                       # a_j, j = 0..N-1
    xr = torch.cat([z, x.flip(-1)], dim=-1)              # a_{N-j}
    s = torch.sin(torch.arange(N, dtype=x.dtype, device=x.device) * (math.pi / N))
    y = s * (xp + xr) + 0.5 * (xp - xr)
    Y = torch.fft.rfft(y, dim=-1)
    out = torch.empty_like(x)
    out[..., 1::2] = -Y.imag[..., 1:1 + M // 2]            # X_{2m}, m = 1..M/2
    C = Y.real
    odd = torch.cumsum(C, dim=-1) - 0.5 * C[..., :1]       # X_{2m+1}, m = 0..(M-1)/2
    out[..., 0::2] = odd[..., :(M + 1) // 2]
    return (out * math.sqrt(2.0 / N)).movedim(-1, dim).contiguous()


def mode_t0(M: int) -> np.ndarray:
    """t_0 of the tridiagonal system of mode k = 1..M: 2 + 4 sin^2(k pi / (2 (M + 1)))."""
    k = np.arange(1, M + 1, dtype=np.float64)
    return 2.0 + 4.0 * np.sin(k * math.pi / (2.0 * (M + 1))) ** 2


class Poisson2D:
    """Solver for an [M, My] grid (My = M by default): Dirichlet in x; Dirichlet (My interior
    nodes, hy = 1 / (My + 1)) or Neumann (My cell centres, hy = 1 / My) in y.  The batch of M
    mode systems is planned once."""

    def __init__(self, M: int, precision: int = _d.PREC_AUTO, device=None, My: int | None = None,
                 bc_y: str = "dirichlet"):
        self.M = int(M)
        self.My = int(My) if My is not None else self.M
        if bc_y not in ("dirichlet", "neumann"):
            raise ValueError("bc_y must be 'dirichlet' or 'neumann'")
        self.bc_y = bc_y
        self.hx = 1.0 / (self.M + 1)
        self.hy = 1.0 / (self.My + 1) if bc_y == "dirichlet" else 1.0 / self.My
        self.h = self.hy
        k = np.arange(1, self.M + 1, dtype=np.float64)
        t0 = 2.0 + (self.hy / self.hx) ** 2 * 4.0 * np.sin(k * math.pi / (2.0 * (self.M + 1))) ** 2
        ones = np.ones(self.M)
        corners = dict(psi=-ones, chi=-ones) if bc_y == "neumann" else {}
        self.batch = _d.Batch(np.full(self.M, self.My, dtype=np.int64), -ones, t0, -ones, precision=precision,
                              **corners)
        self.device = device

    def solve(self, f: torch.Tensor) -> torch.Tensor:
        """u for the right-hand side f ([M, My], float64, CUDA)."""
        if f.shape != (self.M, self.My):
            raise ValueError(f"f must be [{self.M}, {self.My}]")
        rhs = (self.hy * self.hy) * dst1(f, dim=0)                # [k, j]: mode k along y
        v = self.batch.solve(rhs.reshape(-1)).reshape(self.M, self.My)
        return dst1(v, dim=0)

    def status(self) -> int:
        return self.batch.status()
