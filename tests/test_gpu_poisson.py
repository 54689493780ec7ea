"""The 2-D Dirichlet Poisson driver (separation of variables, Sec. 3.2 and Sec. 4): DST-I along x,
the batch of mode systems through the Dichotomy kernels, inverse DST-I; against the oracle's
pipeline (scipy DST + Thomas per mode) and against manufactured solutions."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import poisson as OP  # noqa: E402


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_2469_gb300 import poisson
    return poisson


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_dst1_matches_scipy_and_is_involutory(P):
    import scipy.fft
    a = np.random.default_rng(0).standard_normal((37, 29))
    for dim in (0, 1):
        x = P.dst1(torch.from_numpy(a).cuda(), dim).cpu().numpy()
        assert rel(x, scipy.fft.dst(a, type=1, norm="ortho", axis=dim)) < 1e-14
    back = P.dst1(P.dst1(torch.from_numpy(a).cuda(), 0), 0).cpu().numpy()
    assert rel(back, a) < 1e-14


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("M", [1, 2, 31, 255])
def test_poisson2d_matches_oracle_pipeline(P, M, prec):
    f = np.random.default_rng(M).standard_normal((M, M))
    solver = P.Poisson2D(M, precision=prec)
    u = solver.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert solver.status() == 0
    # both pipelines are FP64; the lowest mode's conditioning (~0.4 (M + 1)^2) amplifies the
    # rounding of the two DST implementations
    assert rel(u, OP.poisson2d(f)) < max(1e-13, 4e-16 * 0.4 * (M + 1) ** 2 * 10)


@pytest.mark.parametrize("p,q", [(1, 1), (7, 3)])
def test_poisson2d_single_mode(P, p, q):
    M = 511
    h = 1.0 / (M + 1)
    x = np.arange(1, M + 1) * h
    f = np.outer(np.sin(p * math.pi * x), np.sin(q * math.pi * x))
    lam = (4 * math.sin(p * math.pi * h / 2) ** 2 + 4 * math.sin(q * math.pi * h / 2) ** 2) / h ** 2
    u = P.Poisson2D(M).solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert rel(u, f / lam) < 1e-12


def test_poisson2d_manufactured(P):
    M = 1023
    us = np.random.default_rng(1).uniform(-1, 1, (M, M))
    f = OP.laplacian5(us)
    u = P.Poisson2D(M).solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert rel(u, us) < 1e-9        # kappa ~ 0.4 (M + 1)^2 = 4e5 times the FP64 unit roundoff


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("M,My", [(1, 2), (31, 17), (255, 300)])
def test_poisson2d_neumann_y_matches_oracle_pipeline(P, M, My, prec):
    """Neumann in y: every mode a quasi-Toeplitz system (eq. 21) in one batch."""
    f = np.random.default_rng(M + My).standard_normal((M, My))
    solver = P.Poisson2D(M, precision=prec, My=My, bc_y="neumann")
    u = solver.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert solver.status() == 0
    assert rel(u, OP.poisson2d_neumann_y(f)) < max(1e-13, 4e-16 * 0.4 * max(M + 1, My) ** 2 * 10)
    assert rel(OP.laplacian5_neumann_y(u), f) < 1e-9


def test_poisson2d_neumann_y_manufactured(P):
    M, My = 511, 400
    us = np.random.default_rng(2).uniform(-1, 1, (M, My))
    f = OP.laplacian5_neumann_y(us)
    u = P.Poisson2D(M, My=My, bc_y="neumann").solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert rel(u, us) < 1e-10
