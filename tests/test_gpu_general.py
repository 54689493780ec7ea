"""General (non-Toeplitz) tridiagonal systems (Sec. 2, the general preliminary step): the CUDA
path through dichotomy_gen_* against the oracle's Thomas solve of the same matrix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_2469_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dominant(N, seed, margin=(0.3, 1.5)):
    rng = np.random.default_rng(seed)
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = (np.abs(a) + np.abs(c) + rng.uniform(*margin, N)) * rng.choice([-1.0, 1.0], N)
    return a, b, c


def gen_solve(D, a, b, c, F, **kw):
    plan = D.GenPlan(a, b, c, **kw)
    x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert plan.status() == 0
    return x, plan.info


@pytest.mark.parametrize("N", [1, 2, 3, 5, 31, 1000, 4097, 100003, 1 << 20])
def test_general_random_dominant(D, N):
    a, b, c = dominant(N, N)
    F = np.random.default_rng(N + 1).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F)
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("bs", [2, 3, 16, 45])
@pytest.mark.parametrize("flags", [0, 1])
def test_general_geometry_and_paths(D, threads, bs, flags):
    N = 77777
    a, b, c = dominant(N, 5)
    F = np.random.default_rng(6).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F, threads=threads, block_size=bs, flags=flags)
    if flags:
        assert info["path"] == 2
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


def test_general_weak_dominance_takes_the_general_path(D):
    N = 300001
    a, b, c = dominant(N, 7, margin=(1e-3, 1e-2))
    F = np.random.default_rng(8).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F)
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


def test_general_with_constant_rows_equals_the_toeplitz_solve(D):
    N = 200000
    t = (-1.2, 2.5, -0.8)
    F = np.random.default_rng(9).standard_normal(N)
    xg, _ = gen_solve(D, np.full(N, t[0]), np.full(N, t[1]), np.full(N, t[2]), F)
    xt = D.Plan(*t, N, precision=D.PREC_F64).solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert rel(xg, xt) < 1e-14


def test_general_series(D):
    N, M = 5000, 4
    a, b, c = dominant(N, 10)
    F = np.random.default_rng(11).standard_normal((M, N))
    plan = D.GenPlan(a, b, c)
    X = plan.solve_series(torch.from_numpy(F).cuda()).cpu().numpy()
    assert plan.status() == 0
    for k in range(M):
        assert rel(X[k], oracle.thomas_tridiag(a, b, c, F[k])) < TOL
