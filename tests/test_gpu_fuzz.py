"""Seeded random cases through the C ABI against the oracle: random dominant Toeplitz matrices
(mixed signs, one-sided, near-equality dominance), sizes from 2 to 1.6e6, every precision form,
window width, block size and flag, series of right-hand sides with padded rows, and batches of
random systems.  The bar is 1e-12 norm-wise against the FP64 oracle; where
the FP64 oracle itself is that far from the binary128 oracle (ill-conditioned draws), the GPU
result must stay within 20 times the FP64 oracle's own error from binary128."""
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


def check(t, F, x):
    e = rel(x, oracle.thomas(t, F))
    if e <= TOL:
        return
    xq = oracle.thomas_q(t, F)
    e_oracle = rel(oracle.thomas(t, F), xq)
    assert rel(x, xq) <= max(TOL, 20 * e_oracle), (t, F.size, e, e_oracle)


def draw_t(rng):
    a, c = rng.uniform(0.05, 1.5) * rng.choice([-1, 1]), rng.uniform(0.05, 1.5) * rng.choice([-1, 1])
    u = rng.uniform()
    if u < 0.1:
        a = 0.0
    elif u < 0.2:
        c = 0.0
    margin = 10 ** rng.uniform(-4, 0.5)
    t0 = (abs(a) + abs(c)) * (1 + margin) * rng.choice([-1, 1])
    return (float(a), float(t0), float(c)), margin


@pytest.mark.parametrize("seed", range(100))
def test_fuzz_single_and_series(D, seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(8):
        t, margin = draw_t(rng)
        N = int(10 ** rng.uniform(0.31, 6.2))
        prec = int(rng.choice([0, 1, 2]))
        if prec == 1 and margin < 1e-2:
            prec = 2                       # forced MIXED only where its error bound is small
        threads = int(rng.choice([0, 64, 128, 256]))
        bs = int(rng.choice([0, 0, 2, 3, 5, 16, 33, 64, 200]))
        flags = int(rng.choice([0, 1, 2, 3]))
        M = int(rng.choice([1, 1, 2, 3]))
        scale = 10 ** rng.uniform(-5, 5)
        try:
            plan = D.Plan(*t, N, precision=prec, threads=threads, block_size=bs, flags=flags)
        except D.DichotomyError as err:   # a block size that leaves a last block of one row
            assert err.code == 1 and bs > 0
            continue
        if M == 1:
            F = rng.standard_normal(N) * scale
            x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
            assert plan.status() == 0
            check(t, F, x)
        else:
            pad = int(rng.integers(0, 9))
            buf = torch.from_numpy(rng.standard_normal((M, N + pad)) * scale).cuda()
            Fs = buf[:, :N]
            X = plan.solve_series(Fs, out=torch.empty((M, N + pad), dtype=torch.float64, device="cuda")[:, :N])
            assert plan.status() == 0
            Fh, Xh = Fs.cpu().numpy(), X.cpu().numpy()
            for k in range(M):
                check(t, Fh[k], Xh[k])


@pytest.mark.parametrize("seed", range(30))
def test_fuzz_batches(D, seed):
    rng = np.random.default_rng(2000 + seed)
    nsys = int(rng.integers(1, 60))
    N = np.array([int(rng.choice([0, 1, 2, 3])) if rng.uniform() < 0.15 else int(10 ** rng.uniform(0.5, 5.3))
                  for _ in range(nsys)], dtype=np.int64)
    ts = [draw_t(rng) for _ in range(nsys)]
    tm1 = np.array([t[0] for t, _ in ts])
    t0 = np.array([t[1] for t, _ in ts])
    tp1 = np.array([t[2] for t, _ in ts])
    prec = int(rng.choice([0, 2]))
    F = rng.standard_normal(int(N.sum()))
    b = D.Batch(N, tm1, t0, tp1, precision=prec)
    x = b.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert b.status() == 0
    off = np.concatenate([[0], np.cumsum(N)[:-1]])
    for s in range(nsys):
        o, n = int(off[s]), int(N[s])
        if n:
            check((tm1[s], t0[s], tp1[s]), F[o:o + n], x[o:o + n])


@pytest.mark.parametrize("seed", range(30))
def test_fuzz_general_matrices(D, seed):
    """Random general tridiagonal matrices (per-row dominance margins from 1e-4 to 3, random
    signs, zero off-diagonals), both preliminary steps, every width and path flag."""
    rng = np.random.default_rng(3000 + seed)
    for _ in range(4):
        N = int(10 ** rng.uniform(0.31, 6.0))
        a = rng.uniform(-1, 1, N) * (rng.uniform(size=N) > 0.05)
        c = rng.uniform(-1, 1, N) * (rng.uniform(size=N) > 0.05)
        margin = 10 ** rng.uniform(-4, 0.5, N)
        b = (np.abs(a) + np.abs(c)) * (1 + margin) + 1e-3 * (np.abs(a) + np.abs(c) == 0)
        b *= rng.choice([-1.0, 1.0], N)
        flags = int(rng.choice([4, 8])) | int(rng.choice([0, 1]))
        threads = int(rng.choice([0, 64, 128, 256]))
        plan = D.GenPlan(a, b, c, threads=threads, flags=flags)
        F = rng.standard_normal(N)
        x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
        assert plan.status() == 0
        ref = oracle.thomas_tridiag(a, b, c, F)
        assert rel(x, ref) < 1e-11, (N, flags, plan.info)


@pytest.mark.parametrize("seed", range(20))
def test_fuzz_quasi_toeplitz(D, seed):
    """Random quasi-Toeplitz matrices (eq. 21): corner entries t_0 + psi, t_0 + chi kept dominant."""
    rng = np.random.default_rng(4000 + seed)
    for _ in range(4):
        t, margin = draw_t(rng)
        N = int(10 ** rng.uniform(0.31, 6.0))
        s0 = np.sign(t[1])
        # |t_0 + psi| >= |t_1| and |t_0 + chi| >= |t_-1| with a margin
        psi = s0 * (abs(t[2]) * (1 + rng.uniform(0.01, 1)) - abs(t[1])) * rng.uniform(0, 0.9)
        chi = s0 * (abs(t[0]) * (1 + rng.uniform(0.01, 1)) - abs(t[1])) * rng.uniform(0, 0.9)
        prec = int(rng.choice([0, 2]))
        try:
            plan = D.Plan(*t, N, psi=psi, chi=chi, precision=prec)
        except D.DichotomyError as err:   # a corner system that is singular or loses dominance
            assert err.code in (2, 3)
            continue
        F = rng.standard_normal(N)
        x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
        assert plan.status() == 0
        assert rel(x, oracle.thomas_quasi(t, psi, chi, F)) < TOL, (t, psi, chi, N, plan.info)
