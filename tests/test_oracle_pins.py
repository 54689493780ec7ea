"""Pins for the CPU oracle: it is checked against things other than itself.

* dense LU of an independently built matrix (numpy.linalg.solve),
* exact rational solutions (golden fixtures written by tests/golden/make_golden.py),
* closed forms: eigenpairs of Toeplitz tridiagonals, Theorem 1 (eq. 20, with the sign
  reading), the Chebyshev forms eq. 24-25,
* the paper's own identities: eq. 15 (first/last values from beta and Z) for any block
  partition, the level process eq. 17-19, P-invariance (Sec. 5), the maximum principle
  |Z| <= 1 under diagonal dominance (Sec. 3.4),
* adjoint identities: <w, T^-1 F> = <T^-T w, F>, central finite differences, the
  eigenvector closed form,
* planted mistakes: each of six mutated builds of oracle.c fails at least one pin.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle.exact import residual_exact, solve_exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

T_CASES = [
    (-1.0, 4.0, -1.0),        # symmetric, strongly dominant
    (-1.2, 2.5, -0.8),        # non-symmetric
    (-0.8, 2.5, -1.2),        # its transpose
    (-1.0, 2.001, -1.0),      # weakly dominant
    (0.7, 2.5, -1.1),         # off-diagonals of opposite sign
    (-1.2, 2.0, -0.8),        # dominance with equality (a root on the unit circle)
    (-1.0, 2.0, -1.0),        # the 1-D Laplacian (double root)
    (0.0, 2.0, -1.0),         # upper bidiagonal
    (-1.0, 2.0, 0.0),         # lower bidiagonal
]


def dense(t, N):
    tm1, t0, tp1 = t
    A = np.diag(np.full(N, float(t0)))
    if N > 1:
        A += np.diag(np.full(N - 1, float(tm1)), -1) + np.diag(np.full(N - 1, float(tp1)), 1)
    return A


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("t", T_CASES)
@pytest.mark.parametrize("N", [1, 2, 3, 5, 17, 64, 257, 512])
def test_thomas_vs_dense_lu(t, N):
    rng = np.random.default_rng(N)
    F = rng.uniform(-1, 1, N)
    ref = np.linalg.solve(dense(t, N), F)
    kappa = np.linalg.cond(dense(t, N), np.inf)
    tol = max(1e-14, 4 * kappa * 2.2e-16)
    assert rel(oracle.thomas(t, F), ref) < tol
    assert rel(oracle.thomas_q(t, F), ref) < tol


def test_thomas_matches_matvec_residual_row_convention():
    # row i reads t_-1 x[i-1] + t_0 x[i] + t_1 x[i+1]: checked by an explicit residual loop
    t = (-1.2, 2.5, -0.8)
    rng = np.random.default_rng(5)
    F = rng.standard_normal(40)
    x = oracle.thomas(t, F)
    for i in range(40):
        v = t[1] * x[i] + (t[0] * x[i - 1] if i > 0 else 0) + (t[2] * x[i + 1] if i < 39 else 0)
        assert abs(v - F[i]) < 1e-14


def _golden_cases():
    out = []
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".txt"):
            continue
        rows = {}
        with open(os.path.join(GOLDEN, name)) as fh:
            for line in fh:
                if line.startswith("#") or not line.strip():
                    continue
                key, *vals = line.split()
                rows[key] = np.array([float.fromhex(v) for v in vals])
        out.append((name, tuple(rows["t"]), rows["F"], rows["x"]))
    return out


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_golden_exact_solutions(case):
    _, t, F, x_exact = case
    # binary128 Thomas rounds to the exact solution within one FP64 ulp
    xq = oracle.thomas_q(t, F)
    ulp = np.spacing(np.abs(x_exact))
    assert np.all(np.abs(xq - x_exact) <= ulp)
    kappa = np.linalg.cond(dense(t, F.size), np.inf)
    assert rel(oracle.thomas(t, F), x_exact) < max(1e-15, 8 * kappa * 1.1e-16)


def test_exact_solver_residual_is_zero():
    rng = np.random.default_rng(3)
    for t in T_CASES:
        F = rng.uniform(-1, 1, 9)
        x = solve_exact(t, F)
        assert all(r == 0 for r in residual_exact(t, x, F))


@pytest.mark.parametrize("t", [(-1.0, 4.0, -1.0), (-1.2, 2.5, -0.8), (-0.5, 3.0, -2.0), (1.0, 3.0, 1.5)])
@pytest.mark.parametrize("N", [7, 100, 1000])
def test_eigenpairs(t, N):
    for k in (1, 2, N // 2, N):
        lam, v = cf.eigenpair(N, t, k)
        # the closed form is an eigenpair of the dense matrix ...
        assert rel(dense(t, N) @ v, lam * v) < 1e-12 if N <= 1000 else True
        # ... and the oracle solves T x = v_k with x = v_k / lambda_k
        assert rel(oracle.thomas(t, v), v / lam) < 1e-12


def test_manufactured_solution_large():
    t = (-1.2, 2.5, -0.8)
    N = 1 << 20
    rng = np.random.default_rng(0)
    xs = rng.uniform(-1, 1, N)
    F = t[1] * xs
    F[1:] += t[0] * xs[:-1]
    F[:-1] += t[2] * xs[1:]
    assert rel(oracle.thomas(t, F), xs) < 1e-14
    assert rel(oracle.thomas_q(t, F), xs) < 1e-15


@pytest.mark.parametrize("t", [(-1.2, 2.5, -0.8), (-1.0, 4.0, -1.0), (0.7, 2.5, -1.1)])
@pytest.mark.parametrize("N", [9, 10, 11, 12])
def test_theorem1_sign_reading(t, N):
    """Theorem 1 (eq. 20) reproduces T^-1 with the factor -1/t_1; as printed (+1/t_1) it does not."""
    inv = np.linalg.inv(dense(t, N))
    assert rel(cf.theorem1_inverse(N, t, sign=-1.0), inv) < 1e-12
    assert rel(cf.theorem1_inverse(N, t, sign=+1.0), inv) > 0.5
    # and the oracle's Green rows (eq. 9) are rows of that inverse
    starts = np.array([0, 3, 6])
    GL, GR, _, _ = oracle.dich_prelim(t, N, starts)
    th = cf.theorem1_inverse(N, t, sign=-1.0)
    for m, s in enumerate(starts):
        e = (starts[m + 1] - 1) if m + 1 < len(starts) else N - 1
        assert rel(GL[m], th[s]) < 1e-12
        assert rel(GR[m], th[e]) < 1e-12


@pytest.mark.parametrize("x", [1.05, 1.5, 3.0, 0.9])
def test_chebyshev_forms_eq24_25(x):
    """Z (eq. 24) and G (eq. 25) of tridiag{-1, 2x, -1} (N intervals, N-1 unknowns)."""
    N = 24
    M = N - 1
    t = (-1.0, 2.0 * x, -1.0)
    starts = np.array([0, 5, 11, 17])         # 0-based block starts over the M unknowns
    GL, GR, ZL, ZR = oracle.dich_prelim(t, M, starts)
    for m, s in enumerate(starts):
        e = (starts[m + 1] - 1) if m + 1 < len(starts) else M - 1
        zl, zr, gl, gr = cf.laplace_prelim(N, x, s + 1, e + 1)   # 1-based
        assert rel(ZL[m][: s + 1], zl[: s + 1]) < 1e-12
        assert rel(ZR[m][e:], zr[e:]) < 1e-12
        assert rel(GL[m][s:e + 1], gl[s:e + 1]) < 1e-12
        assert rel(GR[m][s:e + 1], gr[s:e + 1]) < 1e-12


def _random_partition(rng, N, P):
    """P blocks of random sizes >= 2 summing to N."""
    extra = rng.multinomial(N - 2 * P, np.ones(P) / P)
    sizes = 2 + extra
    return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)


@pytest.mark.parametrize("t", T_CASES[:6])
def test_eq15_first_last_values_exact(t):
    rng = np.random.default_rng(1)
    N = 120
    F = rng.uniform(-1, 1, N)
    x_ref = oracle.thomas_q(t, F)
    kappa = np.linalg.cond(dense(t, N), np.inf)
    tol = max(1e-13, 10 * kappa * 1.1e-16)
    n_tried = 0
    for P in (1, 2, 3, 7, 16, 40):
        starts = _random_partition(rng, N, P)
        out = oracle.dich_eq15(t, F, starts)
        ends = np.append(starts[1:] - 1, N - 1)
        assert rel(out["x_first"], x_ref[starts]) < tol
        assert rel(out["x_last"], x_ref[ends]) < tol
        assert rel(out["x"], x_ref) < tol
        n_tried += 1
    assert n_tried == 6


@pytest.mark.parametrize("t", T_CASES[:6])
@pytest.mark.parametrize("P", [1, 2, 3, 5, 8, 13, 30])
def test_levels_eq17_19(t, P):
    rng = np.random.default_rng(P)
    N = 90
    F = rng.standard_normal(N)
    starts = oracle.even_starts(N, N // P)
    x, levels = oracle.dich_levels(t, F, starts)
    x_ref = oracle.thomas_q(t, F)
    kappa = np.linalg.cond(dense(t, N), np.inf)
    assert rel(x, x_ref) < max(1e-13, 10 * kappa * 1.1e-16)
    assert levels == math.ceil(math.log2(starts.size + 1))


def test_p_invariance():
    """The result does not depend on the number of blocks (Sec. 5)."""
    t = (-1.2, 2.5, -0.8)
    rng = np.random.default_rng(9)
    N = 200
    F = rng.standard_normal(N)
    xs = [oracle.dich_eq15(t, F, oracle.even_starts(N, n))["x"] for n in (2, 3, 7, 25, 100, 200)]
    for x in xs[1:]:
        assert rel(x, xs[0]) < 1e-14


def test_max_principle_Z():
    """|Z| <= 1 when dominant (Sec. 3.4); for lambda > 0 in eq. 22 (no dominance) |Z| exceeds 1."""
    N = 64
    starts = np.array([0, 16, 32, 48])
    for t in [(-1.0, 2.001, -1.0), (-1.2, 2.5, -0.8), (0.7, 2.5, -1.1), (-1.0, 2.0, -1.0)]:
        _, _, ZL, ZR = oracle.dich_prelim(t, N, starts)
        assert np.max(np.abs(ZL)) <= 1 + 1e-14 and np.max(np.abs(ZR)) <= 1 + 1e-14
    # eq. 22 with h^2 lambda = 0.01 > 0: x = 1 - h^2 lambda / 2 < 1
    _, _, ZL, ZR = oracle.dich_prelim((-1.0, 1.99, -1.0), N, starts)
    assert max(np.max(np.abs(ZL)), np.max(np.abs(ZR))) > 1.5


@pytest.mark.parametrize("t", [(-1.2, 2.5, -0.8), (0.7, 2.5, -1.1), (-1.0, 4.0, -1.0)])
def test_adjoint_identities(t):
    rng = np.random.default_rng(2)
    N = 300
    F = rng.uniform(-1, 1, N)
    w = rng.uniform(-1, 1, N)
    x = oracle.thomas(t, F)
    lam, gt = oracle.adjoint(t, w, x)
    # <w, T^-1 F> = <T^-T w, F>
    assert abs(np.dot(w, x) - np.dot(lam, F)) < 1e-13 * np.sum(np.abs(w * x))
    # lambda solves the transposed dense system
    assert rel(lam, np.linalg.solve(dense(t, N).T, w)) < 1e-13
    # central finite differences in each coefficient (h = 1e-6)
    h = 1e-6
    for k in range(3):
        tp = list(t); tm = list(t)
        tp[k] += h; tm[k] -= h
        fd = (np.dot(w, oracle.thomas(tp, F)) - np.dot(w, oracle.thomas(tm, F))) / (2 * h)
        assert abs(fd - gt[k]) <= 1e-6 * max(1.0, abs(gt[k]))


def test_adjoint_eigen_closed_form():
    """F = w = v_k of a symmetric T: x = v_k / lambda_k and dL/dt_0 = -<v_k, v_k> / lambda_k^2."""
    N, k = 200, 3
    t = (-1.0, 2.5, -1.0)
    lam_k, v = cf.eigenpair(N, t, k)
    x = oracle.thomas(t, v)
    _, gt = oracle.adjoint(t, v, x)
    assert abs(gt[1] + np.dot(v, v) / lam_k ** 2) < 1e-12 * np.dot(v, v) / lam_k ** 2


def test_batched_equals_single():
    rng = np.random.default_rng(4)
    Ns = np.array([2, 5, 64, 1000, 3])
    off = np.concatenate([[0], np.cumsum(Ns)[:-1]])
    tm1 = rng.uniform(-1, -0.5, Ns.size)
    tp1 = rng.uniform(-1, -0.5, Ns.size)
    t0 = rng.uniform(2.05, 4, Ns.size)
    F = rng.uniform(-1, 1, Ns.sum())
    x = oracle.thomas_batched(tm1, t0, tp1, Ns, off, F, nthreads=3)
    for s in range(Ns.size):
        sl = slice(off[s], off[s] + Ns[s])
        np.testing.assert_array_equal(x[sl], oracle.thomas((tm1[s], t0[s], tp1[s]), F[sl]))


def test_planted_mistakes_are_caught(tmp_path):
    """Each planted mistake in oracle.c (transposed operand, dropped term, stale pivot,
    wrong sign, T instead of T^T, shift the wrong way) fails at least one pin above."""
    t = (-1.2, 2.5, -0.8)
    N = 50
    rng = np.random.default_rng(8)
    F = rng.uniform(-1, 1, N)
    w = rng.uniform(-1, 1, N)
    ref = np.linalg.solve(dense(t, N), F)
    ref_lam = np.linalg.solve(dense(t, N).T, w)

    def pins_fail(v):
        x = v.thomas(t, F)
        if rel(x, ref) > 1e-12:
            return True
        lam, gt = v.adjoint(t, w, x)
        if rel(lam, ref_lam) > 1e-12:
            return True
        h = 1e-6
        for k in range(3):
            tp = list(t); tm = list(t)
            tp[k] += h; tm[k] -= h
            fd = (np.dot(w, v.thomas(tp, F)) - np.dot(w, v.thomas(tm, F))) / (2 * h)
            if abs(fd - gt[k]) > 1e-6 * max(1.0, abs(gt[k])):
                return True
        return False

    assert not pins_fail(oracle.build_variant(0, str(tmp_path)))
    for k in range(1, 7):
        assert pins_fail(oracle.build_variant(k, str(tmp_path))), f"mutant {k} slipped through"


# ------------------------------------------------------------------ general and quasi-Toeplitz (eq. 21)
@pytest.mark.parametrize("N", [1, 2, 3, 17, 300])
def test_tridiag_vs_dense_lu(N):
    """The general Thomas solve against numpy's dense LU of the same matrix, built row by row."""
    rng = np.random.default_rng(N)
    sub, sup = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    dia = (np.abs(sub) + np.abs(sup) + rng.uniform(0.1, 2.0, N)) * rng.choice([-1.0, 1.0], N)
    A = np.zeros((N, N))
    for i in range(N):
        A[i, i] = dia[i]
        if i > 0:
            A[i, i - 1] = sub[i]
        if i < N - 1:
            A[i, i + 1] = sup[i]
    F = rng.standard_normal(N)
    assert rel(oracle.thomas_tridiag(sub, dia, sup, F), np.linalg.solve(A, F)) < 1e-14


def test_tridiag_constant_arrays_equal_toeplitz():
    t = (-1.2, 2.5, -0.8)
    F = np.random.default_rng(1).standard_normal(5000)
    n = F.size
    x = oracle.thomas_tridiag(np.full(n, t[0]), np.full(n, t[1]), np.full(n, t[2]), F)
    assert np.array_equal(x, oracle.thomas(t, F))
    assert np.array_equal(oracle.thomas_quasi(t, 0.0, 0.0, F), oracle.thomas(t, F))


@pytest.mark.parametrize("t,psi,chi", [((-1.0, 2.5, -1.0), -1.0, -1.0),     # Neumann-type rows [1.5, -1]
                                       ((-1.2, 2.5, -0.8), 0.7, -0.3),
                                       ((-1.0, 4.0, -1.0), 2.0, 0.0),
                                       ((0.7, 2.5, -1.1), -0.5, 1.5)])
def test_quasi_toeplitz_eq21_vs_dense(t, psi, chi):
    """eq. 21: the Toeplitz matrix with t_0 + psi in the first and t_0 + chi in the last row."""
    N = 64
    A = np.diag(np.full(N, t[1])) + np.diag(np.full(N - 1, t[0]), -1) + np.diag(np.full(N - 1, t[2]), 1)
    A[0, 0] = t[1] + psi
    A[N - 1, N - 1] = t[1] + chi
    F = np.random.default_rng(2).standard_normal(N)
    assert rel(oracle.thomas_quasi(t, psi, chi, F), np.linalg.solve(A, F)) < 1e-14


@pytest.mark.parametrize("t,psi,chi", [((-1.0, 2.5, -1.0), -1.0, -1.0), ((0.7, 2.5, -1.1), -0.5, 1.5),
                                       ((-1.2, 2.5, -0.8), 0.0, 0.9)])
def test_quasi_adjoint_vs_dense_and_finite_differences(t, psi, chi):
    """The quasi-Toeplitz adjoint: lambda against a dense solve with A^T, the five gradients
    against central finite differences of L = <w, A(t, psi, chi)^-1 F> with dense solves."""
    N = 40
    rng = np.random.default_rng(3)
    F, w = rng.standard_normal(N), rng.standard_normal(N)

    def dense(p):
        tm1, t0, tp1, ps, ch = p
        A = np.diag(np.full(N, t0)) + np.diag(np.full(N - 1, tm1), -1) + np.diag(np.full(N - 1, tp1), 1)
        A[0, 0] += ps
        A[N - 1, N - 1] += ch
        return A

    p0 = np.array([t[0], t[1], t[2], psi, chi])
    x = np.linalg.solve(dense(p0), F)
    lam, g = oracle.adjoint_quasi(t, psi, chi, w, x)
    assert rel(lam, np.linalg.solve(dense(p0).T, w)) < 1e-13
    assert abs(np.dot(w, x) - np.dot(lam, F)) < 1e-12 * np.abs(w).sum() * np.abs(x).max()
    h = 1e-6
    for k in range(5):
        dp = np.zeros(5)
        dp[k] = h
        fd = (np.dot(w, np.linalg.solve(dense(p0 + dp), F)) - np.dot(w, np.linalg.solve(dense(p0 - dp), F))) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


# ------------------------------------------------------------------ 2-D Poisson by separation of variables
def test_poisson2d_oracle_vs_dense_kronecker():
    """The separation-of-variables oracle against a dense solve of the five-point Laplacian,
    assembled independently as a Kronecker sum."""
    from oracle import poisson as OP
    M = 15
    h = 1.0 / (M + 1)
    T = (np.diag(np.full(M, 2.0)) - np.diag(np.ones(M - 1), 1) - np.diag(np.ones(M - 1), -1)) / (h * h)
    L = np.kron(T, np.eye(M)) + np.kron(np.eye(M), T)          # row-major [i, j] -> i * M + j
    f = np.random.default_rng(4).standard_normal((M, M))
    u = np.linalg.solve(L, f.reshape(-1)).reshape(M, M)
    assert rel(OP.poisson2d(f), u) < 1e-13
    assert rel(OP.laplacian5(u), f) < 1e-12


def test_poisson2d_neumann_y_vs_dense_kronecker():
    """Dirichlet in x, Neumann in y (cell-centred): the separation-of-variables oracle (modes solved
    as quasi-Toeplitz systems, eq. 21) against a dense solve of the Kronecker sum of the two 1-D
    operators, the y one assembled with its Neumann end rows [1, -1] / hy^2."""
    from oracle import poisson as OP
    M, My = 11, 7
    hx, hy = 1.0 / (M + 1), 1.0 / My
    Tx = (np.diag(np.full(M, 2.0)) - np.diag(np.ones(M - 1), 1) - np.diag(np.ones(M - 1), -1)) / (hx * hx)
    Ty = np.diag(np.full(My, 2.0)) - np.diag(np.ones(My - 1), 1) - np.diag(np.ones(My - 1), -1)
    Ty[0, 0] = Ty[-1, -1] = 1.0
    Ty /= hy * hy
    L = np.kron(Tx, np.eye(My)) + np.kron(np.eye(M), Ty)        # row-major [i, j] -> i * My + j
    f = np.random.default_rng(5).standard_normal((M, My))
    u = np.linalg.solve(L, f.reshape(-1)).reshape(M, My)
    assert rel(OP.poisson2d_neumann_y(f), u) < 1e-13
    assert rel(OP.laplacian5_neumann_y(u), f) < 1e-12


def test_poisson2d_neumann_y_second_order():
    """u = sin(pi x) cos(pi y) solves -Laplace u = 2 pi^2 u with u = 0 at x = 0, 1 and du/dy = 0 at
    y = 0, 1: the discrete solution converges to it at second order."""
    from oracle import poisson as OP
    errs = []
    for M in (15, 31, 63):
        My = M + 1
        x = np.arange(1, M + 1) / (M + 1)
        y = (np.arange(My) + 0.5) / My
        us = np.outer(np.sin(math.pi * x), np.cos(math.pi * y))
        errs.append(np.max(np.abs(OP.poisson2d_neumann_y(2 * math.pi ** 2 * us) - us)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


@pytest.mark.parametrize("p,q", [(1, 1), (3, 5), (20, 2)])
def test_poisson2d_single_mode(p, q):
    """f = sin(p pi x) sin(q pi y) excites one mode: u = f / lambda_pq, lambda_pq =
    (4 sin^2(p pi h / 2) + 4 sin^2(q pi h / 2)) / h^2 (the discrete eigenvalue)."""
    from oracle import poisson as OP
    M = 63
    h = 1.0 / (M + 1)
    x = np.arange(1, M + 1) * h
    f = np.outer(np.sin(p * math.pi * x), np.sin(q * math.pi * x))
    lam = (4 * math.sin(p * math.pi * h / 2) ** 2 + 4 * math.sin(q * math.pi * h / 2) ** 2) / h ** 2
    assert rel(OP.poisson2d(f), f / lam) < 1e-13
