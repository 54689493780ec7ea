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
    assert plan.info["precision"] in (0, 1)
    x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert plan.status() == 0
    return x, plan.info


HOST, DEVICE = 4, 8   # where the preliminary step runs (DICH_FLAG_HOST_PRELIM / _DEVICE_PRELIM)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("prelim", [HOST, DEVICE])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 31, 1000, 4097, 100003, 1 << 20])
def test_general_random_dominant(D, N, prelim, prec):
    a, b, c = dominant(N, N)
    F = np.random.default_rng(N + 1).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F, flags=prelim, precision=prec)
    if N > 1:
        assert info["precision"] == (1 if prec else 0)   # strongly dominant: AUTO takes MIXED
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("bs", [2, 3, 16, 45])
def test_general_mixed_geometry_and_paths(D, threads, bs, flags, prelim):
    N = 77777
    a, b, c = dominant(N, 15)
    F = np.random.default_rng(16).standard_normal(N) * 1e-7
    x, info = gen_solve(D, a, b, c, F, threads=threads, block_size=bs, flags=flags | prelim, precision=1)
    assert info["precision"] == 1 and (info["path"] == 2 or not flags)
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


def test_general_mixed_scaled_rows(D):
    """Rows scaled by powers of ten from 1e-9 to 1e9 (factors within 2^40): the window scale and
    the float-float factors keep 1e-12 norm-wise."""
    N = 200003
    a, b, c = dominant(N, 17)
    s = 10.0 ** np.random.default_rng(18).uniform(-9, 9, N)
    a, b, c = a * s, b * s, c * s
    F = np.random.default_rng(19).standard_normal(N) * s
    x, info = gen_solve(D, a, b, c, F, precision=1)
    assert info["precision"] == 1
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("kind", ["zeros", "wide", "1e250", "1e-250", "1e300"])
@pytest.mark.parametrize("flags", [0, 1])
def test_general_mixed_right_hand_side_ranges(D, kind, flags):
    """Tiles outside the fast split and join (exact zeros, 200 decades, the ends of the FP64
    range) take the general conversions; tiles inside take the fast ones; both forms of path."""
    N = 150001
    a, b, c = dominant(N, 21)
    rng = np.random.default_rng(22)
    F = rng.standard_normal(N)
    if kind == "zeros":
        F[rng.integers(0, N, 500)] = 0.0
        F[40000:45000] = 0.0
    elif kind == "wide":
        F *= 10.0 ** rng.uniform(-100, 100, N)
    else:
        F *= float(kind)
    x, info = gen_solve(D, a, b, c, F, precision=1, flags=flags)
    assert info["precision"] == 1 and (info["path"] == 2 or not flags)
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("bs", [2, 3, 16, 45])
@pytest.mark.parametrize("flags", [0, 1])
def test_general_geometry_and_paths(D, threads, bs, flags, prelim):
    N = 77777
    a, b, c = dominant(N, 5)
    F = np.random.default_rng(6).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F, threads=threads, block_size=bs, flags=flags | prelim)
    if flags:
        assert info["path"] == 2
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
def test_general_weak_dominance(D, prelim):
    N = 300001
    a, b, c = dominant(N, 7, margin=(1e-3, 1e-2))
    F = np.random.default_rng(8).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F, flags=prelim)
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
def test_general_slow_decay_takes_the_general_path(D, prelim):
    """Off-diagonals near -1 and a diagonal margin of 0.002..0.01: the coupling between blocks
    decays too slowly for halo windows, so the interface values come from the block scan."""
    N = 300001
    rng = np.random.default_rng(7)
    a, c = -rng.uniform(0.9, 1.0, N), -rng.uniform(0.9, 1.0, N)
    b = np.abs(a) + np.abs(c) + rng.uniform(2e-3, 1e-2, N)
    F = np.random.default_rng(8).standard_normal(N)
    x, info = gen_solve(D, a, b, c, F, flags=prelim)
    assert info["path"] == 2
    assert rel(x, oracle.thomas_tridiag(a, b, c, F)) < TOL, info


@pytest.mark.parametrize("N,bs", [(2, 0), (65, 3), (8192 * 32 + 77, 32), (3 * 8192 * 32 + 1, 32), (1 << 20, 0)])
def test_device_preliminary_matches_the_host_one(D, N, bs):
    """The device preliminary (block composites, chunked prefix and suffix products of 2x2
    elimination matrices) gives the same path and halos as the host's row-by-row pass and
    solutions equal to the last few ulps; sizes span one, several and a ragged last scan chunk
    of 256 blocks."""
    a, b, c = dominant(N, 12 + N)
    F = np.random.default_rng(13 + N).standard_normal(N)
    xh, ih = gen_solve(D, a, b, c, F, flags=HOST, block_size=bs)
    xd, idv = gen_solve(D, a, b, c, F, flags=DEVICE, block_size=bs)
    for k in ("path", "halo_l", "halo_r", "n", "P", "tiles"):
        assert ih[k] == idv[k], (k, ih, idv)
    assert rel(xd, xh) < 1e-13
    assert rel(xd, oracle.thomas_tridiag(a, b, c, F)) < TOL


@pytest.mark.parametrize("k", [None, 3210, 3231])
def test_device_preliminary_refuses_a_zero_pivot(D, k):
    """A weakly dominant matrix with an exactly singular 2x2 diagonal block [[1, 1], [1, 1]]
    (rows k, k+1; a_k = c_{k+1} = 0, so the determinant factorises): both preliminaries refuse it,
    the host one at plan time, the device one at bind time; k = 3231 puts the zero pivot on the
    first row of a block (the whole-system factor carried in from the block before)."""
    if k is None:
        a, b, c = np.array([0.0, 1.0]), np.array([1.0, 1.0]), np.array([1.0, 0.0])
        k = 0
    else:
        N = 100000
        a, b, c = dominant(N, 14)
        a[k], b[k], c[k] = 0.0, 1.0, 1.0
        a[k + 1], b[k + 1], c[k + 1] = 1.0, 1.0, 0.0
    bs = 32 if b.size > 2 else 0
    with pytest.raises(D.DichotomyError) as e:
        D.GenPlan(a, b, c, flags=HOST, block_size=bs)
    assert e.value.code == 3 and "dichotomy_gen_plan" in str(e.value)
    with pytest.raises(D.DichotomyError) as e:
        D.GenPlan(a, b, c, flags=DEVICE, block_size=bs)
    assert e.value.code == 3 and "dichotomy_gen_bind" in str(e.value)


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


def host_residual(a, b, c, F, x):
    """max |F - A x| and the norm-wise backward error, computed on the host (the definition)."""
    ax = b * x
    ax[1:] += a[1:] * x[:-1]
    ax[:-1] += c[:-1] * x[1:]
    r = np.max(np.abs(F - ax))
    nA = np.max(np.abs(np.r_[0.0, a[1:]]) + np.abs(b) + np.abs(np.r_[c[:-1], 0.0]))
    return r, r / (nA * np.max(np.abs(x)) + np.max(np.abs(F)))


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
def test_residual_check_on_dominant_matrices(D, prelim):
    N = 300001
    a, b, c = dominant(N, 21)
    F = np.random.default_rng(22).standard_normal(N)
    plan = D.GenPlan(a, b, c, flags=prelim)
    Fd = torch.from_numpy(F).cuda()
    xd = plan.solve(Fd)
    r, be = plan.residual(Fd, xd)
    rh, beh = host_residual(a, b, c, F, xd.cpu().numpy())
    # both residuals carry FP64 rounding of their own (different orders): agree to ~4 ulp of the scale
    assert abs(be - beh) <= 1e-15 + 1e-3 * beh and be < 1e-15 and plan.info["growth"] == 1.0


@pytest.mark.parametrize("prelim", [HOST, DEVICE])
@pytest.mark.parametrize("N", [5000, 300001])
def test_not_dominant_spd_matrices_with_a_posteriori_check(D, N, prelim):
    """Symmetric positive definite tridiagonal matrices A = L L^T (L lower bidiagonal) are mostly
    not diagonally dominant; with the dominance check waived the solve is compared with LAPACK's
    banded LU with partial pivoting (scipy) and judged by its own residual check (the a posteriori
    check recommended after eq. 33)."""
    linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(N + 23)
    d, e = rng.uniform(1.0, 2.0, N), rng.uniform(-1.0, 1.0, N)
    b = d * d + np.r_[0.0, e[1:] ** 2]
    off = e[1:] * d[:-1]                       # A[i, i-1] = A[i-1, i]
    a, c = np.r_[0.0, off], np.r_[off, 0.0]
    assert np.any(np.abs(b) < np.abs(a) + np.abs(c))    # some rows lose dominance
    F = rng.standard_normal(N)
    with pytest.raises(D.DichotomyError):
        D.GenPlan(a, b, c, flags=prelim)
    plan = D.GenPlan(a, b, c, flags=prelim | D.FLAG_ALLOW_NOT_DOMINANT)
    Fd = torch.from_numpy(F).cuda()
    xd = plan.solve(Fd)
    assert plan.status() == 0 and plan.info["growth"] >= 1.0
    ab = np.zeros((3, N))
    ab[0, 1:] = c[:-1]
    ab[1] = b
    ab[2, :-1] = a[1:]
    ref = linalg.solve_banded((1, 1), ab, F)
    x = xd.cpu().numpy()
    r, be = plan.residual(Fd, xd)
    rh, beh = host_residual(a, b, c, F, x)
    assert abs(be - beh) <= 1e-15 + 1e-3 * beh
    assert be < 1e-13, (be, plan.info)
    assert rel(x, ref) < 1e-10, plan.info


def test_residual_check_reports_what_it_sees(D):
    """A non-dominant matrix with oscillating rows: whatever the solve returns, the residual check
    agrees with the residual computed on the host."""
    N = 20000
    rng = np.random.default_rng(25)
    a, c = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    b = rng.uniform(0.2, 1.5, N) * rng.choice([-1.0, 1.0], N)
    F = rng.standard_normal(N)
    try:
        plan = D.GenPlan(a, b, c, flags=HOST | D.FLAG_ALLOW_NOT_DOMINANT)
    except D.DichotomyError as err:     # a zero pivot in some block: refused as singular
        assert err.code == 3
        return
    Fd = torch.from_numpy(F).cuda()
    xd = plan.solve(Fd)
    x = xd.cpu().numpy()
    if not np.all(np.isfinite(x)):
        return
    r, be = plan.residual(Fd, xd)
    rh, beh = host_residual(a, b, c, F, x)
    assert abs(be - beh) <= 1e-15 + 1e-3 * beh and plan.info["growth"] >= 1.0
