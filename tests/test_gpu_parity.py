"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bar: norm-wise relative error max|x - x_oracle| / max|x_oracle|
<= 1e-12 for diagonally dominant FP64 systems, in both the FP64 and the MIXED form.  For the
ill-conditioned extras (weak dominance, the 1-D Laplacian) the binary128 oracle arbitrates:
the GPU error against it must stay within the FP64 oracle's own error (times a small factor).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as W  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_2469_gb300 as pkg
    return pkg


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_solve(D, t, F, **kw):
    plan = D.Plan(t[0], t[1], t[2], F.size, **kw)
    Fd = torch.from_numpy(F).cuda()
    x = plan.solve(Fd)
    st = plan.status()
    assert st == 0, f"device status {st}"
    return x.cpu().numpy(), plan.info


T_WELL = [(-1.0, 4.0, -1.0), (-1.2, 2.5, -0.8), (-0.8, 2.5, -1.2), (0.7, 2.5, -1.1), (0.0, 2.0, -1.0),
          (-1.0, 2.0, 0.0), (-0.5, 3.0, 0.25), (2.0, -5.0, 1.5)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t", T_WELL)
@pytest.mark.parametrize("N", [2, 3, 5, 31, 64, 257, 1000, 4097, 65537, 300001])
def test_single_well_conditioned(D, t, N, prec):
    rng = np.random.default_rng(N)
    F = rng.uniform(-1, 1, N)
    x, info = gpu_solve(D, t, F, precision=prec)
    assert rel(x, oracle.thomas(t, F)) < TOL, info


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("bs", [2, 3, 7, 32, 45, 100])
def test_block_sizes_and_widths(D, threads, bs, prec):
    t = (-1.2, 2.5, -0.8)
    N = 77777
    F = np.random.default_rng(bs).standard_normal(N)
    x, info = gpu_solve(D, t, F, block_size=bs, threads=threads, precision=prec)
    assert info["n"] <= bs + 2
    assert rel(x, oracle.thomas(t, F)) < TOL, info


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t", [(-1.2, 2.5, -0.8), (-1.0, 4.0, -1.0), (-1.0, 2.001, -1.0)])
def test_general_path_matches_halo_path(D, t, prec):
    N = 1 << 19
    F = np.random.default_rng(7).standard_normal(N)
    xg, ig = gpu_solve(D, t, F, flags=1, precision=prec)
    xh, ih = gpu_solve(D, t, F, precision=prec)
    assert ig["path"] == 2
    ref = oracle.thomas(t, F)
    assert rel(xg, ref) < TOL and rel(xh, ref) < TOL


@pytest.mark.parametrize("t,N", [((-1.0, 2.001, -1.0), 200000), ((-1.0, 2.0, -1.0), 4096),
                                 ((-1.2, 2.0, -0.8), 50000), ((-1.0, 2.0 + 5.88e-7, -1.0), 4096)])
def test_ill_conditioned_against_binary128(D, t, N):
    F = np.random.default_rng(3).uniform(-1, 1, N)
    xq = oracle.thomas_q(t, F)
    e_oracle = rel(oracle.thomas(t, F), xq)
    x, info = gpu_solve(D, t, F)
    assert rel(x, xq) <= max(TOL, 20 * e_oracle), info


def test_c1_full_and_manufactured(D):
    t, F = W.single_c1()
    x, info = gpu_solve(D, t, F, block_size=256)
    assert info["P"] == 256
    assert rel(x, oracle.thomas(t, F)) < TOL
    xs = W.manufactured_x(65536)
    Fm = oracle.matvec(t, xs)
    x2, _ = gpu_solve(D, t, Fm, block_size=256)
    assert rel(x2, oracle.thomas(t, Fm)) < TOL
    assert rel(x2, xs) < 1e-14


@pytest.mark.parametrize("weak", [False, True])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_c2_full_size(D, weak, prec):
    t, F = W.single_c2(weak=weak)
    x, info = gpu_solve(D, t, F, precision=prec)
    ref = oracle.thomas(t, F)
    assert rel(x, ref) < TOL, info
    # and the oracle, sampled: residual rows of the GPU solution
    idx = np.random.default_rng(0).integers(1, F.size - 1, 1000)
    r = t[0] * x[idx - 1] + t[1] * x[idx] + t[2] * x[idx + 1] - F[idx]
    assert np.max(np.abs(r)) < 1e-12 * (abs(t[0]) + abs(t[1]) + abs(t[2])) * np.max(np.abs(x))


def test_determinism_and_p_invariance(D):
    t = (-1.2, 2.5, -0.8)
    N = 123457
    F = np.random.default_rng(11).standard_normal(N)
    plan = D.Plan(*t, N)
    Fd = torch.from_numpy(F).cuda()
    a = plan.solve(Fd).cpu().numpy()
    b = plan.solve(Fd).cpu().numpy()
    assert np.array_equal(a, b)
    xs = [gpu_solve(D, t, F, block_size=bs)[0] for bs in (3, 17, 64, 150)]
    for x in xs:
        assert rel(x, a) < 2e-15


@pytest.mark.parametrize("scale", [1e-300, 1e-30, 1e-20, 1e20, 1e30, 1e300])
def test_mixed_dynamic_range(D, scale):
    """The MIXED form scales each block by an exact power of two, so its accuracy does not
    depend on the magnitude of F (within the FP64 range)."""
    t = (-1.2, 2.5, -0.8)
    N = 50000
    F = np.random.default_rng(6).standard_normal(N) * scale
    F[::7] *= 1e-6   # a wide spread of magnitudes inside every block
    x, info = gpu_solve(D, t, F, precision=1)
    assert info["precision"] == 1
    assert rel(x, oracle.thomas(t, F)) < TOL


def test_mixed_window_classes(D):
    """Windows whose F are all normal and within 2^119 of each other take the MIXED kernel's
    fast conversions; zeros, subnormals, a wider spread or an all-zero stretch take the general
    ones.  One system crossing all of these matches the oracle, overall and per stretch."""
    t = (-1.2, 2.5, -0.8)
    rng = np.random.default_rng(11)
    seg = 12000
    parts = [rng.standard_normal(seg)]                         # fast
    p = rng.standard_normal(seg)
    p[::5] = 0.0
    parts.append(p)                                            # exact zeros
    p = rng.standard_normal(seg)
    p[::7] *= 1e-40
    parts.append(p)                                            # spread beyond 2^119
    parts.append(rng.standard_normal(seg) * 1e-3)              # fast, other scale
    parts.append(np.zeros(seg))                                # all zero
    p = rng.standard_normal(seg)
    p[3::11] = 1e-310
    parts.append(p)                                            # FP64 subnormals
    parts.append(-np.abs(rng.standard_normal(seg - 3)))        # fast, ragged tail
    F = np.concatenate(parts)
    ref = oracle.thomas(t, F)
    for threads, bs in ((0, 0), (64, 12), (256, 16)):
        x, info = gpu_solve(D, t, F, precision=1, threads=threads, block_size=bs)
        assert info["precision"] == 1
        assert rel(x, ref) < TOL
        for k in (0, 1, 2, 3, 5, 6):
            sl = slice(k * seg, min((k + 1) * seg, F.size))
            assert rel(x[sl], ref[sl]) < 1e-11, (threads, bs, k)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t,N", [((-1.2, 2.5, -0.8), 100000), ((-1.0, 4.0, -1.0), 3000), ((-1.0, 2.001, -1.0), 60000),
                                 ((-0.5, 3.0, 0.25), 2), ((-1.0, 4.0, -1.0), 1)])
def test_series_constant_matrix(D, t, N, prec):
    """A series with one matrix (eq. 2): every row of F solved with one plan, rows strided;
    each equals the single-system solve bit for bit and the oracle to the tolerance."""
    M = 5
    rng = np.random.default_rng(N + prec)
    F = rng.standard_normal((M, N))
    plan = D.Plan(*t, N, precision=prec)
    big = torch.zeros((M, N + 3), dtype=torch.float64, device="cuda")
    big[:, :N] = torch.from_numpy(F).cuda()
    X = torch.full((M, N + 7), float("nan"), dtype=torch.float64, device="cuda")
    D.dichotomy_solve_series(plan.handle, big[:, :N], X[:, :N])
    assert plan.status() == 0
    Xh = X.cpu().numpy()
    assert np.all(np.isnan(Xh[:, N:]))                 # nothing written between the rows
    for k in range(M):
        single = plan.solve(torch.from_numpy(F[k]).cuda()).cpu().numpy()
        assert np.array_equal(Xh[k, :N], single)
        assert rel(Xh[k, :N], oracle.thomas(t, F[k])) < TOL


def test_series_many_right_hand_sides(D):
    """More right-hand sides than one launch's grid.y (65535): the series is split in launches."""
    t, N, M = (-1.2, 2.5, -0.8), 40, 70001
    F = torch.from_numpy(np.random.default_rng(5).standard_normal((M, N))).cuda()
    plan = D.Plan(*t, N, precision=D.PREC_AUTO)
    X = plan.solve_series(F)
    assert plan.status() == 0
    for k in (0, 1, 65534, 65535, 65536, M - 1):
        Fk = F[k].cpu().numpy()
        assert rel(X[k].cpu().numpy(), oracle.thomas(t, Fk)) < TOL


def test_series_arguments(D):
    plan = D.Plan(-1.0, 4.0, -1.0, 100)
    F = torch.zeros((3, 100), dtype=torch.float64, device="cuda")
    x = torch.zeros((3, 100), dtype=torch.float64, device="cuda")
    lib = D._lib.load()
    P = D._lib.ctypes.c_void_p
    st = P(torch.cuda.current_stream().cuda_stream)
    assert lib.dichotomy_solve_series(plan.handle, -1, P(F.data_ptr()), 100, P(x.data_ptr()), 100, st) == 1
    assert lib.dichotomy_solve_series(plan.handle, 3, P(F.data_ptr()), 99, P(x.data_ptr()), 100, st) == 1
    assert lib.dichotomy_solve_series(plan.handle, 3, P(F.data_ptr()), 100, P(F.data_ptr() + 800), 100, st) == 7
    assert lib.dichotomy_solve_series(plan.handle, 0, P(F.data_ptr()), 100, P(x.data_ptr()), 100, st) == 0


QUASI = [((-1.0, 2.5, -1.0), -1.0, -1.0),      # Neumann-type ends
         ((-1.2, 2.5, -0.8), 0.7, -0.3),       # Robin-type, non-symmetric
         ((0.7, 2.5, -1.1), -0.5, 1.5),
         ((-1.0, 2.001, -1.0), -0.9, 0.0),     # weakly dominant: long corner columns
         ((-1.0, 4.0, -1.0), 2.0, -2.5),
         ((-1.2, 2.5, -0.8), 0.0, 0.0)]      # zero corners: still a corner plan (five gradients)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t,psi,chi", QUASI)
@pytest.mark.parametrize("N", [2, 3, 50, 4097, 300001])
def test_quasi_toeplitz_eq21(D, t, psi, chi, N, prec):
    """eq. 21 (t_0 + psi in the first row, t_0 + chi in the last) against the oracle's Thomas
    on the same matrix."""
    F = np.random.default_rng(N).standard_normal(N)
    plan = D.Plan(*t, N, precision=prec, psi=psi, chi=chi)
    x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert plan.status() == 0
    assert rel(x, oracle.thomas_quasi(t, psi, chi, F)) < TOL, plan.info


@pytest.mark.parametrize("prec", [0, 1])
def test_quasi_toeplitz_series_and_paths(D, prec):
    """Quasi-Toeplitz plans through the series entry point, on the halo and the general path."""
    t, psi, chi, N, M = (-1.2, 2.5, -0.8), -0.8, 0.4, 70001, 3
    F = np.random.default_rng(9).standard_normal((M, N))
    for flags in (0, 1):
        plan = D.Plan(*t, N, precision=prec, psi=psi, chi=chi, flags=flags)
        X = plan.solve_series(torch.from_numpy(F).cuda()).cpu().numpy()
        assert plan.status() == 0
        for k in range(M):
            assert rel(X[k], oracle.thomas_quasi(t, psi, chi, F[k])) < TOL, (flags, k)


def test_quasi_one_row(D):
    plan = D.Plan(-1.0, 4.0, -1.0, 1, psi=0.5, chi=0.25)
    x = plan.solve(torch.tensor([3.0], dtype=torch.float64, device="cuda")).cpu().numpy()
    assert x[0] == 3.0 / 4.75


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_quasi_toeplitz_batch(D, prec):
    """Batches of quasi-Toeplitz systems (eq. 21) beside plain ones: every system against the
    oracle's Thomas on its own matrix; long-coupling systems (general path), one-row systems and
    systems without corners included."""
    rng = np.random.default_rng(40 + prec)
    nsys = 60
    N = np.where(rng.uniform(size=nsys) < 0.1, rng.integers(1, 4, nsys), (10 ** rng.uniform(0.5, 5.3, nsys)).astype(np.int64))
    tm1, tp1 = -rng.uniform(0.5, 1.0, nsys), -rng.uniform(0.5, 1.0, nsys)
    t0 = (np.abs(tm1) + np.abs(tp1)) * (1 + 10 ** rng.uniform(-3.5, 0.3, nsys))
    psi = np.where(rng.uniform(size=nsys) < 0.7, (np.abs(tp1) * 1.01 - t0) * rng.uniform(0, 0.9, nsys), 0.0)
    chi = np.where(rng.uniform(size=nsys) < 0.7, (np.abs(tm1) * 1.01 - t0) * rng.uniform(0, 0.9, nsys), 0.0)
    F = rng.standard_normal(int(N.sum()))
    b = D.Batch(N, tm1, t0, tp1, precision=prec, psi=psi, chi=chi)
    x = b.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert b.status() == 0
    off = np.concatenate([[0], np.cumsum(N)[:-1]])
    for s_ in range(nsys):
        o, n = int(off[s_]), int(N[s_])
        t = (tm1[s_], t0[s_], tp1[s_])
        ref = oracle.thomas_quasi(t, psi[s_], chi[s_], F[o:o + n])
        assert rel(x[o:o + n], ref) < TOL, (s_, n, t, psi[s_], chi[s_])
    # the adjoint: lambda_s = A_s^-T w_s and the five gradients per system
    wh = rng.uniform(-1, 1, F.size)
    gF, gt = b.adjoint(torch.from_numpy(wh).cuda(), torch.from_numpy(x).cuda())
    assert b.status() == 0 and gt.shape == (nsys, 5)
    lam, g = gF.cpu().numpy(), gt.cpu().numpy()
    for s_ in range(nsys):
        o, n = int(off[s_]), int(N[s_])
        t = (tm1[s_], t0[s_], tp1[s_])
        lref, gref = oracle.adjoint_quasi(t, psi[s_], chi[s_], wh[o:o + n], x[o:o + n])
        assert rel(lam[o:o + n], lref) < TOL, (s_, n)
        sc = np.max(np.abs(lref)) * np.max(np.abs(x[o:o + n]))
        assert np.all(np.abs(g[s_, :3] - gref[:3]) <= TOL * max(np.max(np.abs(gref[:3])), sc)), (s_, g[s_], gref)
        assert np.all(np.abs(g[s_, 3:] - gref[3:]) <= TOL * sc), (s_, g[s_], gref)


@pytest.mark.parametrize("prec,flags", [(0, 0), (1, 0), (2, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("t,psi,chi", QUASI)
@pytest.mark.parametrize("N", [1, 2, 3, 50, 4097, 300001])
def test_quasi_toeplitz_adjoint(D, t, psi, chi, N, prec, flags):
    """Adjoint of a quasi-Toeplitz plan: lambda = A^-T w and the five gradients
    (t_-1, t_0, t_1, psi, chi) against the oracle's quasi adjoint, on the halo and general paths."""
    rng = np.random.default_rng(N + 17)
    F, w = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    plan = D.Plan(*t, N, precision=prec, psi=psi, chi=chi, flags=flags)
    x = plan.solve(torch.from_numpy(F).cuda())
    gF, gt = plan.adjoint(torch.from_numpy(w).cuda(), x)
    assert plan.status() == 0 and gt.numel() == 5
    lam_ref, g_ref = oracle.adjoint_quasi(t, psi, chi, w, oracle.thomas_quasi(t, psi, chi, F))
    lam = gF.cpu().numpy()
    assert rel(lam, lam_ref) < TOL, plan.info
    g = gt.cpu().numpy()
    assert np.all(np.abs(g[:3] - g_ref[:3]) <= TOL * np.max(np.abs(g_ref[:3])) + 1e-300), (g, g_ref)
    scale = np.max(np.abs(lam_ref)) * np.max(np.abs(x.cpu().numpy()))
    assert np.all(np.abs(g[3:] - g_ref[3:]) <= TOL * scale), (g, g_ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t,psi,chi,N", [((-1.2, 2.5, -0.8), 0.0, 0.0, 300001), ((-1.0, 2.5, -1.0), -1.0, -0.5, 70001),
                                         ((-1.0, 4.0, -1.0), 0.5, 0.25, 1), ((0.7, 2.5, -1.1), 0.0, 0.9, 2)])
def test_residual_check(D, t, psi, chi, N, prec):
    """The a posteriori check of a Toeplitz or quasi-Toeplitz solve against the residual computed
    on the host from the definition of the matrix (eq. 21 for the corners)."""
    F = np.random.default_rng(N).standard_normal(N)
    plan = D.Plan(*t, N, precision=prec, psi=psi, chi=chi)
    Fd = torch.from_numpy(F).cuda()
    xd = plan.solve(Fd)
    r, be = plan.residual(Fd, xd)
    x = xd.cpu().numpy()
    d = np.full(N, t[1])
    d[0] += psi
    d[-1] += chi
    ax = d * x
    ax[1:] += t[0] * x[:-1]
    ax[:-1] += t[2] * x[1:]
    rh = np.max(np.abs(F - ax))
    nA = max(abs(t[0]) + abs(t[1]) + abs(t[2]), abs(t[1] + psi) + abs(t[2]), abs(t[0]) + abs(t[1] + chi))
    if N == 1:
        nA = abs(t[1] + psi + chi)
    beh = rh / (nA * np.max(np.abs(x)) + np.max(np.abs(F)))
    assert abs(be - beh) <= 1e-15 + 1e-3 * beh and be < (1e-15 if prec == 0 else 1e-13)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("t", [(1.0, 1.5, -1.0), (1.0, 0.3, -1.0), (0.5, -0.8, -1.0)])
def test_toeplitz_without_dominance(D, t, prec):
    """Matrices without diagonal dominance whose characteristic roots are real and split by the
    unit circle, accepted with DICH_FLAG_ALLOW_NOT_DOMINANT: against LAPACK's banded LU with
    partial pivoting (scipy; Thomas without pivoting is no reference here) and the residual check."""
    linalg = pytest.importorskip("scipy.linalg")
    N = 300001
    F = np.random.default_rng(31).standard_normal(N)
    with pytest.raises(D.DichotomyError):
        D.Plan(*t, N, precision=prec)
    plan = D.Plan(*t, N, precision=prec, flags=D.FLAG_ALLOW_NOT_DOMINANT)
    Fd = torch.from_numpy(F).cuda()
    xd = plan.solve(Fd)
    assert plan.status() == 0
    ab = np.zeros((3, N))
    ab[0, 1:] = t[2]
    ab[1] = t[1]
    ab[2, :-1] = t[0]
    ref = linalg.solve_banded((1, 1), ab, F)
    assert rel(xd.cpu().numpy(), ref) < TOL, plan.info
    r, be = plan.residual(Fd, xd)
    assert be < (1e-15 if plan.info["precision"] == 0 else 1e-13)


def test_trivial_sizes(D):
    for N in (0, 1, 2):
        F = np.arange(1, N + 1, dtype=np.float64)
        plan = D.Plan(-1.0, 4.0, -1.0, N)
        x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
        if N:
            assert rel(x, oracle.thomas((-1.0, 4.0, -1.0), F)) < TOL


def test_nonfinite_is_flagged(D):
    N = 10000
    F = np.ones(N)
    F[5000] = np.inf
    plan = D.Plan(-1.0, 4.0, -1.0, N, flags=2)
    plan.solve(torch.from_numpy(F).cuda())
    assert plan.status() == 5
    assert plan.status() == 0   # the word is cleared by reading it


def test_bad_arguments_are_rejected(D):
    N = 1000
    plan = D.Plan(-1.0, 4.0, -1.0, N)
    Fh = torch.ones(N, dtype=torch.float64)
    Fd = Fh.cuda()
    with pytest.raises(TypeError):
        plan.solve(Fh)                                           # host tensor: no CPU path
    with pytest.raises(D.DichotomyError) as e:
        D.dichotomy_solve(plan.handle, Fd, Fd)                   # x aliases F
    assert e.value.code == 7
    import ctypes
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()
    # a host pointer passed through the C ABI is refused (no CPU fallback)
    rc = lib.dichotomy_solve(plan.handle, ctypes.c_void_p(Fh.data_ptr()), ctypes.c_void_p(Fd.data_ptr()), None)
    assert rc == 1
    # misaligned device pointer
    rc = lib.dichotomy_solve(plan.handle, ctypes.c_void_p(Fd.data_ptr() + 4), ctypes.c_void_p(Fd.data_ptr()), None)
    assert rc == 1


# ------------------------------------------------------------------ batches
def batch_solve(D, N, tm1, t0, tp1, F, **kw):
    b = D.Batch(N, tm1, t0, tp1, **kw)
    x = b.solve(torch.from_numpy(F).cuda())
    assert b.status() == 0
    return x.cpu().numpy(), b


@pytest.mark.parametrize("prec", [0, 2])
def test_batched_uneven_small(D, prec):
    N, off, tm1, t0, tp1, F = W.uneven_c4(nsys=300, hi=1 << 16)
    x, b = batch_solve(D, N, tm1, t0, tp1, F, precision=prec)
    ref = oracle.thomas_batched(tm1, t0, tp1, N, off, F)
    worst = max(rel(x[o:o + n], ref[o:o + n]) for o, n in zip(off, N))
    assert worst < TOL


def test_batched_edge_systems(D):
    N = np.array([1, 2, 3, 0, 5, 64, 65, 4099, 70001, 1])
    off = W.offsets(N)
    rng = np.random.default_rng(5)
    tm1 = rng.uniform(-1, -0.5, N.size)
    tp1 = rng.uniform(-1, -0.5, N.size)
    t0 = rng.uniform(2.05, 4, N.size)
    F = rng.uniform(-1, 1, int(N.sum()))
    x, _ = batch_solve(D, N, tm1, t0, tp1, F)
    ref = oracle.thomas_batched(tm1, t0, tp1, N, off, F)
    for o, n in zip(off, N):
        if n:
            assert rel(x[o:o + n], ref[o:o + n]) < TOL


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batched_general_path_systems(D, prec):
    """Systems whose coupling outlasts half a window (the 1-D Laplacian, weakly dominant and
    low Poisson modes) take the general path inside a batch, beside windowed ones; forward and
    adjoint against the oracle (binary128 arbitrating the ill-conditioned ones)."""
    N = np.array([100000, 3000, 131072, 70001, 1, 50000])
    tm1 = np.array([-1.0, -1.0, -1.0, -1.2, -1.0, -0.7])
    t0 = np.array([2.0, 4.0, 2.0 + 5.88e-7, 2.5, 3.0, 1.7 + 1e-4])
    tp1 = np.array([-1.0, -1.0, -1.0, -0.8, -1.0, -1.0])
    off = W.offsets(N)
    rng = np.random.default_rng(13)
    F = rng.uniform(-1, 1, int(N.sum()))
    w = rng.uniform(-1, 1, int(N.sum()))
    b = D.Batch(N, tm1, t0, tp1, precision=prec)
    Fd = torch.from_numpy(F).cuda()
    x = b.solve(Fd)
    gF, gt = b.adjoint(torch.from_numpy(w).cuda(), x)
    assert b.status() == 0
    x, gF, gt = x.cpu().numpy(), gF.cpu().numpy(), gt.cpu().numpy()
    import math
    for s in range(N.size):
        sl = slice(int(off[s]), int(off[s] + N[s]))
        t = (tm1[s], t0[s], tp1[s])
        xq = oracle.thomas_q(t, F[sl])
        e_or = rel(oracle.thomas(t, F[sl]), xq)
        assert rel(x[sl], xq) <= max(TOL, 20 * e_or), s
        lam, g = oracle.adjoint(t, w[sl], oracle.thomas(t, F[sl]))
        lamq = oracle.thomas_q((tp1[s], t0[s], tm1[s]), w[sl])
        e_lam = rel(lam, lamq)
        assert rel(gF[sl], lamq) <= max(TOL, 20 * e_lam), s
        # dL/dt from the binary128 solutions, summed exactly: the GPU's gradient may be as far
        # from it as its forward and adjoint solutions allow
        gq = -np.array([math.fsum(lamq[1:] * xq[:-1]), math.fsum(lamq * xq), math.fsum(lamq[:-1] * xq[1:])])
        e_g = np.max(np.abs(g - gq)) / np.max(np.abs(gq))
        assert np.max(np.abs(gt[s] - gq)) / np.max(np.abs(gq)) <= max(1e-10, 20 * max(e_or, e_lam, e_g)), s


@pytest.fixture(scope="module")
def c3_reference():
    """C3 inputs, the FP64 oracle and the binary128 oracle for every mode."""
    tm1, t0, tp1, N, rhs = W.poisson_c3()
    F = rhs.reshape(-1)
    off = W.offsets(N)
    ref = oracle.thomas_batched(tm1, t0, tp1, N, off, F)
    refq = np.concatenate([oracle.thomas_q((tm1[k], t0[k], tp1[k]), rhs[k]) for k in range(N.size)])
    return tm1, t0, tp1, N, off, F, ref, refq


@pytest.mark.parametrize("prec", [0, 2])
def test_c3_poisson_full(D, prec, c3_reference):
    """Low Poisson modes have kappa up to 3.4e6, so two FP64 solvers may differ by up to
    kappa * u; there the binary128 oracle decides: the GPU must be within 1e-12 of the
    FP64 oracle, or no farther from the binary128 solution than the FP64 oracle is."""
    tm1, t0, tp1, N, off, F, ref, refq = c3_reference
    x, b = batch_solve(D, N, tm1, t0, tp1, F, precision=prec)
    bad = []
    for k, (o, n) in enumerate(zip(off, N)):
        e_gpu = rel(x[o:o + n], ref[o:o + n])
        if e_gpu < TOL:
            continue
        e_gpu_q = rel(x[o:o + n], refq[o:o + n])
        e_orc_q = rel(ref[o:o + n], refq[o:o + n])
        if e_gpu_q > max(TOL, 2.0 * e_orc_q):
            bad.append((k + 1, e_gpu, e_gpu_q, e_orc_q))
    assert not bad, bad[:10]


def test_c4_full_size_sampled(D):
    N, off, tm1, t0, tp1, _ = W.uneven_c4(with_rhs=False)
    total = int(N.sum())
    Fd = W.device_uniform(total, W.SEED_RHS, "cuda")
    b = D.Batch(N, tm1, t0, tp1, precision=2)
    xd = b.solve(Fd)
    assert b.status() == 0
    pick = np.random.default_rng(0).choice(N.size, 40, replace=False)
    pick = np.concatenate([pick, [int(np.argmax(N)), int(np.argmin(N))]])
    for s in pick:
        o, n = int(off[s]), int(N[s])
        F = Fd[o:o + n].cpu().numpy()
        ref = oracle.thomas((tm1[s], t0[s], tp1[s]), F)
        assert rel(xd[o:o + n].cpu().numpy(), ref) < TOL, s


@pytest.mark.parametrize("k", [-100, -80, -40, 0, 40, 80, 100])
def test_scaled_coefficients(D, k):
    """T scaled by 2^k: AUTO keeps MIXED while the scale factor g stays within 2^-60..2^60 and
    takes FP64 beyond; both stay within the tolerance (and with F scaled the other way)."""
    t = tuple(np.array([-1.2, 2.5, -0.8]) * 2.0 ** k)
    N = 300001
    F = np.random.default_rng(5).standard_normal(N) * 2.0 ** (k // 2)
    x, info = gpu_solve(D, t, F, precision=2)
    assert info["precision"] == (1 if abs(k) <= 40 else 0)
    assert rel(x, oracle.thomas(t, F)) < TOL


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t", [(-1.2, 2.5, -0.8), (0.7, 2.5, -1.1), (-1.0, 4.0, -1.0)])
@pytest.mark.parametrize("N", [1, 2, 50, 4097, 300001])
def test_adjoint_single(D, t, N, prec):
    rng = np.random.default_rng(N)
    F = rng.uniform(-1, 1, N)
    w = rng.uniform(-1, 1, N)
    plan = D.Plan(*t, N, precision=prec)
    x = plan.solve(torch.from_numpy(F).cuda())
    gF, gt = plan.adjoint(torch.from_numpy(w).cuda(), x)
    lam_ref, gt_ref = oracle.adjoint(t, w, oracle.thomas(t, F))
    assert rel(gF.cpu().numpy(), lam_ref) < TOL
    g = gt.cpu().numpy()
    assert np.all(np.abs(g - gt_ref) <= TOL * np.max(np.abs(gt_ref)) + 1e-300)


@pytest.mark.parametrize("kind", ["uniform", "zeros", "wide", "1e200", "1e-200", "1e-300", "1e300", "mixed"])
@pytest.mark.parametrize("bs,threads,flags", [(0, 0, 0), (14, 128, 0), (15, 64, 0), (16, 256, 0), (0, 0, 1)])
def test_adjoint_gradient_sums_x_ranges(D, kind, bs, threads, flags):
    """The MIXED adjoint forms the gradient sums in float-float where the forward solution of a
    window has a narrow exponent range, else on the FP64 pipe: both against the oracle's sums
    with x given directly (zeros, 200 decades, the ends of the FP64 range, windows of both kinds)."""
    t = (-1.2, 2.5, -0.8)
    N = 70001
    rng = np.random.default_rng(17)
    w = rng.uniform(-1, 1, N)
    x = rng.uniform(-1, 1, N)
    if kind == "zeros":
        x[rng.integers(0, N, 50)] = 0.0
    elif kind == "wide":
        x *= 10.0 ** rng.uniform(-100, 100, N)
    elif kind == "mixed":   # every third window of 4096 rows spans 80 decades
        for k in range(0, N, 3 * 4096):
            x[k:k + 4096] *= 10.0 ** rng.uniform(-40, 40, len(x[k:k + 4096]))
    elif kind != "uniform":
        x *= float(kind)
    plan = D.Plan(*t, N, precision=1, block_size=bs, threads=threads, flags=flags)
    gF, gt = plan.adjoint(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda())
    assert plan.status() == 0
    assert (plan.info["path"] == 2) == bool(flags)
    lam_ref, gt_ref = oracle.adjoint(t, w, x)
    assert rel(gF.cpu().numpy(), lam_ref) < TOL
    # each sum against the sum of its terms' magnitudes (the bound of an FP64 dot product)
    mag = np.array([np.dot(np.abs(lam_ref[1:]), np.abs(x[:-1])), np.dot(np.abs(lam_ref), np.abs(x)),
                    np.dot(np.abs(lam_ref[:-1]), np.abs(x[1:]))])
    assert np.all(np.abs(gt.cpu().numpy() - gt_ref) <= TOL * mag), (gt.cpu().numpy(), gt_ref)


def test_adjoint_batched_gradient_sums_x_ranges(D):
    """The batched MIXED adjoint with forward solutions of every kind in one batch: per-system
    sums from float-float and FP64 windows, combined by the fixed-order finalisation."""
    rng = np.random.default_rng(23)
    Ns = np.array([5000, 70001, 4096, 300, 123457, 65536], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)
    tm1 = rng.uniform(-1.0, -0.5, Ns.size)
    tp1 = rng.uniform(-1.0, -0.5, Ns.size)
    t0 = rng.uniform(2.3, 4.0, Ns.size)
    w = rng.uniform(-1, 1, int(Ns.sum()))
    x = rng.uniform(-1, 1, int(Ns.sum()))
    kinds = ["uniform", "zeros", "wide", "1e-250", "mixed", "1e250"]
    for s_, k in enumerate(kinds):
        sl = slice(off[s_], off[s_] + Ns[s_])
        if k == "zeros":
            x[sl][rng.integers(0, Ns[s_], 20)] = 0.0
        elif k == "wide":
            x[sl] *= 10.0 ** rng.uniform(-100, 100, Ns[s_])
        elif k == "mixed":
            x[sl][: Ns[s_] // 2] *= 10.0 ** rng.uniform(-60, 60, Ns[s_] // 2)
        elif k != "uniform":
            x[sl] *= float(k)
    b = D.Batch(Ns, tm1, t0, tp1, precision=1)
    gF, gt = b.adjoint(torch.from_numpy(w).cuda(), torch.from_numpy(x).cuda())
    assert b.status() == 0
    gF, gt = gF.cpu().numpy(), gt.cpu().numpy()
    for s_ in range(Ns.size):
        sl = slice(off[s_], off[s_] + Ns[s_])
        tt = (tm1[s_], t0[s_], tp1[s_])
        lam, g = oracle.adjoint(tt, w[sl], x[sl])
        xs = x[sl]
        mag = np.array([np.dot(np.abs(lam[1:]), np.abs(xs[:-1])), np.dot(np.abs(lam), np.abs(xs)),
                        np.dot(np.abs(lam[:-1]), np.abs(xs[1:]))])
        assert rel(gF[sl], lam) < TOL, kinds[s_]
        assert np.all(np.abs(gt[s_] - g) <= TOL * mag), (kinds[s_], gt[s_], g)


def test_adjoint_general_path(D):
    t = (-1.2, 2.5, -0.8)
    N = 1 << 18
    rng = np.random.default_rng(1)
    F, w = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    plan = D.Plan(*t, N, flags=1)
    x = plan.solve(torch.from_numpy(F).cuda())
    gF, gt = plan.adjoint(torch.from_numpy(w).cuda(), x)
    lam_ref, gt_ref = oracle.adjoint(t, w, oracle.thomas(t, F))
    assert rel(gF.cpu().numpy(), lam_ref) < TOL
    assert np.max(np.abs(gt.cpu().numpy() - gt_ref)) <= TOL * np.max(np.abs(gt_ref))


@pytest.mark.parametrize("prec", [0, 2])
def test_adjoint_batched_c5_reduced(D, prec):
    Ns, off, tm1, t0, tp1, F, w = W.adjoint_c5(nsys=64)
    b = D.Batch(Ns, tm1, t0, tp1, precision=prec)
    x = b.solve(torch.from_numpy(F).cuda())
    gF, gt = b.adjoint(torch.from_numpy(w).cuda(), x)
    gF, gt = gF.cpu().numpy(), gt.cpu().numpy()
    for s in range(Ns.size):
        sl = slice(off[s], off[s] + Ns[s])
        tt = (tm1[s], t0[s], tp1[s])
        lam, g = oracle.adjoint(tt, w[sl], oracle.thomas(tt, F[sl]))
        assert rel(gF[sl], lam) < TOL
        assert np.max(np.abs(gt[s] - g)) <= TOL * np.max(np.abs(g))


def test_adjoint_finite_differences(D):
    """Central differences (h = 1e-6) of L = <w, x(t)> against the adjoint gradient."""
    t = np.array([-1.2, 2.5, -0.8])
    N = 100000
    rng = np.random.default_rng(2)
    F, w = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    Fd, wd = torch.from_numpy(F).cuda(), torch.from_numpy(w).cuda()
    plan = D.Plan(*t, N)
    x = plan.solve(Fd)
    gF, gt = plan.adjoint(wd, x)
    h = 1e-6
    for k in range(3):
        tp, tm = t.copy(), t.copy()
        tp[k] += h
        tm[k] -= h
        lp = float(torch.dot(wd, D.Plan(*tp, N).solve(Fd)))
        lm = float(torch.dot(wd, D.Plan(*tm, N).solve(Fd)))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - float(gt[k])) <= 1e-6 * max(1.0, abs(fd))
    # and in F on a sample of indices
    for i in np.random.default_rng(0).integers(0, N, 8):
        Fp = Fd.clone(); Fp[i] += h
        Fm = Fd.clone(); Fm[i] -= h
        fd = (float(torch.dot(wd, plan.solve(Fp))) - float(torch.dot(wd, plan.solve(Fm)))) / (2 * h)
        assert abs(fd - float(gF[i])) <= 1e-6 * max(1.0, abs(fd))


def test_autograd_function(D):
    t = torch.tensor([-1.2, 2.5, -0.8], dtype=torch.float64, device="cuda", requires_grad=True)
    N = 5000
    F = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, N)).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, N)).cuda()
    x = D.DichotomySolve.apply(F, t)
    (x * w).sum().backward()
    tt = tuple(t.detach().cpu().tolist())
    lam, g = oracle.adjoint(tt, w.cpu().numpy(), oracle.thomas(tt, F.detach().cpu().numpy()))
    assert rel(F.grad.cpu().numpy(), lam) < TOL
    assert np.max(np.abs(t.grad.cpu().numpy() - g)) <= TOL * np.max(np.abs(g))


@pytest.mark.parametrize("corners", [(-0.8, 0.4), (0.0, 0.0), (0.0, 1.1)])
def test_autograd_quasi(D, corners):
    """Autograd through a quasi-Toeplitz solve: gradients of <w, x> with respect to F, t and the
    corners, against the oracle's quasi adjoint."""
    t = torch.tensor([-1.2, 2.5, -0.8], dtype=torch.float64, device="cuda", requires_grad=True)
    c = torch.tensor(corners, dtype=torch.float64, device="cuda", requires_grad=True)
    N = 3001
    F = torch.from_numpy(np.random.default_rng(6).uniform(-1, 1, N)).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, N)).cuda()
    x = D.DichotomySolveQuasi.apply(F, t, c)
    (x * w).sum().backward()
    tt = tuple(t.detach().cpu().tolist())
    lam, g = oracle.adjoint_quasi(tt, corners[0], corners[1], w.cpu().numpy(),
                                  oracle.thomas_quasi(tt, corners[0], corners[1], F.detach().cpu().numpy()))
    assert rel(F.grad.cpu().numpy(), lam) < TOL
    assert np.max(np.abs(t.grad.cpu().numpy() - g[:3])) <= TOL * np.max(np.abs(g[:3]))
    assert np.max(np.abs(c.grad.cpu().numpy() - g[3:])) <= TOL * np.max(np.abs(lam)) * np.max(np.abs(x.detach().cpu().numpy()))


@pytest.mark.parametrize("flags", [0, 32, 64])
def test_mixed_kernel_paths(D, flags):
    """The MIXED form through the register path (flag 32), the shared-memory path (64) and the
    library's choice (0): single plans of halo and one-window shape, a batch with one-window, halo,
    ragged and one-row systems, and a series; all against the oracle."""
    rng = np.random.default_rng(77 + flags)
    for t, N in [((-1.2, 2.5, -0.8), 300001), ((-1.0, 4.0, -1.0), 4096), ((0.7, 2.5, -1.1), 4099),
                 ((-1.0, 2.3, -1.0), 1 << 20)]:
        F = rng.standard_normal(N)
        x, info = gpu_solve(D, t, F, precision=1, flags=flags)
        assert rel(x, oracle.thomas(t, F)) < TOL, (t, N, flags, info)
    Ns = np.array([4096, 4096, 1, 70001, 4100, 300000, 16, 33], dtype=np.int64)
    tm1, tp1 = -rng.uniform(0.5, 1.0, Ns.size), -rng.uniform(0.5, 1.0, Ns.size)
    t0 = (np.abs(tm1) + np.abs(tp1)) * rng.uniform(1.05, 2.0, Ns.size)
    off = np.concatenate([[0], np.cumsum(Ns)[:-1]])
    F = rng.uniform(-1, 1, int(Ns.sum()))
    b = D.Batch(Ns, tm1, t0, tp1, precision=1, flags=flags)
    x = b.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert b.status() == 0
    for s_ in range(Ns.size):
        o, n = int(off[s_]), int(Ns[s_])
        assert rel(x[o:o + n], oracle.thomas((tm1[s_], t0[s_], tp1[s_]), F[o:o + n])) < TOL, (s_, flags)
    plan = D.Plan(-1.2, 2.5, -0.8, 70000, precision=1, flags=flags)
    Fs = rng.standard_normal((3, 70000))
    X = plan.solve_series(torch.from_numpy(Fs).cuda()).cpu().numpy()
    for k in range(3):
        assert rel(X[k], oracle.thomas((-1.2, 2.5, -0.8), Fs[k])) < TOL


@pytest.mark.parametrize("rs", [0.5, 0.5922, 0.5946, 0.5960, 0.62])
@pytest.mark.parametrize("shape", ["random", "one_block", "alternating_scale"])
def test_tree_levels_either_side_of_the_cheap_bound(D, rs, shape):
    """Middle-window trees take their levels by one FMA on the low part when both pair-map factors
    are at most 2^-24 (about |rs|, |ib| <= 0.5946 for 16-row blocks) and by full float-float products
    otherwise: systems on both sides of the bound, with right-hand sides that put all of a window's
    weight in one block (the other blocks' scan values start from zero) or alternate between
    magnitudes 1e-30 and 1, against the oracle."""
    # T = tridiag{-rs, 1 + rs ib, -ib} = (1 - rs E^-1)(1 - ib E) on bi-infinite sequences: the roots
    # of t_1 r^2 + t_0 r + t_-1 are rs and 1 / ib
    ib = 0.7 * rs
    t = (-rs, 1.0 + rs * ib, -ib)
    N = 1 << 18
    rng = np.random.default_rng(int(rs * 1e4))
    if shape == "random":
        F = rng.standard_normal(N)
    elif shape == "one_block":
        F = np.zeros(N)
        for w0 in range(0, N, 4096):
            F[w0 + 2000:w0 + 2016] = rng.standard_normal(16)
    else:
        F = rng.standard_normal(N) * np.where((np.arange(N) // 16) % 2 == 0, 1.0, 1e-30)
    x, info = gpu_solve(D, t, F, precision=1, flags=32)
    assert info["path"] == 1, info
    assert rel(x, oracle.thomas(t, F)) < TOL, (rs, shape)


def test_odd_offsets(D):
    """Systems of a batch at odd row offsets (their rows start 8 bytes past a 16-byte boundary, where
    the register path's bulk copies cannot start) take the shared-memory path: the same solutions, up
    to rounding order, as the batch laid out at even offsets, and the oracle's.  A plan solve on a
    view one element into a buffer likewise."""
    rng = np.random.default_rng(123)
    Ns = np.array([70001, 4099, 65536, 300000, 33, 1 << 17, 8192, 9], dtype=np.int64)
    tm1, tp1 = -rng.uniform(0.5, 1.0, Ns.size), -rng.uniform(0.5, 1.0, Ns.size)
    t0 = (np.abs(tm1) + np.abs(tp1)) * rng.uniform(1.05, 2.0, Ns.size)
    tight = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)   # odd offsets from the second on
    Ne = Ns + (Ns & 1)
    even = np.concatenate([[0], np.cumsum(Ne)[:-1]]).astype(np.int64)
    assert (tight & 1).any() and not (even & 1).any()
    Fs = [rng.uniform(-1, 1, int(n)) for n in Ns]
    out = {}
    for name, off in (("tight", tight), ("even", even)):
        tot = int(off[-1] + Ns[-1])
        F = np.zeros(tot + 1)
        for s_, o in enumerate(off):
            F[int(o):int(o) + int(Ns[s_])] = Fs[s_]
        b = D.Batch(Ns, tm1, t0, tp1, offset=off, precision=1, flags=32)
        x = b.solve(torch.from_numpy(F).cuda()).cpu().numpy()
        assert b.status() == 0
        out[name] = [x[int(o):int(o) + int(n)] for o, n in zip(off, Ns)]
    for s_ in range(Ns.size):
        assert rel(out["tight"][s_], out["even"][s_]) < 1e-13, s_
        assert rel(out["tight"][s_], oracle.thomas((tm1[s_], t0[s_], tp1[s_]), Fs[s_])) < TOL, s_
    t, N = (-1.2, 2.5, -0.8), 200000
    F = rng.standard_normal(N)
    buf = torch.zeros(N + 1, dtype=torch.float64, device="cuda")
    xbuf = torch.zeros(N + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(F).cuda()
    plan = D.Plan(*t, N, precision=1, flags=32)
    plan.solve(buf[1:], out=xbuf[1:])
    assert plan.status() == 0
    assert xbuf[0].item() == 0.0
    assert rel(xbuf[1:].cpu().numpy(), oracle.thomas(t, F)) < TOL


@pytest.mark.parametrize("flags", [32, 64])
def test_windows_of_wide_dynamic_range(D, flags):
    """Right-hand sides whose windows span hundreds of decades with exact zeros (the spectrum of a
    smooth source: the largest values qualify for the fast conversions, the smallest lie far below
    them), through both MIXED paths, against the oracle norm-wise; and the 4096 Poisson modes of
    the smooth source, every mode against the oracle with binary128 arbitrating."""
    rng = np.random.default_rng(91)
    for t, N in [((-1.2, 2.5, -0.8), 300001), ((-1.0, 4.0, -1.0), 4096)]:
        F = rng.standard_normal(N) * 10.0 ** (-rng.uniform(0, 300, N))
        F[rng.uniform(size=N) < 0.2] = 0.0
        F[::1000] = rng.standard_normal(F[::1000].size)     # the windows' largest values stay O(1)
        x, info = gpu_solve(D, t, F, precision=1, flags=flags)
        assert rel(x, oracle.thomas(t, F)) < TOL, (t, N, flags)
    tm1, t0, tp1, Ns, rhs = W.poisson_c3()
    off = W.offsets(Ns)
    F = rhs.reshape(-1)
    b = D.Batch(Ns, tm1, t0, tp1, precision=2, flags=flags)
    x = b.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert b.status() == 0
    ref = oracle.thomas_batched(tm1, t0, tp1, Ns, off, F)
    bad = []
    for k in range(Ns.size):
        sl = slice(int(off[k]), int(off[k] + Ns[k]))
        if rel(x[sl], ref[sl]) < TOL:
            continue
        refq = oracle.thomas_q((tm1[k], t0[k], tp1[k]), F[sl])
        if rel(x[sl], refq) > max(TOL, 2.0 * rel(ref[sl], refq)):
            bad.append(k)
    assert not bad, bad[:10]


def test_autograd_with_cpu_coefficients(D):
    """Coefficients kept on the host (natural for three numbers): their gradients come back on the
    host, for the single, quasi-Toeplitz and batched Functions."""
    N = 4000
    rng = np.random.default_rng(11)
    F = torch.from_numpy(rng.uniform(-1, 1, N)).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.uniform(-1, 1, N)).cuda()
    t = torch.tensor([-1.2, 2.5, -0.8], dtype=torch.float64, requires_grad=True)
    (D.DichotomySolve.apply(F, t) * w).sum().backward()
    assert t.grad.device.type == "cpu"
    tt = tuple(t.detach().tolist())
    lam, g = oracle.adjoint(tt, w.cpu().numpy(), oracle.thomas(tt, F.detach().cpu().numpy()))
    assert np.max(np.abs(t.grad.numpy() - g)) <= TOL * np.max(np.abs(g))
    t2 = torch.tensor([-1.2, 2.5, -0.8], dtype=torch.float64, requires_grad=True)
    c2 = torch.tensor([0.0, 0.0], dtype=torch.float64, requires_grad=True)
    (D.DichotomySolveQuasi.apply(F, t2, c2) * w).sum().backward()
    assert t2.grad.device.type == "cpu" and c2.grad.device.type == "cpu"
    x = oracle.thomas(tt, F.detach().cpu().numpy())
    lq, gq = oracle.adjoint_quasi(tt, 0.0, 0.0, w.cpu().numpy(), x)
    assert np.max(np.abs(c2.grad.numpy() - gq[3:])) <= TOL * np.max(np.abs(lq)) * np.max(np.abs(x))
    Nb = np.array([1000, 3000], dtype=np.int64)
    tb = torch.tensor([[-1.0, 2.5, -1.0], [0.7, 2.5, -1.1]], dtype=torch.float64, requires_grad=True)
    (D.DichotomySolveBatched.apply(F, tb, Nb) * w).sum().backward()
    assert tb.grad.device.type == "cpu" and tb.grad.shape == (2, 3)


def test_autograd_batched_quasi(D):
    """Autograd through a batch of quasi-Toeplitz systems: gradients for F, t and the corners."""
    rng = np.random.default_rng(8)
    N = np.array([3000, 1, 70000, 17], dtype=np.int64)
    tv = np.array([[-1.0, 2.5, -1.0], [-1.0, 4.0, -1.0], [-1.2, 2.5, -0.8], [0.7, 2.5, -1.1]])
    cv = np.array([[-1.0, -1.0], [0.5, 0.25], [0.3, -0.4], [0.0, 0.0]])
    t = torch.tensor(tv, device="cuda", requires_grad=True)
    c = torch.tensor(cv, device="cuda", requires_grad=True)
    F = torch.from_numpy(rng.uniform(-1, 1, int(N.sum()))).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.uniform(-1, 1, int(N.sum()))).cuda()
    x = D.DichotomySolveBatchedQuasi.apply(F, t, c, N)
    (x * w).sum().backward()
    off = np.concatenate([[0], np.cumsum(N)[:-1]])
    Fh, wh, xh = F.detach().cpu().numpy(), w.cpu().numpy(), x.detach().cpu().numpy()
    for s_ in range(N.size):
        o, n = int(off[s_]), int(N[s_])
        lam, g = oracle.adjoint_quasi(tuple(tv[s_]), cv[s_, 0], cv[s_, 1], wh[o:o + n],
                                      oracle.thomas_quasi(tuple(tv[s_]), cv[s_, 0], cv[s_, 1], Fh[o:o + n]))
        assert rel(F.grad.cpu().numpy()[o:o + n], lam) < TOL
        sc = np.max(np.abs(lam)) * np.max(np.abs(xh[o:o + n]))
        assert np.all(np.abs(t.grad.cpu().numpy()[s_] - g[:3]) <= TOL * max(np.max(np.abs(g[:3])), sc))
        assert np.all(np.abs(c.grad.cpu().numpy()[s_] - g[3:]) <= TOL * sc)


@pytest.mark.parametrize("flags", [0, 1])
def test_cuda_graph_capture_and_replay(D, flags):
    """A bound plan's solve only enqueues kernels on the caller's stream (no allocation, no host
    synchronisation), so it can be captured once in a CUDA graph and replayed on new data."""
    t, N = (-1.2, 2.5, -0.8), 100000
    rng = np.random.default_rng(21)
    F = torch.from_numpy(rng.standard_normal(N)).cuda()
    x = torch.empty_like(F)
    plan = D.Plan(*t, N, precision=D.PREC_AUTO, flags=flags)
    plan.solve(F, out=x)                       # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.solve(F, out=x)
    for _ in range(2):
        Fh = rng.standard_normal(N)
        F.copy_(torch.from_numpy(Fh))
        g.replay()
        torch.cuda.synchronize()
        assert rel(x.cpu().numpy(), oracle.thomas(t, Fh)) < TOL
    assert plan.status() == 0


def test_cuda_graph_capture_of_a_batch(D):
    """A batch with both precision forms (the FP64-form windows run on the library's second
    stream, forked from and joined to the caller's) captured and replayed."""
    N, off, tm1, t0, tp1, F = W.uneven_c4(nsys=40, hi=1 << 14)
    t0 = t0.copy()
    t0[:5] = np.abs(tm1[:5]) + np.abs(tp1[:5]) + 1e-4          # weak dominance: the FP64 form under AUTO
    b = D.Batch(N, tm1, t0, tp1, precision=D.PREC_AUTO)
    Fd = torch.from_numpy(F).cuda()
    x = torch.empty_like(Fd)
    b.solve(Fd, out=x)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.solve(Fd, out=x)
    x.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert set(b.info["form"].tolist()) == {0, 1}
    for s in range(N.size):
        sl = slice(int(off[s]), int(off[s] + N[s]))
        t = (tm1[s], t0[s], tp1[s])
        xq = oracle.thomas_q(t, F[sl])
        assert rel(x[sl].cpu().numpy(), xq) <= max(TOL, 20 * rel(oracle.thomas(t, F[sl]), xq)), s
