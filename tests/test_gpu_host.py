"""Solves from and to host memory (dichotomy_solve_host): the kernels reading and writing
pinned host memory directly (chunks = 0), and the pipelined copy-in / solve / copy-out (chunks
>= 1, pageable buffers), give the oracle's solution to 1e-12 norm-wise, for every chunking and
the paths that do not pipeline (one window, the general path, quasi-Toeplitz corners).  The
pipelined solves run the device solve's kernels on device staging buffers and give it bitwise;
the direct reads and writes of host memory keep to the shared-memory path of the window kernel
(bulk copies serve device memory only), so they agree with the device solve -- which takes the
register path for 16-row blocks -- to rounding (1e-13 norm-wise)."""
import ctypes

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


def check_host_solve(D, t, N, chunks, prec, pinned=True, seed=0, **kw):
    F = np.random.default_rng(seed + N).standard_normal(N)
    plan = D.Plan(*t, N, precision=prec, **kw)
    Fh = torch.from_numpy(F)
    if pinned:
        Fh = Fh.pin_memory()
    xh = plan.solve_host(Fh, chunks=chunks)
    assert plan.status() == 0
    xd = plan.solve(torch.from_numpy(F).cuda()).cpu()
    if chunks == 0 and pinned:
        assert rel(xh.numpy(), xd.numpy()) < 1e-13, (N, chunks, plan.info)
    else:
        assert torch.equal(xh, xd), (N, chunks, plan.info)      # same windows, same kernels
    if N <= 1 << 20:
        assert rel(xh.numpy(), oracle.thomas(t, F)) < TOL
    return plan.info


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("chunks", [0, 1, 2, 3, 7, 100000])
@pytest.mark.parametrize("N", [2, 5, 4097, 300001, (1 << 20) + 3])
def test_host_solve_matches_device_solve(D, N, chunks, prec):
    check_host_solve(D, (-1.2, 2.5, -0.8), N, chunks, prec)


@pytest.mark.parametrize("t", [(-1.0, 4.0, -1.0), (0.7, 2.5, -1.1), (-0.5, 3.0, 0.25)])
@pytest.mark.parametrize("bs", [3, 16, 45])
def test_host_solve_halos_and_block_sizes(D, t, bs):
    info = check_host_solve(D, t, 500007, 5, 2, block_size=bs, threads=64)
    assert info["path"] == 1


def test_host_solve_pageable_buffers(D):
    check_host_solve(D, (-1.2, 2.5, -0.8), 700001, 0, 1, pinned=False)


def test_host_solve_general_path_and_quasi_plans_copy_whole(D):
    info = check_host_solve(D, (-1.0, 2.001, -1.0), 200000, 0, 0)
    assert info["path"] == 2
    N = 300001
    F = np.random.default_rng(3).standard_normal(N)
    plan = D.Plan(-1.0, 2.5, -1.0, N, psi=-1.0, chi=-0.5, precision=2)
    xh = plan.solve_host(torch.from_numpy(F).pin_memory())
    xd = plan.solve(torch.from_numpy(F).cuda()).cpu()
    assert torch.equal(xh, xd)


def test_host_solve_full_size(D):
    """The configuration bench.py times end to end: N = 2^26, MIXED form, 16 pieces."""
    N = 1 << 26
    t = (-1.2, 2.5, -0.8)
    F = torch.from_numpy(np.random.default_rng(5).standard_normal(N)).pin_memory()
    plan = D.Plan(*t, N, precision=2)
    xh = plan.solve_host(F)
    xd = plan.solve(F.cuda()).cpu()
    assert plan.status() == 0 and rel(xh.numpy(), xd.numpy()) < 1e-13
    idx = np.random.default_rng(6).integers(0, N - 4096, 4)
    Fn = F.numpy()
    for i0 in idx:   # sampled rows against the oracle on a stretch wide enough for the decay
        lo, hi = max(0, i0 - 2048), min(N, i0 + 4096)
        ref = oracle.thomas(t, Fn[lo:hi])
        k0 = i0 - lo
        assert rel(xh.numpy()[i0:i0 + 256], ref[k0:k0 + 256]) < TOL


def test_host_solve_arguments(D):
    from paper_1002_2469_gb300 import _lib as L
    lib = L.load()
    N = 10000
    plan = D.Plan(-1.2, 2.5, -0.8, N)
    h = plan.handle
    Fh = torch.zeros(N, dtype=torch.float64).pin_memory()
    xh = torch.zeros(N, dtype=torch.float64).pin_memory()
    dF = torch.zeros(N, dtype=torch.float64, device="cuda")
    dx = torch.zeros(N, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    s = P(torch.cuda.current_stream().cuda_stream)
    ok = lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(xh.data_ptr()), P(dF.data_ptr()), P(dx.data_ptr()), 0, s)
    assert ok == 0
    torch.cuda.synchronize()
    assert lib.dichotomy_solve_host(h, P(dF.data_ptr()), P(xh.data_ptr()), P(dF.data_ptr()), P(dx.data_ptr()), 0,
                                    s) == 1                       # F on the device
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(xh.data_ptr()), P(Fh.data_ptr()), P(dx.data_ptr()), 2,
                                    s) == 1                       # staging buffer in host memory
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(Fh.data_ptr() + 8), P(dF.data_ptr()), P(dx.data_ptr()),
                                    0, s) == 7                    # x overlaps F
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(xh.data_ptr()), P(dF.data_ptr()), P(dF.data_ptr()), 2,
                                    s) == 7                       # staging buffers overlap
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr() + 4), P(xh.data_ptr()), P(dF.data_ptr()), P(dx.data_ptr()),
                                    0, s) == 1                    # misaligned
    with pytest.raises(TypeError):
        plan.solve_host(torch.zeros(N, dtype=torch.float64, device="cuda"))
    # pinned buffers and chunks = 0: no staging needed; the copy pipeline needs it
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(xh.data_ptr()), None, None, 0, s) == 0
    assert lib.dichotomy_solve_host(h, P(Fh.data_ptr()), P(xh.data_ptr()), None, None, 2, s) == 1
    Fp = torch.zeros(N, dtype=torch.float64)
    xp = torch.zeros(N, dtype=torch.float64)
    assert lib.dichotomy_solve_host(h, P(Fp.data_ptr()), P(xp.data_ptr()), None, None, 0, s) == 1   # pageable
    torch.cuda.synchronize()
