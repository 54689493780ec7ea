"""dichotomy_solve_noalloc: the single-system solve for callers that cannot allocate device
memory.  It is called here through the C ABI (ctypes) and compared, on two calls in a row, with
the CPU oracle's Thomas solve (the binary128 Thomas arbitrating for the weakly dominant case, as
in the other parity tests) and with the regular entry point (dichotomy_plan + bind +
dichotomy_solve), within the tolerance the other GPU tests use.  The file is named to be
collected last, so a run that stops at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1002_2469_gb300 import _lib as L
    return L.load()


def _noalloc(lib, t, F, x):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.dichotomy_solve_noalloc(t[0], t[1], t[2], F.numel(), ctypes.c_void_p(F.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), stream)


def _close_to_oracle(x, t, F):
    """Within TOL of the FP64 oracle, or (ill-conditioned systems) no farther from the binary128
    solution than the FP64 oracle is, times two."""
    import oracle
    ref = oracle.thomas(t, F)
    if _rel(x, ref) < TOL:
        return True
    refq = oracle.thomas_q(t, F)
    return _rel(x, refq) <= max(TOL, 2.0 * _rel(ref, refq))


# path expected of the library's planner (0 single window, 1 halo windows, 2 general path)
CASES = [((-1.2, 2.5, -0.8), 1 << 20, 1), ((-1.0, 4.0, -1.0), 65537, 1), ((0.7, 2.5, -1.1), 3001, 0),
         ((-1.0, 2.001, -1.0), 200000, 2), ((-1.0, 4.0, -1.0), 1, None), ((-0.5, 3.0, -1.2), 2, 0)]


@pytest.mark.parametrize("t,N,path", CASES)
def test_noalloc_matches_oracle_and_regular_solve_twice(lib, t, N, path):
    import paper_1002_2469_gb300 as D
    rng = np.random.default_rng(N)
    F1h, F2h = rng.standard_normal(N), rng.uniform(-1, 1, N)
    F1, F2 = torch.from_numpy(F1h).cuda(), torch.from_numpy(F2h).cuda()
    plan = D.Plan(*t, N, precision=D.PREC_AUTO)
    if path is not None:
        # the planner the allocation-free call shares puts this system on the expected path
        assert plan.info["path"] == path, plan.info
    ref1 = plan.solve(F1).cpu().numpy()
    ref2 = plan.solve(F2).cpu().numpy()
    x = torch.full_like(F1, float("nan"))
    # two calls in a row on the same stream; the second reuses the library's static array
    assert _noalloc(lib, t, F1, x) == 0
    torch.cuda.synchronize()
    x1h = x.cpu().numpy()
    assert _close_to_oracle(x1h, t, F1h)
    assert _rel(x1h, ref1) < TOL
    x2 = torch.full_like(F2, float("nan"))
    assert _noalloc(lib, t, F2, x2) == 0
    torch.cuda.synchronize()
    x2h = x2.cpu().numpy()
    assert _close_to_oracle(x2h, t, F2h)
    assert _rel(x2h, ref2) < TOL


def test_noalloc_refuses_a_capturing_stream(lib):
    # the staging copy reads a host buffer that later calls overwrite: capture is refused
    N = 4096
    F = torch.ones(N, dtype=torch.float64, device="cuda")
    x = torch.empty_like(F)
    assert _noalloc(lib, (-1.0, 4.0, -1.0), F, x) == 0      # first call on the device: set-up
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="relaxed")
        try:
            rc = _noalloc(lib, (-1.0, 4.0, -1.0), F, x)
        finally:
            g.capture_end()
    assert rc == 11               # DICH_ERR_UNSUPPORTED


def test_noalloc_rejects_what_exceeds_its_static_array(lib):
    # the 1-D Laplacian has no decay: its plan needs end tables for every block (too large for
    # the fixed array) or the general path (scratch growing with N) -- both are refused clearly
    N = 1 << 22
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.empty_like(F)
    rc = _noalloc(lib, (-1.0, 2.0, -1.0), F, x)
    assert rc == 9                # DICH_ERR_WORKSPACE: beyond the static array
    assert _noalloc(lib, (-1.0, 1.0, -1.0), F, x) == 2     # not diagonally dominant
    assert _noalloc(lib, (-1.0, 4.0, -1.0), F, F) == 7     # aliasing
