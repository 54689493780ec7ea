"""dichotomy_solve_noalloc: the single-system solve for callers that cannot allocate device
memory.  It is called here through the C ABI (ctypes) and compared with the regular entry
point (dichotomy_plan + bind + dichotomy_solve) on two calls in a row, within the tolerance
the other GPU tests use.  The file is named to be collected last, so a run that stops at the
first failure has already run every other test; it also passes on its own in a fresh process.
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


@pytest.mark.parametrize("t,N", [((-1.2, 2.5, -0.8), 1 << 20), ((-1.0, 4.0, -1.0), 65537), ((0.7, 2.5, -1.1), 3001),
                                 ((-1.0, 2.001, -1.0), 200000), ((-1.0, 4.0, -1.0), 1), ((-0.5, 3.0, -1.2), 2)])
def test_noalloc_matches_regular_solve_twice(lib, t, N):
    import paper_1002_2469_gb300 as D
    rng = np.random.default_rng(N)
    F1 = torch.from_numpy(rng.standard_normal(N)).cuda()
    F2 = torch.from_numpy(rng.uniform(-1, 1, N)).cuda()
    ref1 = D.Plan(*t, N, precision=D.PREC_AUTO).solve(F1).cpu().numpy()
    ref2 = D.Plan(*t, N, precision=D.PREC_AUTO).solve(F2).cpu().numpy()
    x = torch.full_like(F1, float("nan"))
    # two calls in a row on the same stream; the second reuses the library's static array
    assert _noalloc(lib, t, F1, x) == 0
    torch.cuda.synchronize()
    assert _rel(x.cpu().numpy(), ref1) < TOL
    x2 = torch.full_like(F2, float("nan"))
    assert _noalloc(lib, t, F2, x2) == 0
    torch.cuda.synchronize()
    assert _rel(x2.cpu().numpy(), ref2) < TOL


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
