"""Systems longer than 2^31 rows (64-bit row, block and window indexing): N = 2^31 + 12345 on the
device (17 GB per vector), solved in every precision form and on the general path, checked on
sampled stretches -- the first and last rows and random interior rows -- against the oracle's
Thomas solve of a surrounding stretch wide enough for the coupling to have decayed below 1e-30
at its cut ends (the true ends where the stretch reaches them)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

TOL = 1e-12
N = (1 << 31) + 12345


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 48 * (1 << 30):
        pytest.skip("needs 48 GB of free device memory")
    import paper_1002_2469_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec,flags", [(2, 0), (0, 0), (1, 1)])
def test_beyond_2_31_rows(D, prec, flags):
    t = (-1.2, 2.5, -0.8)
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    F.uniform_(-1.0, 1.0, generator=g)
    x = torch.empty_like(F)
    plan = D.Plan(*t, N, precision=prec, flags=flags)
    plan.solve(F, out=x)
    assert plan.status() == 0
    if flags:
        assert plan.info["path"] == 2
    rng = np.random.default_rng(prec + 10 * flags)
    starts = [0, N - 256, (1 << 31) - 100] + [int(v) for v in rng.integers(0, N - 256, 5)]
    for i0 in starts:
        lo, hi = max(0, i0 - 4096), min(N, i0 + 256 + 4096)
        ref = oracle.thomas(t, F[lo:hi].cpu().numpy())
        got = x[i0:i0 + 256].cpu().numpy()
        want = ref[i0 - lo:i0 - lo + 256]
        assert np.max(np.abs(got - want)) / np.max(np.abs(ref)) < TOL, (i0, plan.info)
    del F, x, plan
    torch.cuda.empty_cache()


def test_batch_beyond_2_31_rows(D):
    """Batch offsets past 2^31: three systems of 2^30 + 7, 2^30 + 5 and 1000 rows back to back."""
    Ns = np.array([(1 << 30) + 7, (1 << 30) + 5, 1000], dtype=np.int64)
    tm1, t0, tp1 = np.array([-1.0, -0.7, -1.1]), np.array([4.0, 2.5, 2.4]), np.array([-1.0, -1.2, -0.6])
    total = int(Ns.sum())
    g = torch.Generator(device="cuda")
    g.manual_seed(8)
    F = torch.empty(total, dtype=torch.float64, device="cuda")
    F.uniform_(-1.0, 1.0, generator=g)
    b = D.Batch(Ns, tm1, t0, tp1, precision=2)
    x = b.solve(F)
    assert b.status() == 0
    off = np.concatenate([[0], np.cumsum(Ns)[:-1]])
    for s in range(3):
        o, n = int(off[s]), int(Ns[s])
        t = (tm1[s], t0[s], tp1[s])
        for i0 in (0, max(0, n - 256), n // 2):
            lo, hi = max(0, i0 - 4096), min(n, i0 + 256 + 4096)
            ref = oracle.thomas(t, F[o + lo:o + hi].cpu().numpy())
            m = min(256, n - i0)
            got = x[o + i0:o + i0 + m].cpu().numpy()
            assert np.max(np.abs(got - ref[i0 - lo:i0 - lo + m])) / np.max(np.abs(ref)) < TOL, (s, i0)
    del F, x, b
    torch.cuda.empty_cache()
