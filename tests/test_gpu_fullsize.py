"""Full-size parity of the batched configurations, every system checked.

* The 10 000 uneven systems (N log-uniform in [256, 2^20], 1.28e9 unknowns): every system of the
  GPU batch solve against the oracle's Thomas on all host cores, norm-wise per system.
* Forward + adjoint over 1024 systems of 65536 rows: lambda = T_s^-T w_s and the three
  coefficient gradients of every system against the oracle's adjoint; central differences
  (h = 1e-6) of L_s = <w_s, x_s> in each of the three coefficients of every system, and in F at
  64 seeded rows per system (one row of every system perturbed per batch solve).

The differences are taken as sum_j w_j (x+_j - x-_j) / 2h per system, which avoids the
cancellation of L+ - L-; they use the FP64 form of the solver (the derivative of the exact
solution map is what they estimate).  Agreement: 1e-6 relative (the truncation and rounding of
the differences), the adjoint against the oracle's adjoint 1e-12."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as W  # noqa: E402

TOL = 1e-12
FD_TOL = 1e-6
H = 1e-6


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1002_2469_gb300 as pkg
    return pkg


def per_system_rel(x, ref, off):
    """max_i |x - ref| / max_i |ref| over each system's rows (off: system starts, ascending)."""
    num = np.maximum.reduceat(np.abs(x - ref), off)
    den = np.maximum.reduceat(np.abs(ref), off)
    return num / np.maximum(den, 1e-300)


@pytest.mark.parametrize("prec", [2, 0])
def test_c4_every_system(D, prec):
    free, _ = torch.cuda.mem_get_info()
    if free < 28 * (1 << 30):
        pytest.skip("needs 28 GB of free device memory")
    N, off, tm1, t0, tp1, _ = W.uneven_c4(with_rhs=False)
    total = int(N.sum())
    Fd = W.device_uniform(total, W.SEED_RHS, "cuda")
    b = D.Batch(N, tm1, t0, tp1, precision=prec)
    xd = b.solve(Fd)
    assert b.status() == 0
    F = Fd.cpu().numpy()
    del Fd
    x = xd.cpu().numpy()
    del xd, b
    torch.cuda.empty_cache()
    ref = oracle.thomas_batched(tm1, t0, tp1, N, off, F)
    err = per_system_rel(x, ref, off)
    worst = int(np.argmax(err))
    assert err[worst] < TOL, (worst, float(err[worst]), int(N[worst]), (tm1[worst], t0[worst], tp1[worst]))


@pytest.fixture(scope="module")
def c5(D):
    Ns, off, tm1, t0, tp1, F, w = W.adjoint_c5()
    Fd, wd = torch.from_numpy(F).cuda(), torch.from_numpy(w).cuda()
    return Ns, off, tm1, t0, tp1, F, w, Fd, wd


@pytest.mark.parametrize("prec", [2, 0])
def test_c5_adjoint_every_system(D, c5, prec):
    Ns, off, tm1, t0, tp1, F, w, Fd, wd = c5
    b = D.Batch(Ns, tm1, t0, tp1, precision=prec)
    x = b.solve(Fd)
    gF, gt = b.adjoint(wd, x)
    assert b.status() == 0
    lam, g, xh = gF.cpu().numpy(), gt.cpu().numpy(), x.cpu().numpy()
    xref = oracle.thomas_batched(tm1, t0, tp1, Ns, off, F)
    assert np.max(per_system_rel(xh, xref, off)) < TOL
    bad = []
    for s in range(Ns.size):
        sl = slice(int(off[s]), int(off[s] + Ns[s]))
        tt = (tm1[s], t0[s], tp1[s])
        lref, gref = oracle.adjoint(tt, w[sl], xref[sl])
        e_l = np.max(np.abs(lam[sl] - lref)) / np.max(np.abs(lref))
        e_g = np.max(np.abs(g[s] - gref)) / np.max(np.abs(gref))
        if not (e_l < TOL and e_g < TOL):
            bad.append((s, e_l, e_g))
    assert not bad, bad[:10]


def _segment_dot(w, dx, nsys, n):
    return (w * dx).view(nsys, n).sum(dim=1)


def test_c5_finite_differences_every_system(D, c5):
    """Central differences of L_s = <w_s, x_s> in t_-1, t_0, t_1 for all 1024 systems and in F at
    64 seeded rows of every system, against the adjoint's gradients (MIXED form, AUTO)."""
    Ns, off, tm1, t0, tp1, F, w, Fd, wd = c5
    nsys, n = Ns.size, int(Ns[0])
    b = D.Batch(Ns, tm1, t0, tp1, precision=2)
    x = b.solve(Fd)
    gF, gt = b.adjoint(wd, x)
    assert b.status() == 0
    g = gt.cpu().numpy()
    t = np.stack([tm1, t0, tp1], axis=1)
    for k in range(3):
        tp, tm = t.copy(), t.copy()
        tp[:, k] += H
        tm[:, k] -= H
        xp = D.Batch(Ns, tp[:, 0], tp[:, 1], tp[:, 2], precision=0).solve(Fd)
        xm = D.Batch(Ns, tm[:, 0], tm[:, 1], tm[:, 2], precision=0).solve(Fd)
        fd = (_segment_dot(wd, xp - xm, nsys, n) / (2 * H)).cpu().numpy()
        scale = np.maximum(np.max(np.abs(g), axis=1), 1.0)
        err = np.abs(fd - g[:, k]) / scale
        assert np.max(err) <= FD_TOL, (k, int(np.argmax(err)), float(np.max(err)))
    # in F: one row of every system per pair of solves, 64 rows per system in all
    bf = D.Batch(Ns, tm1, t0, tp1, precision=0)
    rows = np.random.default_rng(W.SEED_W).integers(0, n, size=(64, nsys))
    base = torch.from_numpy(off).cuda()
    lam = gF.view(nsys, n)
    worst = 0.0
    for r in range(64):
        idx = base + torch.from_numpy(rows[r]).cuda()
        Fp, Fm = Fd.clone(), Fd.clone()
        Fp[idx] += H
        Fm[idx] -= H
        fd = _segment_dot(wd, bf.solve(Fp) - bf.solve(Fm), nsys, n) / (2 * H)
        want = lam[torch.arange(nsys, device="cuda"), torch.from_numpy(rows[r]).cuda()]
        scale = torch.clamp(lam.abs().amax(dim=1), min=1.0)
        worst = max(worst, float(((fd - want).abs() / scale).max()))
    assert worst <= FD_TOL, worst
