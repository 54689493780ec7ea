"""The intermediates of the Dichotomy Algorithm on the GPU against the oracle's literal
restatement of the paper: on the general path the workspace keeps, per block, the beta^L,
beta^R of eq. 16 (computed on the GPU as the 2x2 map of the block-end values) and the first and
last values of eq. 15/18 (from the block scan), which must equal the oracle's eq. 9-16 solve
(`oracle.dich_eq15`: preliminary vectors G, Z and the sums of eq. 15 written out) on the same
block partition."""
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


def ws_doubles(ws, off, count):
    return ws[off:off + 8 * count].view(torch.float64).cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("t,N,n", [((-1.0, 2.001, -1.0), 3000, 16), ((-1.2, 2.5, -0.8), 5003, 16),
                                   ((0.7, 2.5, -1.1), 4000, 25), ((-1.0, 4.0, -1.0), 2050, 7)])
def test_beta_and_interface_values_match_eq16_and_eq15(D, t, N, n, prec):
    F = np.random.default_rng(N).standard_normal(N)
    plan = D.Plan(*t, N, precision=prec, block_size=n, flags=D.FLAG_FORCE_GENERAL)
    info = plan.info
    assert info["path"] == 2 and info["n"] == n and info["beta_offset"] > 0 and info["iface_offset"] > 0
    x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    P = info["P"]
    starts = oracle.even_starts(N, n)
    assert starts.size == P
    ref = oracle.dich_eq15(t, F, starts)
    scale = np.max(np.abs(ref["x"]))
    beta = ws_doubles(plan.workspace, info["beta_offset"], 2 * P).reshape(P, 2)
    iface = ws_doubles(plan.workspace, info["iface_offset"], 2 * P).reshape(P, 2)
    assert np.max(np.abs(beta[:, 0] - ref["beta_L"])) / scale < TOL
    assert np.max(np.abs(beta[:, 1] - ref["beta_R"])) / scale < TOL
    assert np.max(np.abs(iface[:, 0] - ref["x_first"])) / scale < TOL
    assert np.max(np.abs(iface[:, 1] - ref["x_last"])) / scale < TOL
    assert np.max(np.abs(x - ref["x"])) / scale < TOL
