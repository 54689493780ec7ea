"""One system solved in shards (the paper's distributed dichotomy process, Sec. 2.4-2.5) on one GPU:
each shard gets its own copies of its rows of F and its own x (so a shard that touched rows of
another would read or write outside its buffers), the exchanges go through host memory, and the
result is checked against the CPU oracle (the binary128 Thomas arbitrating for the weakly dominant
system, as in the other parity tests) and against the unsharded solve of the same plan."""
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


def close_to_oracle(x, t, F):
    ref = oracle.thomas(t, F)
    if rel(x, ref) < TOL:
        return True
    refq = oracle.thomas_q(t, F)
    return rel(x, refq) <= max(TOL, 2.0 * rel(ref, refq))


def sharded_separate_buffers(D, plan, F, nshards):
    from paper_1002_2469_gb300 import shard as SH
    shards = [SH.Shard(plan, nshards, k) for k in range(nshards)]
    Fk = [torch.from_numpy(F[s.rows].copy()).cuda() for s in shards]
    xk = [torch.empty_like(f) for f in Fk]
    all_maps = [v for s, f, x in zip(shards, Fk, xk) for v in s.reduce(f, x)]
    ends = [s.bounds(all_maps) for s in shards]
    for s, f, x in zip(shards, Fk, xk):
        s.finish(f, x, SH.neighbour_values(ends, s.k))
    assert plan.status() == 0
    rows = [(s.info["row_lo"], s.info["row_hi"]) for s in shards]
    assert rows[0][0] == 0 and rows[-1][1] == F.size and all(rows[i][1] == rows[i + 1][0] for i in range(nshards - 1))
    return np.concatenate([x.cpu().numpy() for x in xk]), ends


CASES = [((-1.2, 2.5, -0.8), 300001, 0, {}), ((-1.2, 2.5, -0.8), 300001, 1, {}),
         ((-1.0, 2.001, -1.0), 200000, 0, {}), ((-1.0, 2.001, -1.0), 200000, 1, {}),
         ((0.7, 2.5, -1.1), 65537, 1, {"flags": 1}), ((-1.0, 4.0, -1.0), 1 << 20, 2, {}),
         ((-1.0, 4.0, -1.0), 50000, 0, {"block_size": 7, "threads": 64})]


@pytest.mark.parametrize("t,N,prec,kw", CASES)
@pytest.mark.parametrize("nshards", [1, 2, 3, 4])
def test_sharded_solve_matches_oracle(D, t, N, prec, kw, nshards):
    plan = D.Plan(*t, N, precision=prec, **kw)
    if nshards > plan.info["tiles"]:
        pytest.skip("fewer windows than shards")
    F = np.random.default_rng(N + nshards).standard_normal(N)
    x, ends = sharded_separate_buffers(D, plan, F, nshards)
    assert close_to_oracle(x, t, F), (plan.info, nshards)
    xu = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    assert rel(x, xu) < 1e-12
    # the values a shard sends its neighbours are the solution at its first and last rows
    from paper_1002_2469_gb300 import shard as SH
    for k in range(nshards):
        info = SH.shard_info(plan, nshards, k)
        assert abs(ends[k][0] - x[info["row_lo"]]) <= 1e-12 * np.max(np.abs(x))
        assert abs(ends[k][1] - x[info["row_hi"] - 1]) <= 1e-12 * np.max(np.abs(x))


def test_sharded_solve_in_one_process_helper(D):
    from paper_1002_2469_gb300 import shard as SH
    t, N = (-1.2, 2.5, -0.8), 1 << 21
    plan = D.Plan(*t, N, precision=2)
    F = np.random.default_rng(3).standard_normal(N)
    x = SH.solve_sharded(plan, torch.from_numpy(F).cuda(), 4).cpu().numpy()
    assert rel(x, oracle.thomas(t, F)) < TOL


def test_shard_arguments(D):
    from paper_1002_2469_gb300 import shard as SH
    plan = D.Plan(-1.2, 2.5, -0.8, 100000)
    with pytest.raises(D.DichotomyError):
        SH.shard_info(plan, plan.info["tiles"] + 1, 0)      # more shards than windows
    with pytest.raises(D.DichotomyError):
        SH.shard_info(plan, 2, 2)                           # no such shard
    qp = D.Plan(-1.0, 2.5, -1.0, 100000, psi=-1.0, chi=-0.5)
    with pytest.raises(D.DichotomyError):
        SH.shard_info(qp, 2, 0)                             # corners: not sharded
