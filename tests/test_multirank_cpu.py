"""Host logic of the multi-rank bench on CPU: two gloo ranks (127.0.0.1) check the max-over-ranks
timing, the whole-job value (replicas: every rank's units over the slowest rank's time) and
that under torchrun only rank 0 of the reference arm prints its line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = [3.0, 5.0][rank]                       # the second rank is slower
    got = bench.max_over_ranks(ms, world)
    value = bench.whole_job_value(1000, ms, world)
    bench.barrier(world)
    out[rank] = (got, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        got, value = out[r]
        assert got == 5.0
        assert value == pytest.approx(2 * 1000 / 5e-3 / 1e9)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1")
    r1 = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "4096", "--steps", "3",
                         "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    env["RANK"] = "0"
    r0 = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "4096", "--steps", "3",
                         "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def _shard_worker(rank, world, port, out):
    """Shard `rank` of a system of 2 x 37 blocks: the composite of its blocks' prefix and suffix maps
    (what dichotomy_shard_reduce returns), exchanged with DistExchange, folded into the prefix
    entering the shard and the suffix beyond it; then the boundary values to the neighbours."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1002_2469_gb300 import shard as SH
    rng = np.random.default_rng(5)
    nb = 37
    a, b = rng.uniform(-0.9, 0.9, world * nb), rng.standard_normal(world * nb)   # A -> a A + b, per block
    c, d = rng.uniform(-0.9, 0.9, world * nb), rng.standard_normal(world * nb)   # B -> c B + d, per block
    lo, hi = rank * nb, (rank + 1) * nb
    pa, pb = 1.0, 0.0
    for i in range(lo, hi):              # prefix composite, left to right
        pa, pb = a[i] * pa, a[i] * pb + b[i]
    sa, sb = 1.0, 0.0
    for i in range(hi - 1, lo - 1, -1):  # suffix composite, right to left
        sa, sb = c[i] * sa, c[i] * sb + d[i]
    ex = SH.DistExchange()
    all_maps = ex.all_gather_maps(rank, [pa, pb, sa, sb])
    A_in, B_in = SH.fold_maps(all_maps, rank)
    ends = [10.0 * rank + 1.0, 10.0 * rank + 2.0]
    nbr = ex.neighbours(rank, ends)
    out[rank] = (A_in, B_in, nbr, len(all_maps))
    dist.destroy_process_group()


def test_shard_exchange_with_two_gloo_ranks():
    """The sharded solve's exchange on host buffers over two gloo ranks: the gathered maps folded in
    shard order give the sequential composition over all blocks (the associativity the paper's
    dichotomy levels rely on, Sec. 2.5), and each shard receives its neighbours' boundary values."""
    import numpy as np
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    rng = np.random.default_rng(5)
    nb = 37
    a, b = rng.uniform(-0.9, 0.9, 2 * nb), rng.standard_normal(2 * nb)
    c, d = rng.uniform(-0.9, 0.9, 2 * nb), rng.standard_normal(2 * nb)
    A = 0.0
    for i in range(nb):                  # prefix entering shard 1: blocks 0 .. nb-1 in sequence
        A = a[i] * A + b[i]
    B = 0.0
    for i in range(2 * nb - 1, nb - 1, -1):   # suffix beyond shard 0: blocks 2 nb - 1 .. nb
        B = c[i] * B + d[i]
    A0, B0, nbr0, n0 = out[0]
    A1, B1, nbr1, n1 = out[1]
    assert n0 == n1 == 8
    assert A0 == 0.0 and B1 == 0.0
    assert abs(A1 - A) <= 1e-14 * max(1.0, abs(A)) and abs(B0 - B) <= 1e-14 * max(1.0, abs(B))
    assert tuple(nbr0) == (0.0, 11.0) and tuple(nbr1) == (2.0, 0.0)
