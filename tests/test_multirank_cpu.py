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
