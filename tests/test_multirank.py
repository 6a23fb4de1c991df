"""The N > 1 path of bench.py on CPU: replicas, max over ranks, one JSON line from rank 0.

Every simulation is independent, so N GPUs run N replicas with no data exchange; the
only collective is the timing reduction.  Two gloo ranks on CPU exercise it here.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r was slower by r milliseconds
    mx = bench.max_over_ranks_of(10.0 + rank, world, "cpu")
    dist.destroy_process_group()
    q.put((rank, mx))


def test_max_over_ranks_gloo_two_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 11.0, 1: 11.0}


def test_replica_throughput_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.replica_throughput(262144, 100, 4, 1, 2.0)
    two = bench.replica_throughput(262144, 100, 4, 2, 2.0)
    assert two == pytest.approx(2 * one)


@pytest.mark.slow
def test_reference_arm_under_two_ranks_prints_once():
    # rank 0 alone times the oracle and prints; rank 1 exits 0 without work
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    outs = []
    for rank in (0, 1):
        env["RANK"] = str(rank)
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                            "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        outs.append(r.stdout.strip())
    line = json.loads(outs[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert outs[1] == ""
