"""Host side of the multi-rank bench path, as world-size-2 process groups on the CPU (gloo).

With N GPUs the bench runs one process per GPU. Each rank steps its own copy of the workload, so
per-GPU work stays fixed as N grows (weak scaling). The copies have the same shapes and rank-offset
seeds, and nothing crosses ranks on the data path. The job's time is the slowest rank's, taken
with an all-reduce, and the job's value counts every rank's updates. These are the only
collectives, and they are checked here without a GPU. The reference arm's other ranks exit
without work.
"""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, workload, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = bench.parse(["--workload", workload])
        cases, _ = bench.workload(args, rank)
        shapes = [(c.ny, c.nx) for c in cases]
        checksum = float(sum(c.rhoA0.sum() + c.rhoB0.sum() for c in cases))
        my_ms = 10.0 + 5.0 * rank  # this rank's timed region
        job_ms = bench.max_over_ranks(my_ms, world, "cpu")
        value = bench.job_mlups(world, sum(c.nx * c.ny for c in cases), 100, job_ms)
        q.put((rank, shapes, checksum, job_ms, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("workload", ["couette", "obstacle"])
def test_two_ranks_share_nothing_but_the_timing(workload):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, workload, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    (_, shapes0, sum0, ms0, v0), (_, shapes1, sum1, ms1, v1) = got
    assert shapes0 == shapes1  # the same workload on every rank
    assert sum0 != sum1  # drawn with rank-offset seeds, so the ranks do not repeat each other's work
    assert ms0 == ms1 == 15.0  # every rank reports the slowest rank's time
    nodes = sum(ny * nx for ny, nx in shapes0)
    assert v0 == v1 == pytest.approx(2 * nodes * 100 / 15e-3 / 1e6)


def test_job_value_alone_is_the_rank_value():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_mlups(1, 1_000_000, 100, 10.0) == pytest.approx(1e4)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
