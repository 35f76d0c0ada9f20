"""Host side of the multi-rank bench path, as world-size-2 process groups on the CPU (gloo).

With N GPUs the bench runs one process per GPU. By default each rank steps its own copy of the
workload, so per-GPU work stays fixed as N grows (weak scaling). The copies have the same shapes and
rank-offset seeds. With --split every rank builds the same workload and steps only its share of the
cases, assigned by node count (strong scaling). Nothing crosses ranks on the data path either way.
The job's time is the slowest rank's, taken with an all-reduce, and the job's value counts every
update of the job. These are the only collectives, and they are checked here without a GPU. The
reference arm's other ranks exit without work.
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


def _split_rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = bench.parse(["--workload", "ensemble", "--split"])
        cases, _ = bench.workload(args, 0)
        mine, job_nodes = bench.shard(cases, rank, world)
        names = sorted(c.name for c in mine)
        my_ms = 20.0 + 4.0 * rank
        job_ms = bench.max_over_ranks(my_ms, world, "cpu")
        value = bench.job_mlups(1, job_nodes, 100, job_ms)
        q.put((rank, names, sum(c.nx * c.ny for c in mine), job_nodes, job_ms, value))
    finally:
        dist.destroy_process_group()


def test_split_ranks_share_out_one_ensemble():
    """--split: every rank builds the same 257-case ensemble and keeps its share.  The shares are
    disjoint and cover the ensemble, the loads differ by less than the largest case, and the job
    value counts the ensemble once, over the slowest rank's time."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    (_, names0, n0, job0, ms0, v0), (_, names1, n1, job1, ms1, v1) = got
    assert not set(names0) & set(names1)
    assert len(names0) + len(names1) == 257
    assert n0 + n1 == job0 == job1
    assert abs(n0 - n1) <= 4096 * 256  # the largest case, the co-current channel
    assert ms0 == ms1 == 24.0
    assert v0 == v1 == pytest.approx(job0 * 100 / 24e-3 / 1e6)


def test_lpt_shares_against_brute_force():
    """The longest-processing-time rule: every case on exactly one rank, the largest load within
    the mean plus the largest case, and within Graham's bound (4/3 - 1/(3 world)) of the best
    partition, found here by trying every assignment of small inputs."""
    import itertools

    import numpy as np

    sys.path.insert(0, ROOT)
    import bench

    rng = np.random.default_rng(11)
    for trial in range(60):
        world = int(rng.integers(2, 4))
        sizes = [int(v) for v in rng.integers(1, 50, size=int(rng.integers(world, 9)))]
        shares = bench.lpt_shares(sizes, world)
        assert sorted(i for sh in shares for i in sh) == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in sh) for sh in shares]
        assert max(loads) <= sum(sizes) / world + max(sizes)
        best = min(max(sum(s for s, r in zip(sizes, a) if r == k) for k in range(world))
                   for a in itertools.product(range(world), repeat=len(sizes)))
        assert max(loads) <= (4 / 3 - 1 / (3 * world)) * best + 1e-9
    # equal sizes: round robin by rank, lowest index first
    assert bench.lpt_shares([5, 5, 5, 5, 5], 2) == [[0, 2, 4], [1, 3]]


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


def test_split_needs_a_workload_of_several_cases():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "sphere3d", "--split"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "--split needs a workload of several cases" in r.stderr
    sys.path.insert(0, ROOT)
    import bench

    with pytest.raises(SystemExit):
        bench.shard([object()] * 3, 0, 4)  # more ranks than cases
