"""The N > 1 path of bench.py on the CPU: two gloo ranks, each an independent
replica of the workload (no data-path collective), aggregate their timed
regions by the maximum over ranks and report the whole job's units over it."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_seconds = [1.5, 2.0][rank]          # the slower replica is rank 1
    worst = bench.max_over_ranks(my_seconds, world, device="cpu")
    value = bench.job_rate(1000.0, world, worst)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, worst, value))


def test_two_replicas_take_the_slowest_rank_and_count_all_units():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, value in res:
        assert worst == 2.0                  # every rank sees the slowest rank's time
        assert value == 1000.0 * 2 / 2.0     # units of both ranks over that time


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
