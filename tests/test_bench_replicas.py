"""The multi-GPU path of the benchmark is replicas only: every rank runs an
independent system and the job's value is all ranks' liftings over the
slowest rank's time. Two gloo ranks on the CPU check the reduction."""
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


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t, n = bench.aggregate(10.0 + 5.0 * rank, 1000 * (rank + 1), ws)
    out[rank] = (t, n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_sum_liftings():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 3000)


def test_one_rank_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(7.5, 42, 1) == (7.5, 42)
