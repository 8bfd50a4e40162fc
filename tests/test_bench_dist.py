"""The multi-rank aggregation of bench.py (replicas; max over ranks) with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    ms_local = 100.0 if rank == 0 else 250.0  # rank 1 is the slowest
    value, ms_max = bench.whole_job_rate(ms_local, 5, world)
    q.put((rank, value, ms_max))
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in out:
        assert ms_max == pytest.approx(250.0)
        assert value == pytest.approx(5 * 2 / 0.25)
