"""The bench's N > 1 path (replicas, one rank per GPU) on CPU ranks with gloo:
the timed region is the slowest rank's, the value is all ranks' units over it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_time = 1.0 + rank  # rank 1 is the slow one
    slowest = bench.max_over_ranks(my_time, dist, None)
    rate = bench.whole_job_rate(4587, world, 10, slowest)
    dist.barrier()
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_replicas_take_slowest_rank_world_size_2():
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
    for _, slowest, rate in res:
        assert slowest == pytest.approx(2.0)
        assert rate == pytest.approx(2 * 4587 * 10 / 2.0)
