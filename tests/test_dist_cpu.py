"""The multi-GPU reporting path of bench.py on CPU: two gloo ranks.

Operations are independent, so ranks share no data; the only collective is
the max over ranks of the step time, and the job rate is the units of all
ranks divided by the slowest rank's time (weak scaling).
"""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    out = bench.aggregate_ranks(ms, 65536, world, dist, "cpu")
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        ms, value = res[rank]
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(2 * 65536 / 0.015)


def test_single_rank_is_identity():
    import bench
    ms, value = bench.aggregate_ranks(20.0, 1000, 1)
    assert ms == 20.0 and value == pytest.approx(1000 / 0.02)
