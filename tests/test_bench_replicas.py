"""The replica aggregation of bench.py across ranks (gloo, world size 2, CPU):
value = sum of the ranks' steps / the slowest rank's time."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 1000.0 * (rank + 1)          # rank 1 is the slowest: 2000 ms
    ms, steps, value = bench.aggregate(ms_local, 3, dist, torch.device("cpu"))
    q.put((rank, ms, steps, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, steps, value in out:
        assert ms == 2000.0 and steps == 6.0
        assert abs(value - 3.0) < 1e-12      # 6 steps in 2 s


def test_single_rank_aggregation():
    import bench
    ms, steps, value = bench.aggregate(500.0, 2)
    assert (ms, steps) == (500.0, 2.0) and abs(value - 4.0) < 1e-12
