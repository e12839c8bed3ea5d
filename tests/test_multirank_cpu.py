"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank runs its own
replica, the job's time is the slowest rank's and its work is the sum of the ranks'."""
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


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank           # rank 1 is slower
    e2e = 40.0 - 3.0 * rank          # rank 0 is slower end to end
    times, counts = bench.reduce_over_ranks(ms, e2e, 1000 * (rank + 1), 2000 * (rank + 1), dist)
    out.put((rank, times, counts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, times, counts in res:
        assert times == [15.0, 40.0]
        assert counts == [3000.0, 6000.0]
