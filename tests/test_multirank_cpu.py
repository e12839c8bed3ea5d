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


def _sweep_rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1701_03784_gb300.batch import partition
    from workloads.sweep import sweep_params, sweep_particles
    import bench
    work = [sweep_particles(i) + sweep_params(i)["n_tri"] for i in range(16)]
    mine = partition(work, world)[rank]
    everyone = [None] * world
    dist.all_gather_object(everyone, mine)
    # the sweep's job figures: slowest rank's time, all ranks' particles
    times, counts = bench.reduce_over_ranks(1.0 + rank, 2.0, sum(work[i] for i in mine), len(mine),
                                            dist)
    out.put((rank, everyone, times, counts, sum(work)))
    dist.barrier()
    dist.destroy_process_group()


def test_sweep_instances_shard_over_two_gloo_ranks():
    """Each rank of a sharded sweep takes its own instances (no data exchanged): together
    the ranks hold every instance once, and the job's work is the sum of theirs."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sweep_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, everyone, times, counts, total in res:
        assert sorted(everyone[0] + everyone[1]) == list(range(16))
        assert not set(everyone[0]) & set(everyone[1])
        assert times == [2.0, 2.0] and counts == [float(total), 16.0]
