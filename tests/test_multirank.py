"""CPU tests of the multi-rank (replica) path of the benchmark: two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r reports times (1 + r, 10 - r): the job is as slow as its slowest rank
    T, T2 = bench.max_over_ranks([1.0 + rank, 10.0 - rank], torch.device("cpu"))
    q.put((rank, T, T2, bench.replica_throughput(world, 1000, 4, T)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, T, T2, thr in out:
        assert T == 2.0 and T2 == 10.0  # element-wise maximum over both ranks
        assert thr == pytest.approx(world * 1000 * 4 / 2.0)
