"""The N > 1 bench path on CPU with gloo, world size 2: independent replicas
(distinct seeds), the job time is the slowest rank's, and the job rate counts
the units of every rank."""
import os
import socket

import pytest
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
    local_ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.job_rate(1000, 4, world, m)
    seeds = bench.replica_seeds(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    q.put((rank, m, rate, gathered))
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate, seeds in out:
        assert m == 150.0
        assert rate == pytest.approx(1000 * 4 * 2 / 0.150)
        assert seeds[0] != seeds[1]
