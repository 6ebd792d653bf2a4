"""The N > 1 path of the benchmark on CPU: two gloo ranks shard the independent
instances without overlap and report the whole-job rate over the slowest
rank's time (the max-reduction is the only collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.shard_seeds(rank, 16)
    tot_ms = 100.0 + 50.0 * rank            # rank 1 is the slower one
    value, t = bench.aggregate(tot_ms, units_per_rank=1000.0, steps=10, world=world, dist=dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    if rank == 0:
        out.put((value, t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    value, t, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 150.0                               # the slowest rank's time
    assert value == pytest.approx(2 * 1000.0 * 10 / 0.150)
    s0, s1 = set(gathered[0]), set(gathered[1])
    assert not (s0 & s1) and len(s0) == len(s1) == 16
