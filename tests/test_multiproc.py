"""The multi-rank path of bench.py on the CPU: two gloo ranks (no GPU)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sh = bench.shard(rank, world)
    got = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    dist.barrier()
    q.put((rank, sh["seed"], sh["frame_begin"], got))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange_and_reduce_the_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [0, 1]           # distinct clips (seed = rank)
    assert len({r[2] for r in res}) == 1           # same output frames on every rank
    assert all(r[3] == 15.0 for r in res)          # every rank sees the slowest rank's time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard(0, 1)["seed"] == 0
