"""Host logic of bench.py's multi-rank runs, on CPU with two gloo ranks: every rank ends up with
the slowest rank's time, and the rank/world bookkeeping comes from the environment."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    got = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    out.put((r, w, local, got))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[0] for r in res] == [0, 1] and all(r[1] == world for r in res)
    assert all(r[3] == 15.0 for r in res)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
