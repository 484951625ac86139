"""The replica (N > 1) path of bench.py on CPU: two gloo ranks, each with its
own timed seconds and iteration count, report the slowest rank's time and
the iterations of both (value = all ranks' iterations / that time)."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs = [2.0, 3.5][rank]
    iters = [1000, 1200][rank]
    out[rank] = bench.aggregate_over_ranks(secs, iters)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (3.5, 2200.0)


def test_single_process_uses_its_own_numbers():
    import bench
    assert not dist.is_initialized()
    assert bench.aggregate_over_ranks(1.25, 40) == (1.25, 40.0)
