"""bench.py's replica logic with two ranks on CPU (gloo): every rank renders its
own views, the whole-job value is the views of all ranks over the slowest
rank's time, and ranks draw distinct cameras.  No data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, local, w = bench.dist_env()
    assert (r, local, w) == (rank, rank, world)
    bench.init_dist(world, "gloo")
    bench.barrier()
    value, total, t_max = bench.aggregate(4 * (rank + 1), 1.0 + rank)
    out[rank] = (value, total, t_max, bench.rank_seed(rank))
    bench.barrier()
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_aggregate_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, total, t_max, seed = res[rank]
        assert total == 4 + 8
        assert t_max == 2.0
        assert value == pytest.approx(6.0)
    assert res[0][3] != res[1][3]


def test_single_process_aggregate_is_local():
    assert bench.aggregate(10, 2.0) == (5.0, 10.0, 2.0)
