"""The benchmark's multi-GPU mode is N independent replicas (the sort does not
shard without exchanging keys). Its host logic — rank environment, max of the
per-rank times, whole-job value — runs here on CPU with two gloo processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
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
    try:
        r, w, local = bench.dist_env()
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (r, w, local, ms_max, bench.replica_value(w, 4, 1 << 20, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for rank in range(world):
        r, w, local, ms_max, value = res[rank]
        assert (r, w, local) == (rank, world, rank)
        assert ms_max == 15.0
        assert abs(value - world * 4 * (1 << 20) / 15e-3 / 1e9) < 1e-12


def test_single_process_value():
    import bench

    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert abs(bench.replica_value(1, 10, 1 << 28, 70.0) - 10 * (1 << 28) / 0.07 / 1e9) < 1e-9
